"""The plan's correlation tables (csrc/xi_table.cu: the l-recurrence kernel and
the interval coefficients) and the lens kernels' table lookup (table_eval in
csrc/lens.cuh, FP64 and double-float) compiled for the host and compared with
the oracle's correlation functions and cubic Hermite tables.

The kernels run on the host one node (or interval) per loop step, with the
thread index as the loop variable.  The oracle's spin-0 sum is pinned against
scipy's Legendre polynomials and its spin-1/2 sums come from the Appendix B
Fourier route, independent of the recurrence the kernel runs."""
import numpy as np
import pytest

import workloads as wl
from oracle import xi
from tests import host_compile as hc

KERNEL_SHIM = r"""
#define __global__
struct Dim { unsigned x; };
static Dim blockIdx = {0}, blockDim = {1}, threadIdx = {0};
struct double2 { double x, y; };
struct float4 { float x, y, z, w; };
static inline float4 make_float4(float x, float y, float z, float w) { return {x, y, z, w}; }
template <class T> static inline T __ldg(const T *p) { return *p; }
"""

DRIVER = r"""
using namespace flints;
static double rd() { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtod(b, nullptr); }
int main() {
    int spin, lmax, has_bb, n, m;
    double t_max;
    while (scanf("%d %d %d %d", &spin, &lmax, &has_bb, &n) == 4) {
        t_max = rd();
        std::vector<double> cl(lmax + 1), bb(lmax + 1);
        for (double &v : cl) v = rd();
        if (has_bb) for (double &v : bb) v = rd();
        const double h = t_max / n;
        std::vector<double> f(n + 1), g(n + 1), fm(n + 1), gm(n + 1);
        for (int k = 0; k <= n; ++k) {  // one thread per node
            threadIdx.x = k;
            xi_table_kernel(spin, lmax, cl.data(), has_bb ? bb.data() : nullptr, h, n, f.data(), g.data(), fm.data(),
                            gm.data());
        }
        for (int k = 0; k <= n; ++k) printf("%a %a %a %a\n", f[k], g[k], fm[k], gm[k]);
        std::vector<Coef64> c64(n);
        std::vector<float4> c32(2 * n);
        const double xi0 = f[0];
        for (int k = 0; k < n; ++k) {  // one thread per interval
            threadIdx.x = k;
            table_coeffs_kernel(f.data(), g.data(), n, h, xi0, c64.data(), c32.data());
        }
        TableDev tab{};
        tab.c64 = c64.data();
        tab.c32 = c32.data();
        tab.t_max = t_max;
        tab.inv_h = n / t_max;
        tab.inv_h_hi = (float)tab.inv_h;
        tab.inv_h_lo = (float)(tab.inv_h - (double)tab.inv_h_hi);
        tab.n = n;
        if (scanf("%d", &m) != 1) return 2;
        for (int i = 0; i < m; ++i) {
            const double t = rd();
            printf("%a %a\n", table_eval<double>(tab, t), df_to(table_eval<df>(tab, df_from(t))));
        }
        printf("end\n");
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    text = (KERNEL_SHIM + "namespace flints {\nconstexpr unsigned FULL = 0xffffffffu;\n"
            + next(ln for ln in open(hc.CSRC + "/common.cuh") if ln.startswith("constexpr double PI"))
            + hc.cut("common.cuh", "struct df {", "// HEALPix RING geometry")
            + hc.cut("common.cuh", "struct alignas(32) Coef64", "struct LensArgs", False)
            + hc.cut("xi_table.cu", "__global__ void xi_table_kernel", "cudaError_t launch_xi_table(", False)
            + hc.cut("lens.cuh", "template <class R>\n__device__ __forceinline__ typename Ops<R>::T table_eval(",
                     "template <class R, int S>\n__device__ __forceinline__ Cx<typename Ops<R>::T> pair_phase_uv(",
                     False)
            + "\n}\n" + DRIVER)
    exe = hc.build(tmp_path_factory.mktemp("xitab"), "xi_host", text)

    def call(spin, cl, bb, t_max, n, ts):
        line = (f"{spin} {cl.size - 1} {0 if bb is None else 1} {n} {t_max.hex()} "
                + " ".join(x.hex() for x in cl) + ("" if bb is None else " " + " ".join(x.hex() for x in bb))
                + f" {ts.size} " + " ".join(x.hex() for x in ts))
        rows = [ln.split() for ln in hc.run(exe, line + "\n").splitlines()]
        assert rows[-1] == ["end"]
        nodes = np.array([[float.fromhex(v) for v in r] for r in rows[:n + 1]])
        ev = np.array([[float.fromhex(v) for v in r] for r in rows[n + 1:-1]])
        return nodes, ev

    return call


def _spectra():
    c1 = wl.C1
    cl1, _ = c1.cl()
    t1, n1 = xi.grid_rule(cl1, c1.K, c1.nside)
    cl2, _ = wl.C2.cl()
    t2, n2 = xi.grid_rule(cl2, wl.C2.K, wl.C2.nside)
    ee, bb = wl.C3.cl()
    t3, n3 = xi.grid_rule(ee + bb, wl.C3.K, wl.C3.nside)
    ell = np.arange(4097.0)
    cle = ell * (ell + 1) * wl.cl_phiphi(4096)  # deflection field: E_l = l(l+1) C^phiphi_l
    t4, n4 = xi.grid_rule(cle, 32, 4096)
    eb = wl.cl_ee(256, 150.0)
    t5, n5 = xi.grid_rule(eb + 0.4 * eb, 24, 128)
    return [("c1", 0, cl1, None, t1, n1), ("c2", 0, cl2, None, t2, n2), ("c3", 2, ee, bb, t3, n3),
            ("deflection", 1, cle, None, t4, n4), ("E and B", 2, eb, 0.4 * eb, t5, n5)]


@pytest.mark.parametrize("case", _spectra(), ids=lambda c: c[0])
def test_tables_and_lookups_match_the_oracle(case, run):
    name, spin, cl, bb, t_max, n = case
    ts = np.concatenate([np.random.default_rng(n).uniform(0, t_max, 3000), [0.0, t_max, t_max * (1 - 1e-16)],
                         np.arange(n) * (t_max / n)])
    nodes, ev = run(spin, cl, bb, t_max, n, ts)
    tk = np.arange(n + 1) * (t_max / n)
    if spin == 0:
        f, g = xi.xi0_direct(cl, tk, deriv=True)
        fm = gm = None
        x0 = float(xi.xi0_direct(cl, np.zeros(1))[0])
        table = xi.spin0_table(cl, t_max, n)[0]
    else:
        f, fm, g, gm = xi.xis_direct(spin, cl, bb, tk, deriv=True)
        x0 = float(f[0])
        table = (xi.spin1_tables if spin == 1 else xi.spin2_tables)(cl, bb, t_max, n)[0]
    # nodes, in units of xi(0) (slopes times the table domain).  Measured on the host:
    # values <= 1.0e-14; slopes <= 1.2e-10 (spin 1 at Nside 2048; spin 2 at Nside 4096:
    # 7.8e-12), the derivative recurrence gathering rounding over the l steps; xi- (a
    # plain three-term recurrence) values <= 2.0e-12, slopes <= 6.4e-11.  A slope error
    # e moves an interpolated value by at most e / n.
    assert np.max(np.abs(nodes[:, 0] - f)) <= 1e-13 * x0
    assert np.max(np.abs(nodes[:, 1] - g)) * t_max <= 1e-9 * x0
    if fm is not None:
        assert np.max(np.abs(nodes[:, 2] - fm)) <= 2e-11 * x0
        assert np.max(np.abs(nodes[:, 3] - gm)) * t_max <= 1e-9 * x0
    # lookups of xi/xi(0): the FP64 form against the oracle's Hermite table, the
    # double-float form within its stated ~1e-12
    want = table(ts)
    assert np.max(np.abs(ev[:, 0] - want)) <= 1e-13
    assert np.max(np.abs(ev[:, 1] - want)) <= 1e-12
    # and both against the direct sum (the grid rule's 1e-11 bound)
    direct = xi.xi0_direct(cl, ts) if spin == 0 else xi.xis_direct(spin, cl, bb, ts)[0]
    assert np.max(np.abs(ev[:, 0] - direct / x0)) <= 2e-11
