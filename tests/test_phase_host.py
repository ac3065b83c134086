"""The K-nearest path's spin-s transport phases (csrc/lens.cuh: pair_phase,
pair_phases_pm, and the mixed path's factorisation through the target,
holonomy32 + transported_phase) compiled for the host in FP64 and double-
float and compared with the oracle's phases (oracle.kriging.pair_phase and
pseudo_phase, pinned there by the addition theorems of the spin harmonics).

The kernels feed these functions the difference d = X_j - X_i and, per end,
(z, sin theta, cos phi, sin phi); the mixed path forms the member-member
phase as conj(Phi_i) Phi_j (1 + delta), Phi the phase from the displaced
target n' to a member and delta the spherical-excess correction in FP32."""
import numpy as np
import pytest

from oracle import kriging as kr
from tests import host_compile as hc

DRIVER = r"""
using namespace flints;
static double rd() { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtod(b, nullptr); }
static void pr(double x) { printf(" %a", x); }
template <class R> static typename Ops<R>::T in(double x) { return Ops<R>::from(x); }
// phase of the pair (a -> b) from positions a, b and both frames
template <class R, int S> static Cx<typename Ops<R>::T> phase(const double *a, const double *b, const double *fa,
                                                            const double *fb) {
    using T = typename Ops<R>::T;
    const T dx = in<R>(b[0] - a[0]), dy = in<R>(b[1] - a[1]), dz = in<R>(b[2] - a[2]);
    return pair_phase<R, S>(dx, dy, dz, in<R>(fa[0]), in<R>(fa[1]), in<R>(fa[2]), in<R>(fa[3]), in<R>(fb[0]),
                            in<R>(fb[1]), in<R>(fb[2]), in<R>(fb[3]));
}
int main() {
    char op[16];
    while (scanf("%15s", op) == 1) {
        // a point: x y z  then its frame: z sin(theta) cos(phi) sin(phi)
        double a[3], b[3], fa[4], fb[4];
        for (double &v : a) v = rd();
        for (double &v : fa) v = rd();
        for (double &v : b) v = rd();
        for (double &v : fb) v = rd();
        const std::string o(op);
        if (o == "p1" || o == "p2") {  // pair_phase in FP64 and in double-float
            const Cx<double> d = o == "p1" ? phase<double, 1>(a, b, fa, fb) : phase<double, 2>(a, b, fa, fb);
            const Cx<df> f = o == "p1" ? phase<df, 1>(a, b, fa, fb) : phase<df, 2>(a, b, fa, fb);
            pr(d.re); pr(d.im); pr(df_to(f.re)); pr(df_to(f.im));
        } else if (o == "pm") {  // both spin-2 phases at once, FP64 and double-float
            Cx<double> hp, hm;
            Cx<df> gp, gm;
            pair_phases_pm<double>(b[0] - a[0], b[1] - a[1], b[2] - a[2], fa[0], fa[1], fa[2], fa[3], fb[0], fb[1],
                                   fb[2], fb[3], hp, hm);
            pair_phases_pm<df>(in<df>(b[0] - a[0]), in<df>(b[1] - a[1]), in<df>(b[2] - a[2]), in<df>(fa[0]),
                               in<df>(fa[1]), in<df>(fa[2]), in<df>(fa[3]), in<df>(fb[0]), in<df>(fb[1]),
                               in<df>(fb[2]), in<df>(fb[3]), gp, gm);
            pr(hp.re); pr(hp.im); pr(hm.re); pr(hm.im);
            pr(df_to(gp.re)); pr(df_to(gp.im)); pr(df_to(gm.re)); pr(df_to(gm.im));
        } else if (o == "h1" || o == "h2") {  // through the target n' (then: n' and its frame)
            double n[3], fn[4];
            for (double &v : n) v = rd();
            for (double &v : fn) v = rd();
            const Cx<df> pa = o == "h1" ? phase<df, 1>(n, a, fn, fa) : phase<df, 2>(n, a, fn, fa);
            const Cx<df> pb = o == "h1" ? phase<df, 1>(n, b, fn, fb) : phase<df, 2>(n, b, fn, fb);
            // tangent-plane coordinates at n' (e_theta, e_phi) and squared chords
            const double et[3] = {fn[0] * fn[2], fn[0] * fn[3], -fn[1]}, ep[3] = {-fn[3], fn[2], 0.0};
            double ua = 0, va = 0, ub = 0, vb = 0, ta = 0, tb = 0, tab = 0;
            for (int k = 0; k < 3; ++k) {
                ua += (a[k] - n[k]) * et[k]; va += (a[k] - n[k]) * ep[k];
                ub += (b[k] - n[k]) * et[k]; vb += (b[k] - n[k]) * ep[k];
                ta += (a[k] - n[k]) * (a[k] - n[k]); tb += (b[k] - n[k]) * (b[k] - n[k]);
                tab += (b[k] - a[k]) * (b[k] - a[k]);
            }
            const Holo32 h = o == "h1" ? holonomy32<1>((float)ua, (float)va, (float)ub, (float)vb, (float)ta,
                                                       (float)tb, (float)tab)
                                       : holonomy32<2>((float)ua, (float)va, (float)ub, (float)vb, (float)ta,
                                                       (float)tb, (float)tab);
            const Cx<df> r = transported_phase(pa, pb, h);
            pr(df_to(r.re)); pr(df_to(r.im));
        } else return 3;
        printf("\n");
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    text = ("namespace flints {\nconstexpr unsigned FULL = 0xffffffffu;\n"
            + hc.cut("common.cuh", "struct df {", "// HEALPix RING geometry")
            + hc.cut("lens.cuh", "template <class T>\nstruct Cx {", "template <int K>\nstruct Shape", False)
            + hc.cut("lens.cuh", "template <class R, int S>\n__device__ __forceinline__ Cx<typename Ops<R>::T> "
                                 "pair_phase_uv(", "// Split left-looking Cholesky", False)
            + "\n}\n" + DRIVER)
    exe = hc.build(tmp_path_factory.mktemp("phase"), "phase_host", text)

    def call(lines):
        out = hc.run(exe, "\n".join(lines) + "\n")
        return np.array([[float.fromhex(t) for t in ln.split()] for ln in out.splitlines()])

    return call


def _frame(v):
    z = v[:, 2]
    s = np.sqrt(v[:, 0] ** 2 + v[:, 1] ** 2)
    return np.stack([z, s, v[:, 0] / s, v[:, 1] / s], axis=1)


def _pairs(rng, n, scale):
    """Random directions a (avoiding the poles) and b at a typical distance ``scale``."""
    a = rng.normal(size=(n, 3))
    a /= np.linalg.norm(a, axis=1)[:, None]
    a = a[np.abs(a[:, 2]) < 0.999]
    b = a + rng.normal(size=a.shape) * scale
    b /= np.linalg.norm(b, axis=1)[:, None]
    return a, b


def _line(op, *vecs):
    parts = []
    for v, f in vecs:
        parts.append(" ".join(x.hex() for x in np.concatenate([v, f])))
    return op + " " + " ".join(parts)


@pytest.mark.parametrize("scale", [3e-4, 1e-2, 0.3])
def test_pair_phases_match_the_oracle(scale, run):
    rng = np.random.default_rng(int(scale * 1e6))
    a, b = _pairs(rng, 1500, scale)
    fa, fb = _frame(a), _frame(b)
    for spin in (1, 2):
        got = run([_line(f"p{spin}", (a[k], fa[k]), (b[k], fb[k])) for k in range(len(a))])
        want = kr.pair_phase(a, b, spin)
        assert np.max(np.abs(got[:, 0] + 1j * got[:, 1] - want)) < 1e-14  # measured 1.1e-15
        # double-float: about 2^-44 relative per operation (measured 4.8e-14)
        assert np.max(np.abs(got[:, 2] + 1j * got[:, 3] - want)) < 5e-13
    pm = run([_line("pm", (a[k], fa[k]), (b[k], fb[k])) for k in range(len(a))])
    for off, tol in ((0, 1e-14), (4, 5e-13)):
        assert np.max(np.abs(pm[:, off] + 1j * pm[:, off + 1] - kr.pair_phase(a, b, 2))) < tol
        assert np.max(np.abs(pm[:, off + 2] + 1j * pm[:, off + 3] - kr.pseudo_phase(a, b, 2))) < tol


def test_coincident_points_have_no_rotation(run):
    a = np.array([[0.6, 0.0, 0.8]])
    f = _frame(a)
    for spin in (1, 2):
        got = run([_line(f"p{spin}", (a[0], f[0]), (a[0], f[0]))])[0]
        assert tuple(got) == (1.0, 0.0, 1.0, 0.0)
    pm = run([_line("pm", (a[0], f[0]), (a[0], f[0]))])[0]
    assert tuple(pm) == (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0)


@pytest.mark.parametrize("spin", [1, 2])
def test_phase_through_the_target_equals_the_direct_phase(spin, run):
    """Stencil geometry of the mixed path: n' the displaced target, a and b two
    members within a few pixels (Nside 4096: a pixel is 2.5e-4 rad)."""
    rng = np.random.default_rng(40 + spin)
    n, _ = _pairs(rng, 3000, 1e-3)
    a = n + rng.normal(size=n.shape) * 4e-4
    a /= np.linalg.norm(a, axis=1)[:, None]
    b = n + rng.normal(size=n.shape) * 4e-4
    b /= np.linalg.norm(b, axis=1)[:, None]
    fn, fa, fb = _frame(n), _frame(a), _frame(b)
    got = run([_line(f"h{spin}", (a[k], fa[k]), (b[k], fb[k]), (n[k], fn[k])) for k in range(len(n))])
    want = kr.pair_phase(a, b, spin)
    err = np.abs(got[:, 0] + 1j * got[:, 1] - want)
    assert np.max(err) < 1e-12, np.max(err)  # measured 1.3e-13
    # the excess correction matters: without it the error is the size of the excess (1e-7)
    direct = kr.pair_phase(n, a, spin).conj() * kr.pair_phase(n, b, spin)
    assert np.median(np.abs(direct - want)) > 1e3 * np.median(err)
