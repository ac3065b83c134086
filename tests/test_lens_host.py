"""The lens kernel's whole per-tile path (csrc/lens.cuh, process_tile:
displacement, stencil search, covariance assembly with transport phases,
bordered factorisation, value and variance, FP64 fallback) run on a host warp
of 32 lanes with the plan's own correlation tables (csrc/xi_table.cu's kernels
run on the host) and compared with the FP64 oracle element by element, for
spin 0, 1, 2 and the augmented spin-2 estimator, FP64 and mixed kernels, at
Nside 64 to 16384 -- beyond the GPU tests' largest sky.

The map is a band-limited realisation synthesised by the oracle exactly on
the rings the stencils reach (every other pixel NaN, so a read outside them
shows); deflections are per-pixel Gaussian.  Tolerances are those of the GPU
parity tests: max |kernel - oracle| / sigma_map <= 1e-9 (FP64) and 1e-6
(mixed), variances in units of xi(0).  Measured: FP64 8e-11 at most (spin 2,
Nside 4096), mixed 4.5e-9 at most; no point needs the FP64 fallback."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
from oracle import kriging as kr
from oracle import sht
from oracle import xi
from tests import host_compile as hc

KERNEL_SHIM = r"""
#include <sys/mman.h>
#define __global__
struct Dim { unsigned x; };
static Dim blockIdx = {0}, blockDim = {1}, threadIdx = {0};
static inline float4 make_float4(float x, float y, float z, float w) { return {x, y, z, w}; }
"""

DRIVER = r"""
using namespace flints;
static double rd() { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtod(b, nullptr); }

template <int K, int SPIN, int MIXED> static void lens(long long N, int lmax, bool has_bb, long long first,
                                                       int count, const char *map_path, long long nmap) {
    std::vector<double> cl(lmax + 1), bb(lmax + 1), defl(2 * count);
    for (double &v : cl) v = rd();
    if (has_bb) for (double &v : bb) v = rd();
    for (double &v : defl) v = rd();
    const int tspin = SPIN == SPIN2_AUG ? 2 : SPIN;
    const TableGrid tg = table_grid(N, K, lmax, cl.data(), (tspin != 0 && has_bb) ? bb.data() : nullptr);
    const int n = tg.n;
    std::vector<double> f(n + 1), g(n + 1), fm(n + 1), gm(n + 1);
    for (int k = 0; k <= n; ++k) {  // xi nodes: one thread per node
        threadIdx.x = k;
        xi_table_kernel(tspin, lmax, cl.data(), has_bb ? bb.data() : nullptr, tg.h, n, f.data(), g.data(), fm.data(),
                        gm.data());
    }
    const double xi0 = f[0];
    std::vector<Coef64> c64(n), cm64(n);
    std::vector<float4> c32(2 * n), cm32(2 * n);
    for (int k = 0; k < n; ++k) {  // interval coefficients: one thread per interval
        threadIdx.x = k;
        table_coeffs_kernel(f.data(), g.data(), n, tg.h, xi0, c64.data(), c32.data());
        if (tspin != 0) table_coeffs_kernel(fm.data(), gm.data(), n, tg.h, xi0, cm64.data(), cm32.data());
    }
    // the whole map, reserved but unbacked: only the synthesised rings are written (NaN elsewhere)
    const int comp = SPIN == 0 ? 1 : 2;
    const size_t map_bytes = (size_t)12 * N * N * comp * sizeof(double);
    double *map = static_cast<double *>(
        mmap(nullptr, map_bytes, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS | MAP_NORESERVE, -1, 0));
    if (map == MAP_FAILED) exit(4);
    FILE *fp = fopen(map_path, "rb");
    std::vector<int64_t> pix(nmap);
    std::vector<double> vals((size_t)nmap * comp);
    if (fread(pix.data(), 8, nmap, fp) != (size_t)nmap || fread(vals.data(), 8, nmap * comp, fp) != (size_t)nmap * comp)
        exit(5);
    fclose(fp);
    int64_t lo = pix[0], hi = pix[0];
    for (int64_t p : pix) { lo = p < lo ? p : lo; hi = p > hi ? p : hi; }
    for (int64_t p = lo; p <= hi; ++p)
        for (int c = 0; c < comp; ++c) map[p * comp + c] = std::nan("");
    for (long long i = 0; i < nmap; ++i)
        for (int c = 0; c < comp; ++c) map[pix[i] * comp + c] = vals[i * comp + c];
    std::vector<double> out((size_t)count * comp), var(count);
    std::vector<uint8_t> status(count);
    LensArgs a{};
    a.nside = N;
    a.first = first;
    a.count = count;
    a.map = map;
    a.defl = defl.data();
    a.out = out.data();
    a.var = var.data();
    a.status = status.data();
    a.tab.c64 = c64.data();
    a.tab.c32 = c32.data();
    a.tab.t_max = tg.t_max;
    a.tab.inv_h = tg.inv_h;
    a.tab.inv_h_hi = (float)tg.inv_h;
    a.tab.inv_h_lo = (float)(tg.inv_h - (double)a.tab.inv_h_hi);
    a.tab.n = n;
    a.tabm = a.tab;
    a.tabm.c64 = cm64.data();
    a.tabm.c32 = cm32.data();
    a.xi0 = xi0;
    a.r2 = tg.r2;
    const int tile_pts = MAX_TILE_POINTS;
    const size_t bytes = warp_smem_bytes<K, SPIN, MIXED>();
    unsigned char *smem = static_cast<unsigned char *>(std::aligned_alloc(16, (bytes + 15) / 16 * 16));
    for (int64_t tile = 0; tile * tile_pts < count; ++tile)
        run_warp([&](int lane) {
            Counters ctr;
            process_tile<K, SPIN, MIXED>(a, tg.R_rings, tile, tile_pts, smem, lane, ctr);
        });
    std::free(smem);
    munmap(map, map_bytes);
    printf("%a\n", xi0);
    for (int p = 0; p < count; ++p) {
        printf("%d %a %a", (int)status[p], out[(size_t)p * comp], var[p]);
        if (comp == 2) printf(" %a", out[(size_t)p * comp + 1]);
        printf("\n");
    }
}

int main() {
    int spin, K, mixed, lmax, has_bb, count;
    long long N, first, nmap;
    char path[512];
    while (scanf("%d %d %d %lld %d %d %lld %d %511s %lld", &spin, &K, &mixed, &N, &lmax, &has_bb, &first, &count,
                 path, &nmap) == 10) {
        const int key = spin * 1000 + K * 10 + mixed;
        switch (key) {
#define CASE(S, KK, M) case S * 1000 + KK * 10 + M: lens<KK, S, M>(N, lmax, has_bb, first, count, path, nmap); break;
            CASE(0, 16, 0) CASE(0, 16, 1) CASE(0, 32, 0) CASE(0, 32, 1) CASE(2, 32, 0) CASE(2, 32, 1)
            CASE(2, 48, 0) CASE(2, 48, 1) CASE(1, 32, 0) CASE(1, 32, 1) CASE(3, 24, 0) CASE(3, 24, 1)
            CASE(2, 16, 0) CASE(2, 16, 1)
#undef CASE
            default: return 3;
        }
    }
    return 0;
}
"""


def _build(d, sanitize=None):
    api = open(hc.CSRC + "/api.cu").read()
    a = api.index("TableGrid table_grid(")
    depth, k = 0, api.index("{", a)
    while True:
        depth += {"{": 1, "}": -1}.get(api[k], 0)
        if depth == 0:
            break
        k += 1
    text = (hc.LENS_SHIM + KERNEL_SHIM + '#include "' + hc.ROOT + '/include/flints.h"\nnamespace flints {\n'
            + hc.cut("common.cuh", "constexpr unsigned FULL", "// Host-side launchers (lens_spin0.cu", False)
            + api[a:k + 1] + "\n"
            + hc.cut("xi_table.cu", "__global__ void xi_table_kernel", "cudaError_t launch_xi_table(", False)
            + hc.cut("lens.cuh", "template <class T>\nstruct Cx {", "// Single-launch kernel", False)
            + "\n}\n" + DRIVER)
    exe = hc.build(d, "lens_host", text, warp="threads", sanitize=sanitize)

    def call(spin, K, mixed, N, cl, bb, first, defl, pix, vals):
        path = os.path.join(str(d), "map.bin")
        with open(path, "wb") as f:
            f.write(np.ascontiguousarray(pix, dtype=np.int64).tobytes())
            f.write(np.ascontiguousarray(vals, dtype=np.float64).tobytes())
        line = (f"{spin} {K} {mixed} {N} {cl.size - 1} {0 if bb is None else 1} {first} {len(defl)} {path} "
                f"{len(pix)} " + " ".join(x.hex() for x in cl)
                + ("" if bb is None else " " + " ".join(x.hex() for x in bb))
                + " " + " ".join(float(x).hex() for x in np.ravel(defl)))
        rows = [ln.split() for ln in hc.run(exe, line + "\n").splitlines()]
        x0 = float.fromhex(rows[0][0])
        status = np.array([int(r[0]) for r in rows[1:]])
        var = np.array([float.fromhex(r[2]) for r in rows[1:]])
        out = np.array([float.fromhex(r[1]) for r in rows[1:]])
        if spin != 0:
            out = out + 1j * np.array([float.fromhex(r[3]) for r in rows[1:]])
        return x0, status, out, var

    return call


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    return _build(tmp_path_factory.mktemp("lens"))


def _inputs(spin, N, lmax, ld, first, count, seed):
    """Spectra, deflections and the map synthesised on the rings the stencils reach."""
    if spin == 1:  # a deflection field d = grad phi: E_l = l(l+1) C^phiphi
        ell = np.arange(lmax + 1.0)
        cl, bb = ell * (ell + 1) * wl.cl_phiphi(lmax), None
        alm = wl.draw_alm(wl.cl_phiphi(lmax), seed)
    else:
        cl = wl.cl_tt(lmax, ld) if spin == 0 else wl.cl_ee(lmax, ld)
        bb = 0.3 * cl if spin == 3 else None
        alm = wl.draw_alm(cl, seed)
    blm = wl.draw_alm(bb, seed + 1) if bb is not None else None
    defl = wl.random_deflection(count, seed + 2) * max(1.0, 4096 / N)
    tv = kr.displace(N, np.arange(first, first + count), defl)
    idx, _ = kr.knn(N, tv, 56)  # the stencils and their near-ties
    r = hp.pix2ring(N, idx.ravel())[0]
    rings = np.arange(max(1, r.min() - 1), min(4 * N - 1, r.max() + 1) + 1)
    if spin == 1:
        pix, v = sht.synth_rings(N, rings, lmax, alm, gradient=True)
    else:
        pix, v = sht.synth_rings(N, rings, lmax, alm, spin=0 if spin == 0 else 2, blm=blm)
        if spin != 0:
            v = np.stack([v.real, v.imag], axis=1)
    return cl, bb, defl, pix, v


class _Band:
    def __init__(self, pix, vals):
        o = np.argsort(pix)
        self.pix, self.vals = pix[o], vals[o]

    def __getitem__(self, key):
        idx, comp = key if isinstance(key, tuple) else (key, None)
        v = self.vals[np.searchsorted(self.pix, idx)]
        return v if comp is None else v[..., comp]


# (spin, Nside, K, lmax, damping, first target): spin 3 is the augmented spin-2 estimator
CASES = [(0, 64, 16, 128, 100.0, 20_000), (0, 2048, 32, 4096, 2500.0, 25_000_000),
         (2, 4096, 32, 4096, 2500.0, 8_390_000), (2, 1024, 48, 2048, 1250.0, 6_000_000),
         (1, 2048, 32, 2048, 1250.0, 40_000_000), (3, 512, 24, 1024, 625.0, 1_500_000),
         (0, 16384, 32, 2048, 1250.0, 3_200_000_000), (2, 16384, 16, 2048, 1250.0, 1_610_000_000)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"spin{c[0]}-nside{c[1]}-K{c[2]}")
def test_lensed_values_and_variances_match_the_oracle(case, run):
    _check_case(case, run, 32)


def test_largest_skies_under_the_sanitizers(tmp_path_factory):
    """The whole per-tile path at Nside 16384 (pixel indices past 2^31), spin 0 and
    spin 2, FP64 and mixed, built with the address sanitizer and the signed-overflow
    and bounds checks: no index computation overflows and no access leaves its array,
    and the results still match the oracle."""
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    run = _build(tmp_path_factory.mktemp("lens_san"), sanitize="address")
    for case in CASES[-2:]:
        _check_case(case, run, 16)


def _check_case(case, run, count):
    spin, N, K, lmax, ld, first = case
    cl, bb, defl, pix, vals = _inputs(spin, N, lmax, ld, first, count, seed=N + K + spin)
    weight = np.abs(cl) + (np.abs(bb) if bb is not None else 0.0)
    t_max, n = xi.grid_rule(weight, K, N)
    if spin == 0:
        tab, x0 = xi.spin0_table(cl, t_max, n)
        tm = None
    else:
        tab, tm, x0 = (xi.spin1_tables if spin == 1 else xi.spin2_tables)(cl, bb, t_max, n)
    ref = kr.lens(N, K, 1 if spin == 1 else (0 if spin == 0 else 2), _Band(pix, vals), defl,
                  np.arange(first, first + count), tab, x0, f_minus=tm if spin == 3 else None)
    sigma = float(np.sqrt(np.mean(vals ** 2) * (1 if vals.ndim == 1 else 2)))  # rms of the field (|P| for spin s)
    for mixed, tol in ((0, 1e-9), (1, 1e-6)):
        kx0, status, out, var = run(spin, K, mixed, N, cl, bb, first, defl, pix, vals)
        assert abs(kx0 - x0) <= 1e-13 * x0
        assert np.all(status & 8 == 0), status  # no FLINTS_ST_FAILED
        assert np.max(np.abs(out - ref.value)) / sigma <= tol, (mixed, np.max(np.abs(out - ref.value)) / sigma)
        assert np.max(np.abs(var - ref.variance)) / x0 <= tol, (mixed, np.max(np.abs(var - ref.variance)) / x0)
