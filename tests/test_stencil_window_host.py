"""The K-nearest search's single-precision candidate window and pre-selection
keys (csrc/lens.cuh, phase B of the lens kernel: the per-ring block that turns
the displaced direction into a pixel window, and the FP32 squared-chord key of
a candidate) compiled for the host and checked against FP64 geometry, up to
Nside 16384, beyond the sizes the GPU parity tests run.

The kernel's stencil is exact only if (1) the rings searched, ring_above(z')
+- R_rings, hold every pixel of the search disc, (2) each ring's window, a
range computed in FP32 and widened by 1/32 pixel, holds every pixel of the
ring inside the disc, and (3) the FP32 keys are within 2^-17 of the squared
chords, so that a gap of 2^-16 between the K-th and (K+1)-th keys proves the
selected set.  The lens kernel's own code for (2) and (3) is cut out of
lens.cuh and run here on random directions (its window ends recorded and
compared with the same ends in long double: the source bounds their FP32
error by 0.02 pixel); the ring geometry and ring_above come from
common.cuh."""
import math

import numpy as np
import pytest

from tests import host_compile as hc

SHIM = r"""
#include <math.h>
struct double2 { double x, y; };
// sinpif (device: 1 ulp): sin(pi x) rounded to float
static inline float sinpif(float x) { return (float)std::sin(M_PI * (double)x); }
using std::floor; using std::fabs; using std::fmax;
"""

DRIVER = r"""
using namespace flints;
static double rd() { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtod(b, nullptr); }

// the window of ring i for direction P (the lens kernel's per-ring block; the test
// records the FP32 window ends lo, hi where the block computes them)
static float g_lo, g_hi;
static bool g_set;
static bool window(int64_t N, int64_t i, const PointA &P, double r2, RingRec &rec, int &cnt) {
    const double inv3N = 1.0 / (3.0 * (double)N), inv3N2 = inv3N / (double)N;
    struct { double r2; } a{r2};
    cnt = 0;
    g_set = false;
    {
__WINDOW__
    return cnt > 0;
}

static float key32(const RingRec &rr, int jj) {
__KEY__
    return k32;
}

int main() {
    long long N;
    int K, n;
    while (scanf("%lld %d %d", &N, &K, &n) == 3) {
        const double r = 1.25 * std::sqrt(K / 3.0) / (double)N, r2 = r * r;
        const int R_rings = (int)std::ceil(1.5 * r * (double)N) + 1;
        long long missed = 0, outside_band = 0, cand = 0, worst_extra = 0;
        double worst_key = 0.0, worst_end = 0.0;
        for (int t = 0; t < n; ++t) {
            double x = rd(), y = rd(), z = rd();
            PointA P{};
            P.x = x; P.y = y; P.z = z;
            P.s = std::sqrt(x * x + y * y);
            P.phi = std::atan2(y, x);
            P.zf = (float)P.z; P.sf = (float)P.s; P.phif = (float)P.phi;
            const int64_t ic = ring_above(N, z);
            for (int64_t i = 1; i <= 4 * N - 1; ++i) {
                const Ring rg = ring_of(N, i);
                // cheap reject: rings far in z cannot reach the disc
                if (std::fabs(rg.z - z) > 2 * r) continue;
                const bool band = i >= ic - R_rings && i <= ic - R_rings + 2 * R_rings + 1;
                RingRec rec{};
                int c = 0;
                const bool active = band && window(N, i, P, r2, rec, c);
                if (active && g_set) {  // the FP32 window ends against the same ends in long double
                    const long double dz = (long double)z - rg.z, ds = (long double)P.s - rg.s;
                    const long double qv = ((long double)r2 * 1.00001L - dz * dz - ds * ds) / (4.0L * P.s * rg.s);
                    const long double half = 2.0L * asinl(sqrtl(qv > 0 ? qv : 0));
                    const long double step = (long double)rg.n_in / (2.0L * 3.14159265358979323846264338327950288L);
                    const long double lo = ((long double)P.phi - half) * step - rg.f;
                    const long double hi = ((long double)P.phi + half) * step - rg.f;
                    const double e = (double)fmaxl(fabsl(g_lo - lo), fabsl(g_hi - hi));
                    if (e > worst_end) worst_end = e;
                }
                long long inside = 0;
                for (int j = 0; j < rg.n_in; ++j) {
                    const double ph = M_PI * ((double)j + rg.f) / (2.0 * (double)rg.nq);
                    const double cx = rg.s * std::cos(ph), cy = rg.s * std::sin(ph), cz = rg.z;
                    const double t2 = (x - cx) * (x - cx) + (y - cy) * (y - cy) + (z - cz) * (z - cz);
                    const bool in_disc = t2 < r2 * (1.0 - 1e-9);
                    bool in_win = false;
                    if (active) {
                        const int dj = ((j - rec.j0) % rg.n_in + rg.n_in) % rg.n_in;
                        in_win = dj < c;
                    }
                    if (in_disc) {
                        ++inside;
                        if (!band) ++outside_band;
                        else if (!in_win) ++missed;
                    }
                    if (in_win) {
                        ++cand;
                        const double k = (double)key32(rec, j);
                        const double rel = std::fabs(k - t2) / std::fmax(t2, 1e-300);
                        if (rel > worst_key) worst_key = rel;
                    }
                }
                if (active && c - inside > worst_extra) worst_extra = c - inside;
            }
        }
        printf("%lld %lld %lld %lld %a %a\n", missed, outside_band, cand, worst_extra, worst_key, worst_end);
    }
    return 0;
}
"""


def _between(src: str, start: str, stop: str) -> str:
    a = src.index(start)
    return src[a:src.index(stop, a)]


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    lens = open(hc.CSRC + "/lens.cuh").read()
    common = open(hc.CSRC + "/common.cuh").read()
    window = _between(lens, "const Ring rg = ring_of(N, i, inv3N, inv3N2);", "            // inclusive scan of counts")
    hi_line = "const float hi = (P.phif + half) * stepf - (float)rg.f;"
    assert hi_line in window
    window = window.replace(hi_line, hi_line + " g_lo = lo; g_hi = hi; g_set = true;")
    key = _between(lens, "int dj = jj - rr.jref;", "sm.u.cand.cpix[c] =")
    driver = DRIVER.replace("__WINDOW__", window).replace("__KEY__", key)
    text = (SHIM + "namespace flints {\nconstexpr unsigned FULL = 0xffffffffu;\n"
            + next(ln for ln in common.splitlines() if ln.startswith("constexpr double PI")) + "\n"
            + hc.cut("common.cuh", "struct Ring {", "// Launch description.")
            + _between(lens, "struct PointA {", "template <int K, int SPIN, class R>\nstruct WarpSmem")
            + "}\n" + driver)
    exe = hc.build(tmp_path_factory.mktemp("window"), "window_host", text)

    def call(N, K, v):
        line = f"{N} {K} {len(v)} " + " ".join(float(x).hex() for x in np.ravel(v))
        t = hc.run(exe, line + "\n").split()
        return int(t[0]), int(t[1]), int(t[2]), int(t[3]), float.fromhex(t[4]), float.fromhex(t[5])

    return call


def _directions(rng, n, N):
    """Random directions, half of them near the poles and the cap/belt edges where the
    window arithmetic changes form."""
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    zs = np.concatenate([1 - rng.uniform(0, 30 / N ** 2, n // 8), -1 + rng.uniform(0, 30 / N ** 2, n // 8),
                         2 / 3 + rng.uniform(-3, 3, n // 8) / N, -2 / 3 + rng.uniform(-3, 3, n // 8) / N])
    ph = rng.uniform(-math.pi, math.pi, zs.size)
    s = np.sqrt(1 - zs ** 2)
    return np.concatenate([v[: n - zs.size], np.stack([s * np.cos(ph), s * np.sin(ph), zs], 1)])


@pytest.mark.parametrize("N,K,n", [(16, 16, 400), (64, 48, 400), (1024, 32, 200), (4096, 32, 120),
                                   (8192, 48, 60), (16384, 32, 40)])
def test_windows_hold_the_disc_and_keys_are_accurate(N, K, n, run):
    missed, outside_band, cand, extra, worst_key, worst_end = run(N, K, _directions(np.random.default_rng(N + K), n, N))
    # the source's bound on the FP32 window ends, which the 1/32-pixel widening covers
    # (measured 0.0003 pixel at Nside 1024, 0.004 at 16384)
    assert worst_end < 0.02, worst_end
    assert missed == 0, "a pixel of the search disc fell outside its ring's window"
    assert outside_band == 0, "a pixel of the search disc lies on a ring that is not searched"
    assert cand > n * K  # windows hold at least the disc (about 1.25^2 K pixels)
    assert extra <= 4  # widened by 1/32 pixel, then floor and ceil: two beyond the disc per side
    assert worst_key < 2.0 ** -17, worst_key  # the pre-selection's stated bound (measured 2^-21)
