"""The tabulated-inverse route's target placement (csrc/paper.cu: pix2vec,
ang2pix and target_of, the FP64 code that decides each target's coarse pixel
and with it the stencil) compiled for the host and compared with the
oracle: RING point location against the oracle's inverse face projection
(oracle.faces.vec2pix, an independent formulation), and the displaced target
against oracle.kriging.displace on both branches of the step (the Taylor
series below |d| = 1/16 and sincos above).

Host stand-ins: sincospi(x) is sin/cos of pi x; sincos and atan2 are the C
library's (the device's are within an ulp or two of the same values)."""
import math

import numpy as np
import pytest

from oracle import faces as fc
from oracle import healpix as hp
from oracle import kriging as kr
from tests import host_compile as hc

SHIM = r"""
#define __host__
#define __device__
#define __forceinline__ inline
#define __global__
struct double2 { double x, y; };
struct float2 { float x, y; };
struct float4 { float x, y, z, w; };
template <class T> static inline T __ldg(const T *p) { return *p; }
static inline void sincospi(double x, double *s, double *c) { *s = std::sin(M_PI * x); *c = std::cos(M_PI * x); }
static inline double __longlong_as_double(long long v) { double d; std::memcpy(&d, &v, 8); return d; }
using std::atan2; using std::floor; using std::fabs; using std::isfinite;
"""

DRIVER = r"""
using namespace flints;
using namespace flints::paper;
static double rd() { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtod(b, nullptr); }
int main() {
    char op[8];
    long long N;
    while (scanf("%7s %lld", op, &N) == 2) {
        const std::string o(op);
        long long n;
        if (scanf("%lld", &n) != 1) return 2;
        if (o == "loc") {  // n unit vectors -> RING pixel at Nside N
            for (long long k = 0; k < n; ++k) {
                const double x = rd(), y = rd(), z = rd();
                printf("%lld\n", (long long)ang2pix(N, x, y, z));
            }
        } else if (o == "ctr") {  // pixel centres of pixels 0..n-1 located back
            for (long long p = 0; p < n; ++p) {
                double x, y, z;
                pix2vec(N, p, x, y, z);
                printf("%a %a %a %lld\n", x, y, z, (long long)ang2pix(N, x, y, z));
            }
        } else if (o == "tgt") {  // coarse Nside, first pixel, then n deflections
            long long Nc, first;
            if (scanf("%lld %lld", &Nc, &first) != 2) return 2;
            std::vector<double> defl(2 * n);
            for (double &v : defl) v = rd();
            ApplyArgs a{};
            a.N = N;
            a.Nc = Nc;
            a.first = first;
            a.count = n;
            a.nside_tgt = 0;
            a.defl = defl.data();
            for (long long p = 0; p < n; ++p) {
                double x = 0, y = 0, z = 0;
                int64_t c = -1;
                target_of(a, p, x, y, z, c);
                printf("%a %a %a %lld\n", x, y, z, (long long)c);
            }
        } else return 3;
        printf("end\n");
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    common = open(hc.CSRC + "/common.cuh").read()
    paper = open(hc.CSRC + "/paper.cu").read()

    def block(src, start):
        a = src.index(start)
        depth, k = 0, src.index("{", a)
        while True:
            depth += {"{": 1, "}": -1}.get(src[k], 0)
            if depth == 0:
                break
            k += 1
        return src[a:k + 1] + (";" if src[k + 1:k + 2] == ";" else "")

    geom = open(hc.CSRC + "/paper_geom.cuh").read().replace("#pragma once", "")
    text = (SHIM + "namespace flints {\n"
            + next(ln for ln in common.splitlines() if ln.startswith("constexpr double PI")) + "\n"
            + hc.cut("common.cuh", "struct Ring {", "// Launch description.")
            + hc.cut("common.cuh", "struct alignas(32) Coef64", "struct LensArgs", False)
            + "}\n" + geom + "namespace flints {\nnamespace paper {\n"
            + block(paper, "struct ApplyArgs {") + "\n"
            + block(paper, "__device__ __forceinline__ void pix2vec(") + "\n"
            + block(paper, "__device__ __forceinline__ int64_t ang2pix(") + "\n"
            + block(paper, "__device__ __forceinline__ void target_of(") + "\n}\n}\n" + DRIVER)
    exe = hc.build(tmp_path_factory.mktemp("locate"), "locate_host", text)

    def call(text):
        out = hc.run(exe, text)
        blocks, cur = [], []
        for ln in out.splitlines():
            if ln == "end":
                blocks.append(cur)
                cur = []
            else:
                cur.append(ln.split())
        return blocks

    return call


def _h(a):
    return " ".join(float(x).hex() for x in np.ravel(a))


@pytest.mark.parametrize("N", [1, 2, 3, 8, 64, 1024, 4096])
def test_point_location_matches_the_oracle(N, run):
    rng = np.random.default_rng(N)
    v = rng.normal(size=(40000, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    # and directions on the special latitudes |z| = 2/3, next to the poles and just
    # below phi = 2 pi (points exactly on a pixel edge or vertex, where either side is
    # a valid answer, are left out)
    zs = np.array([2 / 3, -2 / 3, 1 - 1e-12, -1 + 1e-12, 0.0])
    ph = rng.uniform(0, 2 * math.pi, zs.size)
    extra = np.stack([np.sqrt(1 - zs ** 2) * np.cos(ph), np.sqrt(1 - zs ** 2) * np.sin(ph), zs], 1)
    v = np.concatenate([v, extra, [[0.6, -1e-17, 0.8]]])
    got = np.array([int(r[0]) for r in run(f"loc {N} {len(v)} {_h(v)}\n")[0]])
    want = fc.vec2pix(N, v)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]


@pytest.mark.parametrize("N", [1, 2, 16, 64])
def test_pixel_centres_locate_to_themselves(N, run):
    rows = run(f"ctr {N} {hp.npix(N)}\n")[0]
    xyz = np.array([[float.fromhex(t) for t in r[:3]] for r in rows])
    assert np.array_equal([int(r[3]) for r in rows], np.arange(hp.npix(N)))
    assert np.max(np.abs(xyz - hp.pix2vec(N, np.arange(hp.npix(N))))) < 1e-15  # a few ulps


@pytest.mark.parametrize("N,Nc,first", [(64, 32, 0), (4096, 4096, 100_000_000), (4096, 2048, 201_000_000),
                                        (2048, 1024, 5)])
def test_displaced_targets_match_the_oracle(N, Nc, first, run):
    rng = np.random.default_rng(first + N)
    n = 4000
    # lensing-sized steps (Taylor branch) and steps around and above |d| = 1/16 (sincos)
    mag = np.concatenate([rng.uniform(0, 1e-3, n // 2), rng.uniform(0.05, 0.08, n // 4),
                          rng.uniform(0.1, 1.5, n - n // 2 - n // 4)])
    ang = rng.uniform(0, 2 * math.pi, n)
    d = np.stack([mag * np.cos(ang), mag * np.sin(ang)], 1)
    d[0] = 0.0
    d[1] = [1.0 / 16 - 1e-12, 0.0]
    d[2] = [1.0 / 16 + 1e-12, 0.0]
    first = min(first, hp.npix(N) - n)
    rows = run(f"tgt {N} {n} {Nc} {first} {_h(d)}\n")[0]
    got = np.array([[float.fromhex(t) for t in r[:3]] for r in rows])
    pix = np.arange(first, first + n)
    want = kr.displace(N, pix, d)
    assert np.max(np.abs(got - want)) < 2e-15
    assert np.array_equal([int(r[3]) for r in rows], fc.vec2pix(Nc, got))
