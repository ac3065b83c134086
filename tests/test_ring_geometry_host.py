"""The K-nearest path's HEALPix RING geometry (csrc/common.cuh: ring_of,
pix_ring, ring_above) compiled for the host and checked against the oracle's
RING geometry without a GPU: ring records (first pixel, pixel count, phase
offset exact; z and sin(theta) within a few ulps, the device multiplying by
reciprocals where the oracle divides), pixel-to-ring decomposition of every
pixel at small Nside and of sampled pixels up to Nside 8192, and the ring
bracketing of arbitrary z.

The section between the RING geometry banner and the launch description is
compiled as host C++ (double sqrt and floor are correctly rounded on both)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import healpix as hp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMMON = os.path.join(ROOT, "paper_1003_4984_gb300", "csrc", "common.cuh")

DRIVER = r"""
int main() {
    char op[16];
    long long N;
    while (scanf("%15s %lld", op, &N) == 2) {
        if (op[0] == 'r') {  // every ring of Nside N
            for (long long i = 1; i <= 4 * N - 1; ++i) {
                const Ring r = ring_of(N, i);
                printf("%a %a %lld %d %d %a\n", r.z, r.s, (long long)r.first, r.n_in, r.nq, r.f);
            }
        } else if (op[0] == 'p') {  // count, then pixels
            long long n, p;
            if (scanf("%lld", &n) != 1) return 2;
            for (long long k = 0; k < n; ++k) {
                if (scanf("%lld", &p) != 1) return 2;
                int64_t ring, j;
                pix_ring(N, p, ring, j);
                printf("%lld %lld\n", (long long)ring, (long long)j);
            }
        } else if (op[0] == 'a') {  // count, then z values
            long long n;
            char b[64];
            if (scanf("%lld", &n) != 1) return 2;
            for (long long k = 0; k < n; ++k) {
                if (scanf("%63s", b) != 1) return 2;
                printf("%lld\n", (long long)ring_above(N, strtod(b, nullptr)));
            }
        } else return 3;
        printf("end\n");
    }
    return 0;
}
"""


def _section() -> str:
    src = open(COMMON).read()
    a = src.index("struct Ring {")
    b = src.index("// Launch description.")
    body = src[a:b]
    body = body[:body.rindex("// ----")]
    return body.replace("__device__ __forceinline__", "static inline")


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("ringgeom")
    src = d / "ring_host.cpp"
    src.write_text("#include <cmath>\n#include <cstdint>\n#include <cstdio>\n#include <cstdlib>\n"
                   "using std::sqrt; using std::floor; using std::fabs; using std::fmax;\n"
                   + _section() + DRIVER)
    exe = d / "ring_host"
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

    def call(text):
        p = subprocess.run([str(exe)], input=text, capture_output=True, text=True)
        assert p.returncode == 0, p.stderr
        blocks, cur = [], []
        for ln in p.stdout.splitlines():
            if ln == "end":
                blocks.append(cur)
                cur = []
            else:
                cur.append(ln.split())
        return blocks

    return call


def _ulps(a, b):
    return np.abs(a - b) / np.spacing(np.maximum(np.abs(a), np.abs(b)))


@pytest.mark.parametrize("N", [1, 2, 3, 16, 64, 1024, 4096, 8192])
def test_ring_records_match_the_oracle(N, run):
    rows = run(f"r {N}\n")[0]
    i = np.arange(1, 4 * N)
    first, n_in, z, s, f, nq = hp.ring_info(N, i)
    dz = np.array([float.fromhex(r[0]) for r in rows])
    ds = np.array([float.fromhex(r[1]) for r in rows])
    assert np.array_equal([int(r[2]) for r in rows], first)
    assert np.array_equal([int(r[3]) for r in rows], n_in)
    assert np.array_equal([int(r[4]) for r in rows], nq)
    assert np.array_equal([float.fromhex(r[5]) for r in rows], f)
    assert np.max(_ulps(dz, z)) <= 4 and np.max(_ulps(ds, s)) <= 4
    assert np.max(np.abs(dz * dz + ds * ds - 1.0)) < 1e-15
    assert np.all(np.diff(dz) < 0)  # rings strictly ordered from north to south
    assert np.array_equal(dz, -dz[::-1])  # the south mirrors the north exactly


@pytest.mark.parametrize("N", [1, 2, 5, 32, 128])
def test_every_pixel_decomposes_into_ring_and_position(N, run):
    pix = np.arange(hp.npix(N))
    rows = run(f"p {N} {pix.size} " + " ".join(map(str, pix)) + "\n")[0]
    ring, j = hp.pix2ring(N, pix)
    assert np.array_equal([int(r[0]) for r in rows], ring)
    assert np.array_equal([int(r[1]) for r in rows], j)


@pytest.mark.parametrize("N", [2048, 4096, 8192])
def test_sampled_pixels_at_large_nside(N, run):
    rng = np.random.default_rng(N)
    npix = hp.npix(N)
    ncap = 2 * N * (N - 1)
    edges = [0, 1, 2, 3, 4, ncap - 1, ncap, ncap + 1, npix - ncap - 1, npix - ncap, npix - 1, npix - 2]
    pix = np.unique(np.concatenate([rng.integers(0, npix, 20000), edges])).astype(np.int64)
    rows = run(f"p {N} {pix.size} " + " ".join(map(str, pix)) + "\n")[0]
    ring, j = hp.pix2ring(N, pix)
    assert np.array_equal([int(r[0]) for r in rows], ring)
    assert np.array_equal([int(r[1]) for r in rows], j)


@pytest.mark.parametrize("N", [1, 4, 64, 4096])
def test_ring_above_brackets_z(N, run):
    rng = np.random.default_rng(7 + N)
    rz = run(f"r {N}\n")[0]
    ringz = np.array([float.fromhex(r[0]) for r in rz])
    z = np.concatenate([rng.uniform(-1, 1, 20000), [1.0, -1.0, 0.0, 2.0 / 3.0, -2.0 / 3.0],
                        ringz, np.nextafter(ringz, 2.0), np.nextafter(ringz, -2.0)])
    got = np.array([int(r[0]) for r in run(f"a {N} {z.size} " + " ".join(x.hex() for x in z) + "\n")[0]])
    # the defining property with the device's own ring latitudes: z(i) >= z > z(i + 1)
    zi = np.concatenate([[np.inf], ringz, [-np.inf]])  # index 0: above the north pole
    assert np.all(zi[got] >= z) and np.all(z > zi[got + 1])
    # and the oracle's answer wherever z is not within a few ulps of a ring latitude
    oz = np.sort(hp.ring_info(N, np.arange(1, 4 * N))[2])
    k = np.clip(np.searchsorted(oz, z), 1, oz.size - 1)
    far = np.minimum(np.abs(z - oz[k - 1]), np.abs(z - oz[k])) > 1e-13
    assert np.array_equal(got[far], hp.ring_above(N, z[far]))
