"""The tabulated-inverse path's integer face geometry (csrc/paper_geom.cuh, host-
device code) compiled for the host and checked against the oracle without a
GPU: face coordinates of every RING pixel and back, the ordered level-y
stencils of every coarse pixel, and the symmetry classes (the same partition
of the coarse pixels as the oracle's class representatives)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import faces as fc
from oracle import healpix as hp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEOM = os.path.join(ROOT, "paper_1003_4984_gb300", "csrc", "paper_geom.cuh")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include "paper_geom.cuh"
using namespace flints::paper;
int main(int argc, char **argv) {
    const int64_t N = atoll(argv[2]);
    if (argv[1][0] == 'x') {
        for (int64_t p = 0; p < 12 * N * N; ++p) {
            int64_t i, j;
            ring_and_pos(N, p, i, j);
            const Xyf x = ring2xyf(N, i, j);
            int64_t r, q;
            const int64_t back = xyf2ring(N, x.ix, x.iy, x.f, r, q);
            printf("%lld %lld %d %lld\n", (long long)x.ix, (long long)x.iy, x.f, (long long)back);
        }
        return 0;
    }
    const int k = 1 << (atoi(argv[3]) - 1);
    int32_t out[STENCIL_MAX];
    printf("%lld\n", (long long)slot_count(N));
    for (int64_t c = 0; c < 12 * N * N; ++c) {
        const int n = stencil_members(N, k, c, out);
        int64_t i, j;
        ring_and_pos(N, c, i, j);
        const int64_t s = slot_of(N, i, j);
        printf("%lld %lld %d", (long long)s, (long long)slot_rep(N, s), n);
        for (int m = 0; m < n; ++m) printf(" %d", out[m]);
        printf("\n");
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def geom_bin(tmp_path_factory):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is not available")
    d = tmp_path_factory.mktemp("geom")
    src = d / "geom_driver.cu"
    src.write_text(DRIVER)
    exe = d / "geom_driver"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.dirname(GEOM), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    return str(exe)


def _run(exe, *args):
    return subprocess.run([exe, *map(str, args)], check=True, capture_output=True, text=True).stdout.splitlines()


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 16])
def test_face_coordinates_match_the_oracle(geom_bin, N):
    out = np.array([list(map(int, line.split())) for line in _run(geom_bin, "x", N)], dtype=np.int64)
    ix, iy, f = fc.ring2xyf(N, np.arange(hp.npix(N)))
    assert np.array_equal(out[:, 0], ix) and np.array_equal(out[:, 1], iy) and np.array_equal(out[:, 2], f)
    assert np.array_equal(out[:, 3], np.arange(hp.npix(N)))


@pytest.mark.parametrize("n_c,y", [(1, 1), (2, 1), (4, 1), (8, 1), (2, 2), (4, 2)])
def test_ordered_stencils_and_classes_match_the_oracle(geom_bin, n_c, y):
    lines = _run(geom_bin, "s", n_c, y)
    nslot = int(lines[0])
    rows = [list(map(int, line.split())) for line in lines[1:]]
    cen = np.arange(hp.npix(n_c))
    ordered = fc.stencil_ordered(n_c << (y - 1), y, cen)
    for c, r in enumerate(rows):
        assert r[2] == ordered[c].size and r[3:] == list(ordered[c]), f"coarse pixel {c}"
    slot = np.array([r[0] for r in rows])
    rep_dev = np.array([r[1] for r in rows])
    rep = fc.class_representative(n_c, cen)[0]
    assert np.unique(slot).size == nslot == np.unique(rep).size
    assert np.array_equal(rep_dev, rep)  # the device's representative of each class is the oracle's
