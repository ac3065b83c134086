"""The lens kernel's whole K-nearest stencil search (csrc/lens.cuh,
process_tile in stencil mode: displacement, ring windows, FP32 pre-selection,
FP64 decision, near-tie handling and the warp sorts) run on a host warp of 32
threads, for the FP64 and the mixed kernels, and compared with the oracle's
exact K-nearest search at Nside up to 16384 -- sizes and stencil sizes the
GPU parity tests do not reach -- on both polar caps, the cap/belt edges and
the belt.  Where the K-th and (K+1)-th neighbours tie to 1e-11, any valid
K-nearest set is accepted (the same rule as the GPU stencil test).

The lens kernel's device code is compiled for the host as a whole (host
stand-ins: tests/host_compile.py); the plan's grid rule (table_grid) gives
the search disc."""
import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
from oracle import kriging as kr
from tests import host_compile as hc



DRIVER = r"""
using namespace flints;
static double rd() { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtod(b, nullptr); }

static double g_r2_scale = 1.0;  // test knob: shrink the search disc to reach its window check

template <int K, int MIXED> static void stencil(long long N, long long first, int count) {
    std::vector<double> defl(2 * count);
    for (double &v : defl) v = rd();
    const double cl[3] = {0.0, 0.0, 1.0};
    TableGrid tg = table_grid(N, K, 2, cl, nullptr);  // the plan's search disc
    tg.r2 *= g_r2_scale;
    std::vector<int64_t> st((size_t)count * K, -7);
    std::vector<uint8_t> status(count, 255);
    LensArgs a{};
    a.nside = N;
    a.first = first;
    a.count = count;
    a.defl = defl.data();
    a.stencil = st.data();
    a.status = status.data();
    a.r2 = tg.r2;
    a.xi0 = 1.0;
    const int tile_pts = MAX_TILE_POINTS;
    const size_t bytes = warp_smem_bytes<K, 0, MIXED>();
    unsigned char *smem = static_cast<unsigned char *>(std::aligned_alloc(16, (bytes + 15) / 16 * 16));
    const int64_t ntiles = (count + tile_pts - 1) / tile_pts;
    for (int64_t tile = 0; tile < ntiles; ++tile)
        run_warp([&](int lane) {
            Counters ctr;
            process_tile<K, 0, MIXED>(a, tg.R_rings, tile, tile_pts, smem, lane, ctr);
        });
    std::free(smem);
    for (int p = 0; p < count; ++p) {
        printf("%d", (int)status[p]);
        for (int k = 0; k < K; ++k) printf(" %lld", (long long)st[(size_t)p * K + k]);
        printf("\n");
    }
}

template <int K> static void dispatch(int mixed, long long N, long long first, int count) {
    if (mixed) stencil<K, 1>(N, first, count); else stencil<K, 0>(N, first, count);
}

int main() {
    long long N, first;
    int K, mixed, count;
    while (scanf("%lld %d %d %lld %d %lf", &N, &K, &mixed, &first, &count, &g_r2_scale) == 6) {
        switch (K) {
            case 16: dispatch<16>(mixed, N, first, count); break;
            case 24: dispatch<24>(mixed, N, first, count); break;
            case 32: dispatch<32>(mixed, N, first, count); break;
            case 48: dispatch<48>(mixed, N, first, count); break;
            default: return 3;
        }
    }
    return 0;
}
"""


def _build(tmpdir, sanitize=None):
    api = open(hc.CSRC + "/api.cu").read()
    a = api.index("TableGrid table_grid(")
    depth, k = 0, api.index("{", a)
    while True:
        depth += {"{": 1, "}": -1}.get(api[k], 0)
        if depth == 0:
            break
        k += 1
    text = (hc.LENS_SHIM + '#include "' + hc.ROOT + '/include/flints.h"\nnamespace flints {\n'
            + hc.cut("common.cuh", "constexpr unsigned FULL", "// Host-side launchers (lens_spin0.cu", False)
            + api[a:k + 1] + "\n"
            + hc.cut("lens.cuh", "template <class T>\nstruct Cx {", "// Single-launch kernel", False)
            + "\n}\n" + DRIVER)
    exe = hc.build(tmpdir, "stencil_host", text, warp="threads", sanitize=sanitize)

    def call(N, K, mixed, first, defl, r2_scale=1.0):
        line = f"{N} {K} {mixed} {first} {len(defl)} {r2_scale!r} " + " ".join(float(x).hex() for x in np.ravel(defl))
        rows = [ln.split() for ln in hc.run(exe, line + "\n").splitlines()]
        return np.array([int(r[0]) for r in rows]), np.array([[int(t) for t in r[1:]] for r in rows])

    return call


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    return _build(tmp_path_factory.mktemp("stencil"))


def _check(N, K, first, defl, status, idx):
    assert np.all(status == 0), np.unique(status)
    tv = kr.displace(N, np.arange(first, first + len(defl)), defl)
    ref, key = kr.knn(N, tv, K + 1)
    kK, kK1 = key[:, K - 1], key[:, K]
    tie = (kK1 - kK) <= 1e-11 * kK1
    same = np.all(idx == ref[:, :K], axis=1)
    assert np.all(same | tie), f"{np.sum(~same & ~tie)} stencils differ"
    for p in np.nonzero(~same)[0]:  # a tie for the last place: the set must still be a K-nearest set
        got = np.sort(np.sum((hp.pix2vec(N, idx[p]) - tv[p]) ** 2, axis=1))
        assert np.allclose(got, np.sort(key[p, :K]), rtol=1e-10, atol=0)


# (Nside, K, first target pixel): north cap from pixel 0, the north cap/belt edge, the
# equator, the south cap/belt edge and the last pixels of the south cap
def _ranges(N, n):
    ncap = 2 * N * (N - 1)
    npix = 12 * N * N
    return [0, ncap - n // 2, npix // 2 - n // 2, npix - ncap - n // 2, npix - n]


@pytest.mark.parametrize("N,K", [(64, 24), (2048, 32), (4096, 16), (8192, 48), (16384, 32), (16384, 48)])
@pytest.mark.parametrize("mixed", [0, 1])
def test_stencils_match_the_oracle(N, K, mixed, run):
    rng = np.random.default_rng(N + K + mixed)
    n = 96
    for first in _ranges(N, n):
        # lensing-sized deflections, and some of a pixel or two
        scale = np.where(rng.random(n) < 0.5, wl.DEFLECTION_RMS * 4096 / N, 2.0 / N)
        defl = rng.normal(size=(n, 2)) * scale[:, None]
        status, idx = run(N, K, mixed, first, defl)
        _check(N, K, first, defl, status, idx)


def test_targets_at_pixel_centres_keep_their_pixel_first(run):
    for mixed in (0, 1):
        status, idx = run(16384, 32, mixed, 1_600_000_000, np.zeros((40, 2)))
        assert np.all(status == 0)
        assert np.array_equal(idx[:, 0], np.arange(1_600_000_000, 1_600_000_040))


def test_stencils_outside_a_shrunken_disc_are_flagged(run):
    """The window check (FLINTS_ST_WINDOW | FLINTS_ST_FAILED when the K-th neighbour lies
    outside the search disc), never reached with the plan's disc, on a disc shrunk to 0.6
    of its area: flagged exactly where the oracle's K-th squared chord exceeds it."""
    N, K = 4096, 32
    rng = np.random.default_rng(3)
    first, n = 50_000_000, 192
    defl = rng.normal(size=(n, 2)) * (2.0 / N)
    r = 1.25 * np.sqrt(K / 3.0) / N
    for mixed in (0, 1):
        status, idx = run(N, K, mixed, first, defl, 0.6)
        tv = kr.displace(N, np.arange(first, first + n), defl)
        _, key = kr.knn(N, tv, K)
        outside = key[:, K - 1] > 0.6 * r * r
        assert 0 < np.sum(outside) < n  # both outcomes occur
        near = np.abs(key[:, K - 1] / (0.6 * r * r) - 1) < 1e-6  # too close to call
        flagged = status == (4 | 8)
        assert np.array_equal(flagged[~near], outside[~near])
        assert np.all(status[~flagged] == 0) and np.all(idx[flagged] == -1)


def test_largest_sky_under_the_sanitizers(tmp_path_factory):
    """The search at Nside 16384 (3.2e9 pixels, past 32-bit signed indices) and K = 48
    built with the address sanitizer and the signed-overflow and bounds checks: no
    index computation overflows and no access leaves its array, on both caps, both
    cap/belt edges and the equator, FP64 and mixed kernels."""
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    run = _build(tmp_path_factory.mktemp("stencil_san"), sanitize="address")
    N, K, n = 16384, 48, 24
    rng = np.random.default_rng(7)
    for mixed in (0, 1):
        for first in _ranges(N, n):
            defl = rng.normal(size=(n, 2)) * wl.DEFLECTION_RMS / 4
            status, idx = run(N, K, mixed, first, defl)
            _check(N, K, first, defl, status, idx)
