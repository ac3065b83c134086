"""The lens kernel's warp sorts (csrc/lens.cuh: bitonic_sort of (key, id) pairs
and bitonic_sort_packed of 64-bit keys, element e = 32 s + lane) run on a host
warp of 32 threads that meet at every shuffle, for every register count the
kernels use (32 * SPL = 128 and 256 candidate slots, and the smaller ones),
with ties, padding keys and already ordered or reversed inputs.  The K-nearest
selection reads the first K sorted entries, so the order must be exact:
ascending keys, equal keys by ascending id."""
import numpy as np
import pytest

from tests import host_compile as hc

DRIVER = r"""
using namespace flints;
template <int SPL> static void one(bool packed) {
    constexpr int NE = 32 * SPL;
    std::vector<unsigned long long> key(NE);
    std::vector<unsigned> id(NE);
    for (int e = 0; e < NE; ++e) {
        if (scanf("%llu", &key[e]) != 1) exit(2);
        if (!packed && scanf("%u", &id[e]) != 1) exit(2);
    }
    run_warp([&](int lane) {
        unsigned long long k[SPL];
        unsigned d[SPL];
        for (int s = 0; s < SPL; ++s) {
            k[s] = key[s * 32 + lane];
            d[s] = id[s * 32 + lane];
        }
        if (packed) bitonic_sort_packed<SPL>(k, lane);
        else bitonic_sort<SPL>(k, d, lane);
        __syncwarp();
        for (int s = 0; s < SPL; ++s) {
            key[s * 32 + lane] = k[s];
            id[s * 32 + lane] = d[s];
        }
    });
    for (int e = 0; e < NE; ++e) printf(packed ? "%llu\n" : "%llu %u\n", key[e], id[e]);
}
int main() {
    int spl, packed;
    while (scanf("%d %d", &spl, &packed) == 2) {
        switch (spl) {
            case 1: one<1>(packed); break;
            case 2: one<2>(packed); break;
            case 4: one<4>(packed); break;
            case 8: one<8>(packed); break;
            default: return 3;
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    text = ("#include <vector>\nnamespace flints {\nconstexpr unsigned FULL = 0xffffffffu;\n"
            + hc.cut("lens.cuh", "__device__ __forceinline__ bool key_less(",
                     "template <class R>\n__device__ __forceinline__ typename Ops<R>::T table_eval(", False)
            + "\n}\n" + DRIVER)
    exe = hc.build(tmp_path_factory.mktemp("sort"), "sort_host", text, warp="threads")

    def call(spl, keys, ids=None):
        packed = ids is None
        vals = keys if packed else np.stack([keys, ids], 1).ravel()
        out = hc.run(exe, f"{spl} {int(packed)} " + " ".join(str(int(v)) for v in vals) + "\n")
        rows = np.array([[int(t) for t in ln.split()] for ln in out.splitlines()], dtype=np.uint64)
        return rows[:, 0] if packed else (rows[:, 0], rows[:, 1])

    return call


def _cases(rng, n):
    pad = np.uint64(0xFFFFFFFFFFFFFFFF)
    yield rng.integers(0, 2 ** 63, n, dtype=np.uint64)  # distinct (almost surely)
    yield rng.integers(0, 5, n).astype(np.uint64)  # many ties
    k = rng.integers(0, 2 ** 40, n, dtype=np.uint64)
    k[rng.random(n) < 0.3] = pad  # padding slots, as for unused candidates
    yield k
    yield np.sort(rng.integers(0, 2 ** 50, n, dtype=np.uint64))
    yield np.sort(rng.integers(0, 2 ** 50, n, dtype=np.uint64))[::-1].copy()


@pytest.mark.parametrize("spl", [1, 2, 4, 8])
def test_pair_sort_orders_by_key_then_id(spl, run):
    rng = np.random.default_rng(spl)
    n = 32 * spl
    for keys in _cases(rng, n):
        ids = rng.permutation(n).astype(np.uint64)
        k, i = run(spl, keys, ids)
        order = np.lexsort((ids, keys))
        assert np.array_equal(k, keys[order]) and np.array_equal(i, ids[order])


@pytest.mark.parametrize("spl", [1, 2, 4, 8])
def test_packed_sort(spl, run):
    rng = np.random.default_rng(10 + spl)
    n = 32 * spl
    for keys in _cases(rng, n):
        # packed keys: FP32 key bits above a 32-bit candidate index, as the pre-selection builds them
        if keys.max() < 2 ** 32:
            keys = (keys << np.uint64(32)) | rng.permutation(n).astype(np.uint64)
        assert np.array_equal(run(spl, keys), np.sort(keys))
