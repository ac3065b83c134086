"""Multi-rank host logic (paper_1003_4984_gb300.ranks) on gloo ranks on the CPU:
one sky's targets split into contiguous RING ranges balanced by count, each
rank lensing its range of a replicated source map with no data-path
collective, the outputs gathered to rank 0, and the barrier + MAX reduction of
the timings.  The lens call is a host stand-in (a fixed function of the target
index and its deflection), so no GPU is needed."""
import os
import socket

import numpy as np
import pytest

from paper_1003_4984_gb300 import ranks

NPIX = 12 * 16 * 16 + 5  # not a multiple of the rank count


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sky_inputs():
    """The one sky every rank holds: a source map and the deflections of all targets."""
    rng = np.random.default_rng(3)
    return rng.standard_normal(NPIX), rng.standard_normal((NPIX, 2))


def _stub_lens(src, defl):
    """Stand-in for a lens call on [first, first+count): reads the replicated source
    around each target (as a stencil does, across range boundaries) and its
    deflection, returns (value, variance)."""
    import torch

    def lens_range(first, count):
        idx = np.arange(first, first + count)
        nb = (idx[:, None] + np.arange(-3, 4)[None, :]) % NPIX
        v = src[nb].mean(1) + 0.1 * defl[idx, 0]
        s2 = 1.0 + defl[idx, 1] ** 2
        return torch.from_numpy(v), torch.from_numpy(s2)

    return lens_range


def _worker(rank, world, port, q, npix=NPIX):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    try:
        w, r, local = ranks.rank_env()
        dist = ranks.init("gloo")
        src, defl = _sky_inputs()
        bounds = ranks.shard_bounds(npix, w)
        ranks.barrier(dist)
        val, var = ranks.lens_shard(_stub_lens(src, defl), bounds[r], batch=100)
        full_v = ranks.gather_shards(val, bounds, dist, r)
        full_s = ranks.gather_shards(var, bounds, dist, r)
        # the slowest rank's time is every rank's time
        t = ranks.max_over_ranks(10.0 + 5.0 * r, dist)
        windows = [ranks.step_window(bounds[r], i, 64) for i in range(6)]
        q.put((r, w, local, t, bounds[r], windows, None if full_v is None else (full_v.numpy(), full_s.numpy()),
               ranks.job_rate(1000, t, w)))
        ranks.barrier(dist)
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, "error", repr(e)))


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_shard_one_sky(world):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[1] != "error" for r in res), res
    res.sort(key=lambda r: r[0])
    assert [r[0] for r in res] == list(range(world)) and all(r[1] == world and r[2] == r[0] for r in res)
    assert all(r[3] == 10.0 + 5.0 * (world - 1) for r in res)  # MAX over ranks
    # the ranges tile [0, NPIX) exactly once, balanced by count
    b = [r[4] for r in res]
    assert b[0][0] == 0 and b[-1][1] == NPIX and all(b[i][1] == b[i + 1][0] for i in range(world - 1))
    sizes = [s1 - s0 for s0, s1 in b]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == NPIX
    # benchmark steps stay inside the rank's range
    for r in res:
        for first, count in r[5]:
            assert r[4][0] <= first and first + count <= r[4][1] and count == min(64, r[4][1] - r[4][0])
    # the gathered sky equals one rank lensing the whole range
    src, defl = _sky_inputs()
    one_v, one_s = ranks.lens_shard(_stub_lens(src, defl), (0, NPIX), batch=NPIX)
    full_v, full_s = res[0][6]
    assert all(r[6] is None for r in res[1:])
    np.testing.assert_array_equal(full_v, one_v.numpy())
    np.testing.assert_array_equal(full_s, one_s.numpy())
    assert res[0][7] == pytest.approx(world * 1000 / (10.0 + 5.0 * (world - 1)))  # whole-job rate


def test_gloo_ranks_with_empty_ranges():
    """A sky of fewer targets than ranks: the ranks past its end hold empty ranges
    and still take part in the gather; rank 0 gets exactly the sky."""
    import torch.multiprocessing as mp

    world, npix = 3, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, npix)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[1] != "error" for r in res), res
    res.sort(key=lambda r: r[0])
    assert [r[4] for r in res] == [(0, 1), (1, 2), (2, 2)]
    assert res[2][5] == [(2, 0)] * 6  # the empty range's benchmark windows are empty
    src, defl = _sky_inputs()
    one_v, one_s = ranks.lens_shard(_stub_lens(src, defl), (0, npix), batch=npix)
    full_v, full_s = res[0][6]
    np.testing.assert_array_equal(full_v, one_v.numpy())
    np.testing.assert_array_equal(full_s, one_s.numpy())


def test_shard_bounds_cover_the_sky_once():
    for n in (1, 7, 12 * 4096 * 4096):
        for world in (1, 2, 3, 8):
            b = ranks.shard_bounds(n, world)
            cover = np.zeros(min(n, 10_000), dtype=int)
            if n <= 10_000:
                for s0, s1 in b:
                    cover[s0:s1] += 1
                assert np.all(cover == 1)
            assert b[0][0] == 0 and b[-1][1] == n and sum(s1 - s0 for s0, s1 in b) == n


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert ranks.rank_env() == (1, 0, 0)
    assert ranks.init("gloo") is None
    assert ranks.max_over_ranks(3.5, None) == 3.5
    ranks.barrier(None)
    v = np.arange(5.0)
    assert ranks.gather_shards(v, [(0, 5)], None, 0) is v
