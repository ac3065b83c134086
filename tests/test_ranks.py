"""Multi-rank host logic of the benchmark (paper_1003_4984_gb300.ranks) on two
gloo ranks on the CPU: the layout that lets every GPU lens its own problem
with no data-path collective, and the barrier + MAX reduction of the timings."""
import os
import socket

import pytest

from paper_1003_4984_gb300 import ranks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    try:
        w, r, local = ranks.rank_env()
        dist = ranks.init("gloo")
        ranks.barrier(dist)
        # the slowest rank's time is every rank's time
        t = ranks.max_over_ranks(10.0 + 5.0 * r, dist)
        # ranks lens different batches and maps
        batches = [ranks.batch_index(r, i, 12) for i in range(5)]
        q.put((r, w, local, t, batches, ranks.seed(r, 1234), ranks.job_rate(1000, t, w)))
        ranks.barrier(dist)
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, "error", repr(e)))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[1] != "error" for r in res), res
    res.sort()
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 and r[2] == r[0] for r in res)
    assert all(r[3] == 15.0 for r in res)  # MAX over ranks
    assert not set(res[0][4]) & set(res[1][4])  # distinct batches within a sky's first steps
    assert res[0][5] != res[1][5]  # independent maps
    assert res[0][6] == pytest.approx(2 * 1000 / 15.0)  # whole-job rate: all ranks' points / slowest time


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert ranks.rank_env() == (1, 0, 0)
    assert ranks.init("gloo") is None
    assert ranks.max_over_ranks(3.5, None) == 3.5
    ranks.barrier(None)
