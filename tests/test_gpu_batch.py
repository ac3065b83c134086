"""Batched persistent launches (many plans of different Nside, K, spin and
precision in one launch per precision class), CUDA-graph capture and replay,
and the launch-shape autotuner: every result must equal the single-plan
launch of the same target range (same per-point code; tolerance 1e-12 of the
parity metric) and, through the single-plan path, the oracle."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
from tests.gpu_common import parity_metric, require_gpu, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fl():
    return require_gpu()


def _make(fl, torch, spin, nside, K, precision, seed):
    lmax = 2 * nside
    cl = wl.cl_tt(lmax, 0.61 * lmax) if spin == 0 else wl.cl_ee(lmax, 0.61 * lmax)
    npix = hp.npix(nside)
    m = torch.from_numpy(wl.white_map(npix, 1 if spin == 0 else 2, seed)).cuda()
    d = torch.from_numpy(wl.random_deflection(npix, seed + 1) * 4).cuda()
    plan = fl.Plan(nside, cl, spin=spin, K=K, precision=precision)
    return plan, m, d


def _outputs(torch, plan, count):
    o = torch.full((count,) if plan.spin == 0 else (count, 2), float("nan"), dtype=torch.float64, device="cuda")
    v = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.full((count,), 255, dtype=torch.uint8, device="cuda")
    return o, v, s


SPECS = [(0, 32, 16, "mixed", 1), (2, 16, 48, "mixed", 2), (0, 64, 24, "fp64", 3), (2, 32, 32, "fp64", 4),
         (2, 64, 32, "mixed", 5), (0, 16, 48, "fp64", 6), (2, 16, 24, "mixed", 7), (0, 32, 32, "mixed", 8)]


def _jobs(fl, torch, ranges):
    plans, jobs, refs = [], [], []
    for (spin, nside, K, prec, seed), (f, c) in zip(SPECS, ranges):
        plan, m, d = _make(fl, torch, spin, nside, K, prec, 10 * seed)
        c = min(c, plan.npix - f)
        dd = d[f:f + c].contiguous()
        o, v, s = _outputs(torch, plan, c)
        r = plan.lens(m, dd, *_outputs(torch, plan, c), first=f, count=c)
        plans.append(plan)
        jobs.append((plan, f, c, m, dd, o, v, s))
        refs.append(r)
    torch.cuda.synchronize()
    return plans, jobs, refs


def _check(jobs, refs, tol=1e-12):
    for (plan, f, c, m, d, o, v, s), (ro, rv, rs) in zip(jobs, refs):
        if c == 0:
            continue
        scale = float(to_host(m).std())
        assert parity_metric(to_host(o), to_host(ro), scale) <= tol
        assert parity_metric(to_host(v), to_host(rv), plan.info().xi0) <= tol
        assert np.array_equal(to_host(s), to_host(rs))


def test_batch_matches_single_launches(fl):
    import torch

    ranges = [(0, 12288), (100, 777), (5, 3000), (0, 12288), (20000, 29000), (0, 0), (17, 1), (4000, 8191)]
    plans, jobs, refs = _jobs(fl, torch, ranges)
    before = [p.stats()["points"] for p in plans]
    b = fl.Batch(16)
    b.run(jobs)
    torch.cuda.synchronize()
    _check(jobs, refs)
    after = [p.stats()["points"] for p in plans]
    assert [a - x for a, x in zip(after, before)] == [j[2] for j in jobs]
    for cfg in (fl.LaunchCfg(2, 1, 16), fl.LaunchCfg(8, 0, 12), fl.LaunchCfg(4, 2, 7)):
        for j in jobs:
            j[5].fill_(float("nan"))
        b.run(jobs, cfg)
        torch.cuda.synchronize()
        _check(jobs, refs)
    # the convenience entry point
    for j in jobs:
        j[5].fill_(float("nan"))
    fl.lens_batch(jobs)
    _check(jobs, refs)
    b.close()


def test_batch_graph_capture_and_restage(fl):
    import torch

    ranges = [(0, 4096)] * len(SPECS)
    plans, jobs, refs = _jobs(fl, torch, ranges)
    b = fl.Batch(16)
    cfg = fl.LaunchCfg(4, 0, 16)
    b.run(jobs, cfg)  # first launch with this shape happens before capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    for j in jobs:
        j[5].fill_(float("nan"))
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        b.launch(cfg, stream=s)
    g.replay()
    torch.cuda.synchronize()
    _check(jobs, refs)
    # restage: same buffers, other target ranges; the captured graph runs the new table
    ranges2 = [(1000, 3000)] * len(SPECS)
    jobs2, refs2 = [], []
    for (plan, f, c, m, d, o, v, st), (f2, c2) in zip(jobs, ranges2):
        npix = plan.npix
        c2 = min(c2, npix - f2)
        d2 = torch.from_numpy(wl.random_deflection(c2, f2 + 5) * 4).cuda()
        d[:c2].copy_(d2)
        r = plan.lens(m, d[:c2].contiguous(), *_outputs(torch, plan, c2), first=f2, count=c2)
        jobs2.append((plan, f2, c2, m, d, o, v, st))
        refs2.append(r)
    torch.cuda.synchronize()
    b.stage(jobs2, cfg.tile_points)
    g.replay()
    torch.cuda.synchronize()
    trimmed = [(p, f, c, m, d, o[:c], v[:c], st[:c]) for (p, f, c, m, d, o, v, st) in jobs2]
    _check(trimmed, refs2)
    b.close()


def test_autotuner_picks_and_caches(fl, tmp_path):
    import torch

    from paper_1003_4984_gb300 import autotune

    plan, m, d = _make(fl, torch, 2, 64, 32, "mixed", 90)
    n = 8192
    ref = plan.lens(m, d[:n].contiguous(), *_outputs(torch, plan, n), first=0, count=n)
    cache = str(tmp_path / "tune.json")
    cands = [fl.LaunchCfg(2, 0, 16), fl.LaunchCfg(4, 0, 16), fl.LaunchCfg(8, 0, 8)]
    cfg = autotune.tune_plan(plan, m, d[:n].contiguous(), 0, n, cache=cache, cands=cands)
    assert cfg.key() in [c.key() for c in cands]
    assert os.path.exists(cache)
    got = plan.lens(m, d[:n].contiguous(), *_outputs(torch, plan, n), first=0, count=n)
    torch.cuda.synchronize()
    assert parity_metric(to_host(got[0]), to_host(ref[0]), 1.0) <= 1e-12
    # a second plan of the same class reuses the cached choice without timing
    plan2, _, _ = _make(fl, torch, 2, 64, 32, "mixed", 91)
    cfg2 = autotune.tune_plan(plan2, m, d[:n].contiguous(), 0, n, cache=cache, cands=[fl.LaunchCfg(1, 1, 1)])
    assert cfg2.key() == cfg.key()
