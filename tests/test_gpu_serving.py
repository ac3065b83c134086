"""Continuous-batching server: requests that arrive while others run are mixed
into shared batched launches; each result must equal the same request lensed
alone (tolerance 1e-12 of the parity metric), memory must be returned, and
latencies recorded."""
import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
from tests.gpu_common import parity_metric, require_gpu, to_host

pytestmark = pytest.mark.gpu


def test_each_result_is_the_same_alone_and_in_the_mix():
    fl = require_gpu()
    import torch

    from paper_1003_4984_gb300.serving import LensServer, Request, latency_stats

    rng = np.random.default_rng(5)
    server = LensServer(hbm_budget=2e8, batch_points=20000, chunk_points=7000, max_jobs=16)
    for nside in (32, 64):
        for spin in (0, 2):
            lmax = 2 * nside
            cl = wl.cl_tt(lmax, 0.61 * lmax) if spin == 0 else wl.cl_ee(lmax, 0.61 * lmax)
            m = torch.from_numpy(wl.white_map(hp.npix(nside), 1 if spin == 0 else 2, nside + spin)).cuda()
            server.register_map(nside, spin, m, cl)
    reqs = []
    for rid in range(24):
        nside = int(rng.choice([32, 64]))
        spin = int(rng.choice([0, 2]))
        K = int(rng.choice([16, 32]))
        npix = hp.npix(nside)
        count = int(rng.integers(1, min(npix, 20000)))
        first = int(rng.integers(0, npix - count + 1))
        d = torch.from_numpy(wl.random_deflection(count, 700 + rid) * 4).cuda()
        reqs.append(Request(rid, (nside, spin), K, first, count, d, arrival=0.02 * rid))
    done = server.run(reqs)
    torch.cuda.synchronize()
    assert len(done) == len(reqs) and server.in_use == 0
    assert server.launches < sum(-(-r.count // 7000) for r in reqs)  # chunks of several requests shared launches
    for r in done:
        alone = fl.Plan(r.map_key[0], server.spectra[r.map_key][0], spin=r.map_key[1], K=r.K, precision=r.precision)
        ref, rvar, _ = alone.lens(server.maps[r.map_key], r.defl,
                                  var=torch.empty(r.count, dtype=torch.float64, device="cuda"), first=r.first,
                                  count=r.count)
        torch.cuda.synchronize()
        assert parity_metric(to_host(r.out), to_host(ref), 1.0) <= 1e-12
        assert parity_metric(to_host(r.var), to_host(rvar), alone.info().xi0) <= 1e-12
        alone.close()
    st = latency_stats(done)
    assert st["requests"] == 24 and st["p99_ms"] >= st["p50_ms"] > 0
    server.close()


def _server_with_maps(budget, batch_points=20000, chunk_points=7000):
    import torch

    from paper_1003_4984_gb300.serving import LensServer

    server = LensServer(hbm_budget=budget, batch_points=batch_points, chunk_points=chunk_points, max_jobs=16)
    for nside in (32, 64):
        for spin in (0, 2):
            lmax = 2 * nside
            cl = wl.cl_tt(lmax, 0.61 * lmax) if spin == 0 else wl.cl_ee(lmax, 0.61 * lmax)
            m = torch.from_numpy(wl.white_map(hp.npix(nside), 1 if spin == 0 else 2, nside + spin)).cuda()
            server.register_map(nside, spin, m, cl)
    return server


def _alone(fl, server, r):
    import torch

    alone = fl.Plan(r.map_key[0], server.spectra[r.map_key][0], spin=r.map_key[1], K=r.K, precision=r.precision)
    ref, rvar, _ = alone.lens(server.maps[r.map_key], r.defl, var=torch.empty(r.count, dtype=torch.float64,
                                                                             device="cuda"), first=r.first,
                              count=r.count)
    torch.cuda.synchronize()
    x0 = alone.info().xi0
    alone.close()
    return to_host(ref), to_host(rvar), x0


def test_deflections_made_on_the_device_at_admission():
    """Deflections produced by a callable on the GPU at admission (as the benchmark's
    serving load does) are complete before the launch streams read them."""
    fl = require_gpu()
    import torch

    from paper_1003_4984_gb300.serving import Request

    server = _server_with_maps(2e8)

    def maker(count, seed):
        def make():
            g = torch.Generator(device="cuda")
            g.manual_seed(seed)
            d = torch.randn((count, 2), dtype=torch.float64, device="cuda", generator=g) * 4e-3
            return d * 1.0  # more queued work before the launch reads it
        return make

    rng = np.random.default_rng(11)
    reqs = []
    for rid in range(12):
        nside, spin, K = int(rng.choice([32, 64])), int(rng.choice([0, 2])), int(rng.choice([16, 32]))
        npix = hp.npix(nside)
        count = int(rng.integers(1000, min(npix, 20000)))
        first = int(rng.integers(0, npix - count + 1))
        reqs.append(Request(rid, (nside, spin), K, first, count, maker(count, 900 + rid), arrival=0.01 * rid))
    done = server.run(reqs)
    torch.cuda.synchronize()
    assert len(done) == 12 and server.in_use == 0
    for r in done:
        ref, rvar, x0 = _alone(fl, server, r)
        assert parity_metric(to_host(r.out), ref, 1.0) <= 1e-12
        assert parity_metric(to_host(r.var), rvar, x0) <= 1e-12
    server.close()


def test_budget_admission_waits_and_oversized_request_runs_alone():
    """With room for one request beside the resident maps and plans, requests wait
    for memory: their admitted intervals never overlap; a request larger than the
    whole remaining budget is still served, alone."""
    fl = require_gpu()
    import torch

    from paper_1003_4984_gb300.serving import LensServer, Request

    count = 6000
    probe = Request(0, (64, 0), 16, 0, count, None)
    nb = LensServer.request_bytes(probe)
    server = _server_with_maps(1.0)
    for key in ((64, 0), (64, 2)):  # plans first: they are resident and counted
        server.plan_for(Request(0, key, 16, 0, 1, None))
    server.budget = server.used_bytes() + 1.5 * nb
    reqs = []
    for rid in range(6):
        key = (64, rid % 2 * 2)
        d = torch.from_numpy(wl.random_deflection(count, 40 + rid) * 4).cuda()
        reqs.append(Request(rid, key, 16, 1000 * rid, count, d, arrival=0.0))
    big = 3 * count  # its buffers alone exceed what the budget leaves
    d = torch.from_numpy(wl.random_deflection(big, 99) * 4).cuda()
    reqs.append(Request(6, (64, 0), 16, 100, big, d, arrival=0.0))
    assert server.used_bytes() + LensServer.request_bytes(reqs[-1]) > server.budget
    done = server.run(reqs)
    torch.cuda.synchronize()
    assert len(done) == 7 and server.in_use == 0
    spans = sorted((r.admitted_at, r.finished_at) for r in done)
    for (a0, f0), (a1, f1) in zip(spans, spans[1:]):
        assert a1 >= f0, "two requests were admitted at once although only one fits"
    for r in done:
        ref, rvar, x0 = _alone(fl, server, r)
        assert parity_metric(to_host(r.out), ref, 1.0) <= 1e-12
    server.close()


def test_cancel_pending_and_running_requests():
    """A cancelled pending request never runs; a cancelled running request gets no
    further chunks and returns its memory; the other requests are unaffected."""
    fl = require_gpu()
    import torch

    from paper_1003_4984_gb300.serving import Request

    server = _server_with_maps(2e8, batch_points=4000, chunk_points=2000)
    reqs = []
    for rid in range(6):
        key = (64, 0 if rid % 2 else 2)
        count = 12000
        d = torch.from_numpy(wl.random_deflection(count, 300 + rid) * 4).cuda()
        reqs.append(Request(rid, key, 32, 500 * rid, count, d, arrival=0.0 if rid < 5 else 30.0))
    state = {"running": False, "pending": False}

    def tick(srv, now):
        if not state["running"] and any(r.rid == 1 and r.done_points > 0 for r in srv.active):
            state["running"] = srv.cancel(1)
        if not state["pending"] and any(r.rid == 5 for r in srv.pending):
            state["pending"] = srv.cancel(5)

    done = server.run(reqs, on_tick=tick, time_scale=0.01)
    torch.cuda.synchronize()
    assert state["running"] and state["pending"]
    assert sorted(r.rid for r in done) == [0, 2, 3, 4]
    assert sorted(r.rid for r in server.cancelled) == [1, 5]
    c1 = next(r for r in server.cancelled if r.rid == 1)
    assert 0 < c1.done_points < c1.count and server.in_use == 0 and not server.active
    assert server.cancel(1) is False
    for r in done:
        ref, rvar, x0 = _alone(fl, server, r)
        assert parity_metric(to_host(r.out), ref, 1.0) <= 1e-12
    server.close()


def test_empty_and_invalid_requests():
    """A request with no targets finishes at admission instead of keeping the loop
    alive; a request outside its map is refused before anything runs."""
    fl = require_gpu()
    import torch

    from paper_1003_4984_gb300.serving import Request

    server = _server_with_maps(2e8)
    d = torch.from_numpy(wl.random_deflection(3000, 61) * 4).cuda()
    empty = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    reqs = [Request(0, (32, 0), 16, 10, 3000, d, arrival=0.0), Request(1, (64, 2), 32, 5, 0, empty, arrival=0.0)]
    done = server.run(reqs)
    torch.cuda.synchronize()
    assert sorted(r.rid for r in done) == [0, 1] and server.in_use == 0 and not server.active
    assert next(r for r in done if r.rid == 1).latency is not None
    ref, _, x0 = _alone(fl, server, next(r for r in done if r.rid == 0))
    assert parity_metric(to_host(done[[r.rid for r in done].index(0)].out), ref, 1.0) <= 1e-12
    with pytest.raises(ValueError, match="outside the map"):
        server.run([Request(2, (32, 0), 16, 12 * 32 * 32 - 5, 10, d[:10])])
    with pytest.raises(ValueError, match="no map registered"):
        server.run([Request(3, (128, 0), 16, 0, 10, d[:10])])
    assert not server.pending and not server.active
    server.close()
