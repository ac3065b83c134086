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
