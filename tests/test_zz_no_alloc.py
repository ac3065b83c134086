"""The entry point that allocates nothing (flints_lens_noalloc) against the
plan-based entry point.

It serves callers that cannot call cudaMalloc -- code running under CUDA
stream capture, serving runtimes whose device memory belongs to their own
pool, hosts that forbid library allocations -- by keeping the library's
working memory in a fixed device array.  This file is collected last so that
a run stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
from oracle import sht
from tests.gpu_common import parity_metric, require_gpu, to_host

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-9, "mixed": 1e-6}


def _case(spin, nside, lmax, seed):
    cl = wl.cl_tt(lmax, 0.6 * lmax) if spin == 0 else wl.cl_ee(lmax, 0.6 * lmax)
    alm = wl.draw_alm(cl, seed)
    m = sht.synth_map(nside, lmax, alm, spin=spin)
    if spin == 2:
        m = np.stack([m.real, m.imag], axis=1)
    defl = wl.random_deflection(hp.npix(nside), seed + 1) * 4
    return cl, np.ascontiguousarray(m), defl


def test_noalloc_matches_plan_on_two_calls_in_a_row():
    fl = require_gpu()
    import torch

    from paper_1003_4984_gb300.api import lens_noalloc

    cases = [(0, 64, 128, 16, "fp64", 61), (2, 32, 64, 32, "mixed", 71)]
    for spin, nside, lmax, K, precision, seed in cases:
        cl, m, defl = _case(spin, nside, lmax, seed)
        npix = hp.npix(nside)
        md, dd = torch.from_numpy(m).cuda(), torch.from_numpy(defl).cuda()
        oshape = (npix,) if spin == 0 else (npix, 2)
        plan = fl.Plan(nside, cl, spin=spin, K=K, precision=precision)
        ref_out, ref_var, _ = plan.lens(md, dd, var=torch.empty(npix, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        ref_o, ref_v = to_host(ref_out), to_host(ref_var)
        sigma = float(np.sqrt(np.mean(m ** 2) * (1 if spin == 0 else 2)))
        for call in range(2):
            out = torch.full(oshape, float("nan"), dtype=torch.float64, device="cuda")
            var = torch.full((npix,), float("nan"), dtype=torch.float64, device="cuda")
            status = torch.full((npix,), 255, dtype=torch.uint8, device="cuda")
            lens_noalloc(nside, cl, md, dd, out, var, status, spin=spin, K=K, precision=precision)
            torch.cuda.synchronize()
            o, v = to_host(out), to_host(var)
            assert parity_metric(o, ref_o, sigma) <= TOL[precision], (spin, precision, call)
            assert parity_metric(v, ref_v, plan.info().xi0) <= TOL[precision], (spin, precision, call)
            assert np.all(to_host(status) & fl.ST_FAILED == 0)
        plan.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    require_gpu()
    import torch

    from paper_1003_4984_gb300.api import FlintsError, lens_noalloc

    z = torch.zeros((12, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(FlintsError, match="8192"):
        lens_noalloc(1, np.ones(9000), z[:, 0].contiguous(), z, z[:, 0].contiguous(), count=12, K=16)
