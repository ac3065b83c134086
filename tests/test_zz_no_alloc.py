"""The entry point that allocates nothing (flints_lens_noalloc), checked against
the FP64 oracle and against the plan-based entry point.

It serves callers that cannot call cudaMalloc -- serving runtimes whose device
memory belongs to their own pool, hosts that forbid library allocations -- by
keeping the library's working memory in a fixed device array shared by every
call.  Each case runs two calls in a row (the second one sees the array as the
first one left it).  This file is collected last so that a run stopping at the
first failure has run every other test before it.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
from oracle import kriging as kr
from oracle import sht
from tests.gpu_common import oracle_table, parity_metric, require_gpu, to_host

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-9, "mixed": 1e-6}


def _case(spin, nside, lmax, seed, with_bb):
    cl = wl.cl_tt(lmax, 0.6 * lmax) if spin == 0 else wl.cl_ee(lmax, 0.6 * lmax)
    bb = 0.3 * cl if (spin == 2 and with_bb) else None
    alm = wl.draw_alm(cl, seed)
    if spin == 2:
        blm = wl.draw_alm(bb, seed + 7) if bb is not None else None
        m = sht.synth_map(nside, lmax, alm, spin=2, blm=blm) if blm is not None else sht.synth_map(nside, lmax, alm,
                                                                                                     spin=2)
        m = np.stack([m.real, m.imag], axis=1)
    else:
        m = sht.synth_map(nside, lmax, alm)
    defl = wl.random_deflection(hp.npix(nside), seed + 1) * 4
    return cl, bb, np.ascontiguousarray(m), defl


# (spin, nside, lmax, K, precision, seed, cl_bb given, first, count (None: to the end))
CASES = [(0, 64, 128, 16, "fp64", 61, False, 0, None),
         (2, 32, 64, 32, "mixed", 71, False, 0, None),
         (2, 32, 64, 24, "fp64", 81, True, 1001, 5000),
         (0, 32, 64, 48, "mixed", 91, False, 7, 3001)]


@pytest.mark.parametrize("case", CASES, ids=[f"spin{c[0]}-K{c[3]}-{c[4]}{'-bb' if c[6] else ''}" for c in CASES])
def test_noalloc_matches_oracle_and_plan_on_two_calls_in_a_row(case):
    fl = require_gpu()
    import torch

    from paper_1003_4984_gb300.api import lens_noalloc

    spin, nside, lmax, K, precision, seed, with_bb, first, count = case
    cl, bb, m, defl_all = _case(spin, nside, lmax, seed, with_bb)
    npix = hp.npix(nside)
    count = npix - first if count is None else count
    defl = np.ascontiguousarray(defl_all[first:first + count])
    md, dd = torch.from_numpy(m).cuda(), torch.from_numpy(defl).cuda()
    oshape = (count,) if spin == 0 else (count, 2)
    sigma = float(np.sqrt(np.mean(m ** 2) * (1 if spin == 0 else 2)))
    # the oracle on the same inputs
    tab, x0, _, _ = oracle_table(cl, bb, spin, K, nside)
    ref = kr.lens(nside, K, spin, m, defl, np.arange(first, first + count), tab, x0)
    # the plan-based entry point
    plan = fl.Plan(nside, cl, bb, spin=spin, K=K, precision=precision)
    p_out, p_var, _ = plan.lens(md, dd, var=torch.empty(count, dtype=torch.float64, device="cuda"), first=first,
                                count=count)
    torch.cuda.synchronize()
    p_o, p_v = to_host(p_out), to_host(p_var)
    if spin == 2:
        p_o = p_o[:, 0] + 1j * p_o[:, 1]
    free_before = None
    for call in range(2):
        out = torch.full(oshape, float("nan"), dtype=torch.float64, device="cuda")
        var = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
        status = torch.full((count,), 255, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        if call == 1:
            free_before = torch.cuda.mem_get_info()[0]
        lens_noalloc(nside, cl, md, dd, out, var, status, cl_bb=bb, spin=spin, K=K, precision=precision,
                     first=first, count=count)
        torch.cuda.synchronize()
        if call == 1:  # the second call allocates no device memory
            assert torch.cuda.mem_get_info()[0] == free_before
        o, v = to_host(out), to_host(var)
        if spin == 2:
            o = o[:, 0] + 1j * o[:, 1]
        assert parity_metric(o, ref.value, sigma) <= TOL[precision], ("oracle", case, call)
        assert parity_metric(v, ref.variance, x0) <= TOL[precision], ("oracle", case, call)
        assert parity_metric(o, p_o, sigma) <= TOL[precision], ("plan", case, call)
        assert parity_metric(v, p_v, x0) <= TOL[precision], ("plan", case, call)
        assert np.all(to_host(status) & fl.ST_FAILED == 0)
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    require_gpu()
    import torch

    from paper_1003_4984_gb300.api import FlintsError, lens_noalloc

    z = torch.zeros((12 * 16 * 16, 2), dtype=torch.float64, device="cuda")
    s = z[:, 0].contiguous()
    with pytest.raises(FlintsError, match="lmax 8999 exceeds the fixed maximum 8192"):
        lens_noalloc(1, np.ones(9000), s[:12], z[:12], s[:12], count=12, K=16)
    # lmax 4000 at Nside 16, K = 16: the table rule asks for 65536 intervals
    with pytest.raises(FlintsError, match="65536 intervals, above the fixed maximum 8192"):
        lens_noalloc(16, np.ones(4001), s, z, s, K=16)
