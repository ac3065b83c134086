"""GPU parity of the paper's estimator route with tabulated inverses (Secs.
2.3-2.5; flints_paper_*): the level-y pixel-centred stencil, L^-1 (the factor
of S^-1) per symmetry class of central pixels, two triangular matrix-vector
products per target.

Checked against the oracle (oracle/faces.py):
  * the stencil table: for every coarse pixel the GPU's member list equals the
    oracle's, in the oracle's own implementation of the ordering rule
    (bit-exact), and the GPU's classes are the oracle's (same partition of the
    coarse pixels);
  * the L^-1 blocks against the oracle's inverse Cholesky factor of each class
    representative's covariance (same correlation table rule);
  * lensed and supersampled values and variances against the oracle's class
    route (class_estimate) and against the per-target solve route (the
    Cholesky solve on each target's own stencil geometry):
    max |gpu - oracle| <= 1e-9 sigma_map and 1e-9 xi(0) for the FP64 path, 1e-6
    for the mixed (double-float) path, the two parity tolerances of this library;
  * at Nside 2048, lmax 4096 (y = 1, 2) on sampled targets of the full-sky call.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import faces as fc
from oracle import healpix as hp
from oracle import kriging as kr
from oracle import sht
from oracle import xi
from tests.gpu_common import require_gpu, to_host

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-9, "mixed": 1e-6}


@pytest.fixture(scope="module")
def fl():
    return require_gpu()


@pytest.fixture(scope="module")
def torch():
    import torch

    return torch


def _table(cl, nside, y):
    t_max, n = fc.paper_grid_rule(cl, nside, y)
    tab, x0 = xi.spin0_table(cl, t_max, n)
    return tab, x0, t_max, n


def _pixel_size(nside):
    return np.sqrt(4 * np.pi / hp.npix(nside))


@pytest.mark.parametrize("nside,y", [(1, 1), (2, 1), (4, 1), (8, 1), (16, 1), (2, 2), (4, 2), (8, 2), (32, 2)])
def test_stencil_table_and_classes(fl, torch, nside, y):
    cl = wl.cl_tt(3 * nside, 2.0 * nside)
    plan = fl.PaperPlan(nside, cl, y)
    info = plan.info()
    n_c = nside >> (y - 1)
    t_max, n = fc.paper_grid_rule(cl, nside, y)
    assert info["nside_coarse"] == n_c and info["K"] == 9 * 4 ** (y - 1)
    assert info["t_max"] == t_max and info["n_intervals"] == n
    assert info["max_pair_t"] <= t_max and info["failed_slots"] == 0
    mem, slot, _ = plan.tables()
    torch.cuda.synchronize()
    mem, slot = to_host(mem).astype(np.int64), to_host(slot).astype(np.int64)
    cen = np.arange(hp.npix(n_c))
    ref = fc.stencil_ordered(nside, y, cen)
    for c in cen:
        k = ref[c].size
        assert np.array_equal(mem[c][:k], ref[c]) and np.all(mem[c][k:] == -1), f"stencil of coarse pixel {c}"
    # the GPU's classes are the oracle's: slot and representative determine each other
    rep = fc.class_representative(n_c, cen)[0]
    assert slot.min() == 0 and slot.max() == info["slots"] - 1
    assert np.unique(slot).size == info["slots"] == np.unique(rep).size
    pairs = np.unique(np.stack([slot, rep], axis=1), axis=0)
    assert pairs.shape[0] == info["slots"]


def _unpack(packed, K):
    """Dense L^-1 from a class block: packed by columns (K = 9) or in the
    lane-step layout of include/flints.h (K = 36)."""
    L = np.zeros((K, K))
    if K != 36:
        off = 0
        for j in range(K):
            L[j:, j] = packed[off:off + K - j]
            off += K - j
        return L
    assert packed.size == 704
    for u in range(17):
        for lane in range(32):
            p, t = lane // 2, (u if lane % 2 == 0 else 17 + u)
            r, c = (p, t) if t <= p else (31 - p, t - p - 1)
            if c <= r:
                L[r, c] = packed[32 * u + lane]
            else:
                assert packed[32 * u + lane] == 0
    for t in range(5):
        for lane in range(32):
            r, c = 32 + lane % 4, lane // 4 + 8 * t
            if c <= r:
                L[r, c] = packed[544 + 32 * t + lane]
            else:
                assert packed[544 + 32 * t + lane] == 0
    return L


@pytest.mark.parametrize("nside,y", [(8, 1), (16, 2)])
def test_linv_blocks_match_oracle(fl, torch, nside, y):
    cl = wl.cl_tt(3 * nside, 2.0 * nside)
    tab, x0, _, _ = _table(cl, nside, y)
    plan = fl.PaperPlan(nside, cl, y)
    _, slot, linv = plan.tables()
    torch.cuda.synchronize()
    slot, linv = to_host(slot), to_host(linv)
    n_c = nside >> (y - 1)
    reps = np.unique(fc.class_representative(n_c, np.arange(hp.npix(n_c)))[0])
    for r, mem in zip(reps, fc.stencil_ordered(nside, y, reps)):
        k = mem.size
        X = hp.pix2vec(nside, mem)
        S = tab(np.sum((X[:, None] - X[None]) ** 2, axis=-1).reshape(-1)).reshape(1, k, k)
        L, nug = kr.factor_with_nugget(S, kr.EPS_NUGGET)
        assert nug[0] == kr.EPS_NUGGET
        ref = np.linalg.inv(L[0])
        G = _unpack(linv[slot[r]], plan.K)
        assert np.all(G[k:, :] == 0) and np.all(G[:, k:] == 0)
        assert np.max(np.abs(G[:k, :k] - ref)) <= 1e-9 * np.max(np.abs(ref)), f"class of coarse pixel {r}"


def _solve_route(nside, m, tv, idx, tab, x0):
    """Per-target Cholesky solve on each target's own stencil (grouped by member count)."""
    v = np.empty(tv.shape[0])
    s2 = np.empty(tv.shape[0])
    cnt = np.sum(idx >= 0, axis=1)
    for k in np.unique(cnt):
        rows = np.nonzero(cnt == k)[0]
        st = np.stack([r[r >= 0] for r in idx[rows]])
        v[rows], s2[rows], _ = kr.estimate(nside, 0, m, tv[rows], st, tab, x0)
    return v, s2


def _lens_case(fl, torch, nside, lmax, y, seed, first=0, count=None, precision="fp64"):
    cl = wl.cl_tt(lmax, 0.7 * lmax)
    m = sht.synth_map(nside, lmax, wl.draw_alm(cl, seed))
    npix = hp.npix(nside)
    count = npix - first if count is None else count
    # deflections of about half a pixel so targets spread over their coarse pixels
    defl = wl.random_deflection(count, seed + 1, rms=0.5 * _pixel_size(nside))
    plan = fl.PaperPlan(nside, cl, y, precision)
    md = torch.from_numpy(m).cuda()
    dd = torch.from_numpy(np.ascontiguousarray(defl)).cuda()
    st = torch.empty(count, dtype=torch.uint8, device="cuda")
    out, var = plan.lens(md, dd, first=first, count=count, status=st)
    torch.cuda.synchronize()
    tab, x0, _, _ = _table(cl, nside, y)
    pix = np.arange(first, first + count)
    ref = fc.paper_lens(nside, y, m, defl, pix, tab, x0, classes=True)
    own = _solve_route(nside, m, ref[3], ref[2], tab, x0)
    return plan, to_host(out), to_host(var), to_host(st), ref, own, float(np.std(m)), x0


def _check(v, s2, ref, own, sigma, x0, precision="fp64"):
    for rv, rs2 in ((ref[0], ref[1]), own):
        assert np.max(np.abs(v - rv)) <= TOL[precision] * sigma
        assert np.max(np.abs(s2 - rs2)) <= TOL[precision] * x0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nside,lmax,y", [(1, 8, 1), (2, 12, 1), (8, 16, 1), (32, 64, 1), (2, 12, 2), (16, 32, 2),
                                          (32, 64, 2)])
def test_lens_parity_whole_sky(fl, torch, nside, lmax, y, precision):
    plan, v, s2, st, ref, own, sigma, x0 = _lens_case(fl, torch, nside, lmax, y, 300 + nside + y,
                                                      precision=precision)
    _check(v, s2, ref, own, sigma, x0, precision)
    assert not np.any(st & (fl.ST_WINDOW | fl.ST_FAILED))
    assert plan.info()["window"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("y", [1, 2])
def test_lens_ragged_range(fl, torch, y, precision):
    # a range starting mid-ring and ending mid-tile
    plan, v, s2, st, ref, own, sigma, x0 = _lens_case(fl, torch, 16, 32, y, 77, first=1001, count=1234,
                                                      precision=precision)
    _check(v, s2, ref, own, sigma, x0, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nside,nout,y", [(16, 32, 1), (16, 64, 2), (8, 24, 1)])
def test_supersample_parity(fl, torch, nside, nout, y, precision):
    lmax = 2 * nside
    cl = wl.cl_tt(lmax, 0.7 * lmax)
    m = sht.synth_map(nside, lmax, wl.draw_alm(cl, 91))
    plan = fl.PaperPlan(nside, cl, y, precision)
    out, var = plan.supersample(torch.from_numpy(m).cuda(), nout)
    torch.cuda.synchronize()
    tab, x0, _, _ = _table(cl, nside, y)
    pix = np.arange(hp.npix(nout))
    ref = fc.paper_supersample(nside, nout, y, m, pix, tab, x0, classes=True)
    own = _solve_route(nside, m, ref[3], ref[2], tab, x0)
    _check(to_host(out), to_host(var), ref, own, float(np.std(m)), x0, precision)


def test_zero_deflection_reproduces_the_map(fl, torch):
    # at a pixel centre the target is a stencil member: the estimate returns the
    # pixel's value up to the nugget, and the variance is the nugget's share
    nside, lmax = 16, 32
    cl = wl.cl_tt(lmax, 0.7 * lmax)
    m = sht.synth_map(nside, lmax, wl.draw_alm(cl, 5))
    plan = fl.PaperPlan(nside, cl, 1)
    out, var = plan.lens(torch.from_numpy(m).cuda(), torch.zeros((hp.npix(nside), 2), dtype=torch.float64,
                                                                 device="cuda"))
    torch.cuda.synchronize()
    assert np.max(np.abs(to_host(out) - m)) <= 1e-6 * np.std(m)


def test_argument_errors(fl, torch):
    cl = wl.cl_tt(32, 20.0)
    with pytest.raises(fl.FlintsError, match="level y"):
        fl.PaperPlan(16, cl, 3)
    with pytest.raises(fl.FlintsError, match="divisible"):
        fl.PaperPlan(15, cl, 2)
    plan = fl.PaperPlan(16, cl, 1)
    md = torch.zeros(hp.npix(16), dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FlintsError, match="outside"):
        plan.lens(md, torch.zeros((10, 2), dtype=torch.float64, device="cuda"), first=hp.npix(16) - 5, count=10)


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("y", [1, 2])
def test_fullsize_2048_sampled(fl, torch, y, precision):
    # the whole-sky Nside 2048, lmax 4096 lensing call; outputs at sampled targets
    # (north cap, cap/belt boundary, equator, south cap) against the oracle on a
    # map known exactly on the rings those stencils reach
    W = wl.C2
    cl, _ = W.cl()
    alm = wl.draw_alm(cl, W.seed_map)
    npix = W.npix
    defl = wl.random_deflection(npix, 4242)
    samples = []
    for ring in (5, W.nside // 2, W.nside, W.nside + 1, 2 * W.nside, 4 * W.nside - 9):
        f, n_in = [int(x[0]) for x in hp.ring_info(W.nside, np.array([ring]))[:2]]
        samples.append(np.arange(f + n_in // 5, f + n_in // 5 + 48))
    pix = np.concatenate(samples)
    tv = kr.displace(W.nside, pix, defl[pix])
    idx = fc.stencil(W.nside, tv, y)
    rings = np.unique(hp.pix2ring(W.nside, idx[idx >= 0])[0])
    bp, bv = sht.synth_rings(W.nside, rings, W.lmax, alm)
    m = np.zeros(npix)
    m[bp] = bv
    plan = fl.PaperPlan(W.nside, cl, y, precision)
    md = torch.from_numpy(m).cuda()
    out, var = plan.lens(md, torch.from_numpy(defl).cuda())
    torch.cuda.synchronize()
    out, var = to_host(out)[pix], to_host(var)[pix]
    tab, x0, _, _ = _table(cl, W.nside, y)
    ref = fc.paper_lens(W.nside, y, m, defl[pix], pix, tab, x0, classes=True)
    own = _solve_route(W.nside, m, ref[3], ref[2], tab, x0)
    _check(out, var, ref, own, float(np.std(bv)), x0, precision)
    assert plan.info()["window"] == 0


def test_mixed_plan_tables(fl, torch):
    cl = wl.cl_tt(32, 20.0)
    plan = fl.PaperPlan(16, cl, 2, "mixed")
    assert plan.info()["precision"] == fl.FLINTS_MIXED
    mem, slot, linv = plan.tables()
    assert linv is None and mem.shape == (12 * 64, 36)


# ------------------------------------------------------------------ spin 2
def _spin2_inputs(nside, lmax, seed, bb_frac=0.3):
    cl = wl.cl_ee(lmax, 0.7 * lmax)
    bb = bb_frac * cl
    P = sht.synth_map(nside, lmax, wl.draw_alm(cl, seed), spin=2, blm=wl.draw_alm(bb, seed + 1))
    m = np.ascontiguousarray(np.stack([P.real, P.imag], axis=1))
    return cl, bb, m, float(np.sqrt(np.mean(np.abs(P) ** 2)))


def _spin2_table(cl, bb, nside, y):
    t_max, n = fc.paper_grid_rule(cl, nside, y, bb)
    tab, _, x0 = xi.spin2_tables(cl, bb, t_max, n)
    return tab, x0, t_max, n


def _spin2_solve_route(nside, m, tv, idx, tab, x0):
    v = np.empty(tv.shape[0], dtype=np.complex128)
    s2 = np.empty(tv.shape[0])
    cnt = np.sum(idx >= 0, axis=1)
    for k in np.unique(cnt):
        rows = np.nonzero(cnt == k)[0]
        st = np.stack([r[r >= 0] for r in idx[rows]])
        v[rows], s2[rows], _ = kr.estimate(nside, 2, m, tv[rows], st, tab, x0)
    return v, s2


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nside,lmax,y", [(2, 12, 1), (8, 16, 1), (32, 64, 1), (4, 24, 2), (16, 32, 2), (32, 64, 2)])
def test_spin2_lens_parity_whole_sky(fl, torch, nside, lmax, y, precision):
    # Q/U lensed with the paper stencil: the class's complex L^-1 (conjugated for the
    # southern classes) against the oracle's class route and per-target solve
    cl, bb, m, sigma = _spin2_inputs(nside, lmax, 400 + nside + y)
    npix = hp.npix(nside)
    defl = wl.random_deflection(npix, 401 + nside, rms=0.5 * _pixel_size(nside))
    plan = fl.PaperPlan(nside, cl, y, precision, spin=2, cl_bb=bb)
    t_max, n = fc.paper_grid_rule(cl, nside, y, bb)
    info = plan.info()
    assert info["spin"] == 2 and info["t_max"] == t_max and info["n_intervals"] == n
    st = torch.empty(npix, dtype=torch.uint8, device="cuda")
    out, var = plan.lens(torch.from_numpy(m).cuda(), torch.from_numpy(np.ascontiguousarray(defl)).cuda(), status=st)
    torch.cuda.synchronize()
    o = to_host(out)
    v = o[:, 0] + 1j * o[:, 1]
    s2 = to_host(var)
    tab, x0, _, _ = _spin2_table(cl, bb, nside, y)
    rv, rs2, idx, tv = fc.paper_lens(nside, y, m, defl, np.arange(npix), tab, x0, classes=True, spin=2)
    ov, os2 = _spin2_solve_route(nside, m, tv, idx, tab, x0)
    for a_v, a_s2 in ((rv, rs2), (ov, os2)):
        assert np.max(np.abs(v - a_v)) <= TOL[precision] * sigma
        assert np.max(np.abs(s2 - a_s2)) <= TOL[precision] * x0
    assert not np.any(to_host(st) & (fl.ST_WINDOW | fl.ST_FAILED))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nside,nout,y", [(16, 32, 1), (16, 32, 2)])
def test_spin2_supersample_and_ragged(fl, torch, nside, nout, y, precision):
    cl, bb, m, sigma = _spin2_inputs(nside, 2 * nside, 501)
    plan = fl.PaperPlan(nside, cl, y, precision, spin=2, cl_bb=bb)
    first, count = 777, 1501
    out, var = plan.supersample(torch.from_numpy(m).cuda(), nout, first=first, count=count)
    torch.cuda.synchronize()
    o = to_host(out)
    v = o[:, 0] + 1j * o[:, 1]
    tab, x0, _, _ = _spin2_table(cl, bb, nside, y)
    rv, rs2, idx, tv = fc.paper_supersample(nside, nout, y, m, np.arange(first, first + count), tab, x0,
                                            classes=True, spin=2)
    assert np.max(np.abs(v - rv)) <= TOL[precision] * sigma
    assert np.max(np.abs(to_host(var) - rs2)) <= TOL[precision] * x0


def test_spin2_linv_blocks(fl, torch):
    nside, y = 8, 1
    cl = wl.cl_ee(24, 16.0)
    bb = 0.3 * cl
    tab, x0, _, _ = _spin2_table(cl, bb, nside, y)
    plan = fl.PaperPlan(nside, cl, y, "fp64", spin=2, cl_bb=bb)
    _, slot, linv = plan.tables()
    torch.cuda.synchronize()
    slot, linv = to_host(slot), to_host(linv)
    reps = np.unique(fc.class_representative(nside, np.arange(hp.npix(nside)))[0])
    for r, mem in zip(reps, fc.stencil_ordered(nside, y, reps)):
        k = mem.size
        C = fc.class_covariance(nside, mem, tab, 2)
        L, nug = kr.factor_with_nugget(C[None], kr.EPS_NUGGET)
        ref = np.linalg.inv(L[0])
        blk = linv[slot[r]]
        G = _unpack(blk[:, 0], plan.K) + 1j * _unpack(blk[:, 1], plan.K)
        assert np.max(np.abs(G[:k, :k] - ref)) <= 1e-9 * np.max(np.abs(ref)), f"class of coarse pixel {r}"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nside,lmax,y", [(8, 16, 1), (16, 32, 2)])
def test_spin1_deflection_field_parity(fl, torch, nside, lmax, y, precision):
    # a deflection field d = grad(phi) (spin 1, E_l = l(l+1) C^phiphi_l) lensed with
    # the paper stencil: spin-1 phases carry the direction-of-travel sign
    phi = wl.draw_alm(wl.cl_phiphi(lmax), 600 + nside)
    ell = np.arange(lmax + 1)
    cl_e = ell * (ell + 1.0) * wl.cl_phiphi(lmax)
    m = np.ascontiguousarray(sht.synth_map(nside, lmax, phi, gradient=True))
    sigma = float(np.sqrt(np.mean(np.sum(m ** 2, axis=1))))
    npix = hp.npix(nside)
    defl = wl.random_deflection(npix, 601, rms=0.5 * _pixel_size(nside))
    plan = fl.PaperPlan(nside, cl_e, y, precision, spin=1)
    out, var = plan.lens(torch.from_numpy(m).cuda(), torch.from_numpy(np.ascontiguousarray(defl)).cuda())
    torch.cuda.synchronize()
    o = to_host(out)
    v = o[:, 0] + 1j * o[:, 1]
    t_max, n = fc.paper_grid_rule(cl_e, nside, y)
    tab, _, x0 = xi.spin1_tables(cl_e, None, t_max, n)
    rv, rs2, idx, tv = fc.paper_lens(nside, y, m, defl, np.arange(npix), tab, x0, classes=True, spin=1)
    cnt = np.sum(idx >= 0, axis=1)
    ov = np.empty(npix, dtype=np.complex128)
    os2 = np.empty(npix)
    for k in np.unique(cnt):
        rows = np.nonzero(cnt == k)[0]
        st = np.stack([r[r >= 0] for r in idx[rows]])
        ov[rows], os2[rows], _ = kr.estimate(nside, 1, m, tv[rows], st, tab, x0)
    for a_v, a_s2 in ((rv, rs2), (ov, os2)):
        assert np.max(np.abs(v - a_v)) <= TOL[precision] * sigma
        assert np.max(np.abs(to_host(var) - a_s2)) <= TOL[precision] * x0


@pytest.fixture(scope="module")
def qu4096():
    """The Nside 4096, lmax 4096 Q/U workload (c3 spectra, B = 0): targets sampled on
    rings of the north cap, the cap/belt boundary, the equator and the south cap,
    deflected by 2.5 arcmin Gaussian steps, and the map synthesised exactly on the
    rings their level-1 and level-2 stencils reach."""
    W = wl.C3
    cl, bb = W.cl()
    samples = []
    for ring in (5, W.nside // 2, W.nside, W.nside + 1, 2 * W.nside, 4 * W.nside - 9):
        f, n_in = [int(x[0]) for x in hp.ring_info(W.nside, np.array([ring]))[:2]]
        samples.append(np.arange(f + n_in // 7, f + n_in // 7 + 32))
    pix = np.concatenate(samples)
    d = wl.random_deflection(pix.size, 4343)
    tv = kr.displace(W.nside, pix, d)
    rings = np.unique(np.concatenate([hp.pix2ring(W.nside, s[s >= 0])[0]
                                      for s in (fc.stencil(W.nside, tv, 1), fc.stencil(W.nside, tv, 2))]))
    alm = wl.draw_alm(cl, W.seed_map)
    bp, bv = sht.synth_rings(W.nside, rings, W.lmax, alm, spin=2)
    m = np.zeros((W.npix, 2))
    m[bp, 0] = bv.real
    m[bp, 1] = bv.imag
    return W, cl, bb, pix, d, m, float(np.sqrt(np.mean(np.abs(bv) ** 2)))


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("y", [1, 2])
def test_fullsize_4096_qu_sampled(fl, torch, qu4096, y, precision):
    # the whole-sky Nside 4096 Q/U lensing call with the paper stencil; sampled
    # outputs against the oracle's class route and per-target solve
    W, cl, bb, pix, d, m, sigma = qu4096
    defl = torch.zeros((W.npix, 2), dtype=torch.float64, device="cuda")
    defl[torch.from_numpy(pix).cuda()] = torch.from_numpy(d).cuda()
    plan = fl.PaperPlan(W.nside, cl, y, precision, spin=2, cl_bb=bb)
    out, var = plan.lens(torch.from_numpy(m).cuda(), defl)
    torch.cuda.synchronize()
    o = to_host(out)[pix]
    v = o[:, 0] + 1j * o[:, 1]
    s2 = to_host(var)[pix]
    assert plan.info()["window"] == 0
    plan.close()
    tab, x0, _, _ = _spin2_table(cl, bb, W.nside, y)
    rv, rs2, idx, tv = fc.paper_lens(W.nside, y, m, d, pix, tab, x0, classes=True, spin=2)
    ov, os2 = _spin2_solve_route(W.nside, m, tv, idx, tab, x0)
    for a_v, a_s2 in ((rv, rs2), (ov, os2)):
        assert np.max(np.abs(v - a_v)) <= TOL[precision] * sigma
        assert np.max(np.abs(s2 - a_s2)) <= TOL[precision] * x0


# ------------------------------------------------------- augmented spin 2
@pytest.mark.parametrize("nside,lmax,y", [(2, 12, 1), (8, 16, 1), (32, 64, 1), (16, 32, 2), (32, 64, 2)])
def test_augmented_lens_parity(fl, torch, nside, lmax, y):
    # the widely linear (xi+, xi-) estimator on the paper stencil: the class's real
    # 2K x 2K factor (D L^-1 D for the southern classes) against the oracle's
    # augmented class route and its per-target augmented solve
    cl, bb, m, sigma = _spin2_inputs(nside, lmax, 700 + nside + y)
    npix = hp.npix(nside)
    defl = wl.random_deflection(npix, 701 + nside, rms=0.5 * _pixel_size(nside))
    plan = fl.PaperPlan(nside, cl, y, "fp64", spin=2, cl_bb=bb, augmented=True)
    assert plan.info()["flags"] == fl.FLINTS_SPIN2_AUGMENTED
    st = torch.empty(npix, dtype=torch.uint8, device="cuda")
    out, var = plan.lens(torch.from_numpy(m).cuda(), torch.from_numpy(np.ascontiguousarray(defl)).cuda(), status=st)
    torch.cuda.synchronize()
    o = to_host(out)
    v = o[:, 0] + 1j * o[:, 1]
    s2 = to_host(var)
    t_max, n = fc.paper_grid_rule(cl, nside, y, bb)
    tp, tm, x0 = xi.spin2_tables(cl, bb, t_max, n)
    rv, rs2, idx, tv = fc.paper_lens(nside, y, m, defl, np.arange(npix), tp, x0, classes=True, spin=2, f_minus=tm)
    cnt = np.sum(idx >= 0, axis=1)
    ov = np.empty(npix, dtype=np.complex128)
    os2 = np.empty(npix)
    for k in np.unique(cnt):
        rows = np.nonzero(cnt == k)[0]
        stn = np.stack([r[r >= 0] for r in idx[rows]])
        ov[rows], os2[rows], _ = kr.estimate(nside, 2, m, tv[rows], stn, tp, x0, f_minus=tm)
    for a_v, a_s2 in ((rv, rs2), (ov, os2)):
        assert np.max(np.abs(v - a_v)) <= TOL["fp64"] * sigma
        assert np.max(np.abs(s2 - a_s2)) <= TOL["fp64"] * x0
    assert not np.any(to_host(st) & (fl.ST_WINDOW | fl.ST_FAILED))


def test_augmented_supersample_ragged(fl, torch):
    nside, nout, y = 16, 32, 2
    cl, bb, m, sigma = _spin2_inputs(nside, 2 * nside, 801)
    plan = fl.PaperPlan(nside, cl, y, "fp64", spin=2, cl_bb=bb, augmented=True)
    first, count = 333, 1701
    out, var = plan.supersample(torch.from_numpy(m).cuda(), nout, first=first, count=count)
    torch.cuda.synchronize()
    o = to_host(out)
    t_max, n = fc.paper_grid_rule(cl, nside, y, bb)
    tp, tm, x0 = xi.spin2_tables(cl, bb, t_max, n)
    rv, rs2, _, _ = fc.paper_supersample(nside, nout, y, m, np.arange(first, first + count), tp, x0, classes=True,
                                         spin=2)
    # the Hermitian and augmented estimates differ (B != E): check against the augmented route
    tv = hp.pix2vec(nout, np.arange(first, first + count))
    av, as2, _ = fc.class_estimate(nside, y, m, tv, tp, x0, spin=2, f_minus=tm)
    assert np.max(np.abs(o[:, 0] + 1j * o[:, 1] - av)) <= TOL["fp64"] * sigma
    assert np.max(np.abs(to_host(var) - as2)) <= TOL["fp64"] * x0
    assert np.max(np.abs(av - rv)) > 1e-6 * sigma  # the two estimators are distinct here
