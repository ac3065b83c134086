"""GPU parity on whole small skies: xi tables, stencils (bit-exact indices) and
lensed values/variances of the CUDA path against the FP64 oracle.

Tolerances (parity metric = max |gpu - oracle| / sigma_map for values and
max |gpu - oracle| / xi(0) for variances): FP64 path 1e-9, mixed path 1e-6.
"""

import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
from oracle import kriging as kr
from oracle import sht
from oracle import xi
from tests.gpu_common import (oracle_table, parity_metric, realistic_inputs, require_gpu, to_host,
                              unexplained_mismatches)

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-6}


@pytest.fixture(scope="module")
def fl():
    return require_gpu()


@pytest.fixture(scope="module")
def torch():
    import torch as t

    return t


# ---------------------------------------------------------------- xi tables
@pytest.mark.parametrize("spin,nside,lmax,ld,K", [(0, 64, 128, 100.0, 16), (0, 2048, 4096, 2500.0, 32),
                                                    (2, 4096, 4096, 2500.0, 32), (2, 256, 512, 312.0, 48),
                                                    (1, 2048, 4096, 2500.0, 32), (1, 64, 128, 100.0, 16)])
def test_xi_table_matches_oracle(fl, spin, nside, lmax, ld, K):
    if spin == 1:  # deflection spectrum l(l+1) C^phiphi
        cl = wl.cl_phiphi(lmax) * np.arange(lmax + 1) * np.arange(1, lmax + 2)
    else:
        cl = wl.cl_tt(lmax, ld) if spin == 0 else wl.cl_ee(lmax, ld)
    bb = None if spin == 0 else 0.1 * cl
    plan = fl.Plan(nside, cl, bb, spin=spin, K=K)
    info = plan.info()
    weight = np.abs(cl) if spin == 0 else np.abs(cl) + np.abs(bb)
    t_max, n = xi.grid_rule(weight, K, nside)
    assert info.t_max == t_max and info.n_intervals == n
    nodes = np.arange(n + 1) * (t_max / n)
    f, g = plan.table(0)
    if spin == 0:
        ref, dref = xi.xi0_direct(cl, nodes, deriv=True)
    else:
        xp, xm, dxp, dxm = xi.xis_direct(spin, cl, bb, nodes, deriv=True)
        ref, dref = xp, dxp
        fm, gm = plan.table(1)
        np.testing.assert_allclose(fm, xm / xp[0], rtol=0, atol=2e-11)
        np.testing.assert_allclose(gm * t_max, dxm / xp[0] * t_max, rtol=0, atol=1e-9)
    assert abs(info.xi0 - ref[0]) <= 1e-13 * ref[0]
    # absolute bounds in units of xi(0), slopes in units of the table domain: 10x and
    # more above what the same kernel source gives compiled for the host
    # (tests/test_xi_table_host.py: values 1e-14, slopes up to 1.2e-10 for spin 1,
    # xi- values 2e-12); a slope error e moves an interpolated value by e / n at most
    np.testing.assert_allclose(f, ref / ref[0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(g * t_max, dref / ref[0] * t_max, rtol=0, atol=1e-9)


# ------------------------------------------------------------------ stencil
def _near_tie(nside, targets, K):
    idx, key = kr.knn(nside, targets, K + 1)
    gap = (key[:, K] - key[:, K - 1]) / np.maximum(key[:, K], 1e-300)
    return idx[:, :K], gap < 1e-11


@pytest.mark.parametrize("nside,K", [(64, 16), (64, 48), (16, 24), (128, 32)])
def test_stencil_bit_exact(fl, torch, nside, K):
    npix = hp.npix(nside)
    cl = wl.cl_tt(2 * nside, 1.2 * nside)
    plan = fl.Plan(nside, cl, spin=0, K=K)
    defl = wl.random_deflection(npix, 31 + K) * 2.0 * (64 / nside)
    idx, st = plan.stencil(torch.from_numpy(defl).cuda())
    idx, st = to_host(idx), to_host(st)
    assert np.all(st == 0)
    tv = kr.displace(nside, np.arange(npix), defl)
    ref, tie = _near_tie(nside, tv, K)
    same = np.all(idx == ref, axis=1)
    assert np.all(same | tie), f"{np.sum(~same & ~tie)} stencils differ"
    # where the K-th and (K+1)-th neighbours tie, the GPU set must still be a valid K-nearest set
    for p in np.nonzero(~same)[0]:
        keys = np.sum((hp.pix2vec(nside, idx[p]) - tv[p]) ** 2, axis=1)
        refk = np.sum((hp.pix2vec(nside, ref[p]) - tv[p]) ** 2, axis=1)
        assert abs(keys.max() - refk.max()) <= 1e-12 * refk.max()


def test_stencil_at_pixel_centres_is_the_pixel(fl, torch):
    nside, K = 32, 16
    plan = fl.Plan(nside, wl.cl_tt(64, 40.0), spin=0, K=K)
    npix = hp.npix(nside)
    idx, st = plan.stencil(torch.zeros((npix, 2), dtype=torch.float64, device="cuda"))
    idx = to_host(idx)
    assert np.array_equal(idx[:, 0], np.arange(npix))


# ------------------------------------------------------------- lensed maps
@pytest.fixture(scope="module")
def c1_inputs():
    W = wl.C1
    cl, _ = W.cl()
    alm, m, defl = realistic_inputs(W.nside, W.lmax, 0, cl, W.seed_map, W.seed_phi)
    tab, x0, _, _ = oracle_table(cl, None, 0, W.K, W.nside)
    ref = kr.lens(W.nside, W.K, 0, m, defl, np.arange(W.npix), tab, x0)
    return W, cl, alm, m, defl, ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c1_full_sky_parity(fl, torch, c1_inputs, precision):
    W, cl, alm, m, defl, ref = c1_inputs
    plan = fl.Plan(W.nside, cl, spin=0, K=W.K, precision=precision)
    md, dd = torch.from_numpy(m).cuda(), torch.from_numpy(defl).cuda()
    out = torch.empty(W.npix, dtype=torch.float64, device="cuda")
    var = torch.empty_like(out)
    plan.lens_full(md, dd, out, var)
    torch.cuda.synchronize()
    v, s2 = to_host(out), to_host(var)
    sigma = float(np.std(m))
    assert parity_metric(v, ref.value, sigma) <= TOL[precision]
    assert parity_metric(s2, ref.variance, ref.variance.max() * 0 + plan.info().xi0) <= TOL[precision]
    st = plan.stats()
    assert st["failed"] == 0 and st["window"] == 0
    if precision == "fp64":
        assert st["fallback"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c1_ragged_ranges(fl, torch, c1_inputs, precision):
    W, cl, alm, m, defl, ref = c1_inputs
    plan = fl.Plan(W.nside, cl, spin=0, K=W.K, precision=precision)
    md = torch.from_numpy(m).cuda()
    for first, count in [(0, 1), (777, 45), (W.npix - 33, 33), (12345, 0), (100, 1000)]:
        dd = torch.from_numpy(np.ascontiguousarray(defl[first:first + count])).cuda()
        status = torch.empty(count, dtype=torch.uint8, device="cuda")
        var = torch.empty(count, dtype=torch.float64, device="cuda")
        out, var, status = plan.lens(md, dd, var=var, status=status, first=first, count=count)
        torch.cuda.synchronize()
        if count == 0:
            continue
        sigma = float(np.std(m))
        assert parity_metric(to_host(out), ref.value[first:first + count], sigma) <= TOL[precision]
        assert np.all(to_host(status) & fl.ST_FAILED == 0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("K", [16, 24, 32, 48])
def test_spin2_sky_parity(fl, torch, precision, K):
    nside, lmax = 32, 64
    cl = wl.cl_ee(lmax, 50.0)
    bb = 0.2 * cl
    alm = wl.draw_alm(cl, 41)
    blm = wl.draw_alm(bb, 42)
    P = sht.synth_map(nside, lmax, alm, spin=2, blm=blm)
    m = np.ascontiguousarray(np.stack([P.real, P.imag], axis=1))
    defl = wl.random_deflection(hp.npix(nside), 43) * 8
    tab, x0, _, _ = oracle_table(cl, bb, 2, K, nside)
    ref = kr.lens(nside, K, 2, m, defl, np.arange(hp.npix(nside)), tab, x0)
    plan = fl.Plan(nside, cl, bb, spin=2, K=K, precision=precision)
    out = torch.empty((hp.npix(nside), 2), dtype=torch.float64, device="cuda")
    var = torch.empty(hp.npix(nside), dtype=torch.float64, device="cuda")
    plan.lens_full(torch.from_numpy(m).cuda(), torch.from_numpy(defl).cuda(), out, var)
    torch.cuda.synchronize()
    v = to_host(out)
    sigma = float(np.sqrt(np.mean(P.real ** 2 + P.imag ** 2)))
    assert parity_metric(v[:, 0] + 1j * v[:, 1], ref.value, sigma) <= TOL[precision]
    assert parity_metric(to_host(var), ref.variance, x0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("K,bb_frac", [(16, 0.0), (32, 0.0), (48, 0.0), (32, 0.4)])
def test_spin2_augmented_parity(fl, torch, precision, K, bb_frac):
    # FLINTS_SPIN2_AUGMENTED: the widely linear estimator (xi+ and xi-) against the oracle's
    nside, lmax = 32, 64
    cl = wl.cl_ee(lmax, 50.0)
    bb = bb_frac * cl
    P = sht.synth_map(nside, lmax, wl.draw_alm(cl, 46), spin=2, blm=wl.draw_alm(bb, 47) if bb_frac else None)
    m = np.ascontiguousarray(np.stack([P.real, P.imag], axis=1))
    npix = hp.npix(nside)
    defl = wl.random_deflection(npix, 48) * 8
    weight = np.abs(cl) + np.abs(bb)
    t_max, n = xi.grid_rule(weight, K, nside)
    tp, tm, x0 = xi.spin2_tables(cl, bb, t_max, n)
    ref = kr.lens(nside, K, 2, m, defl, np.arange(npix), tp, x0, f_minus=tm)
    plan = fl.Plan(nside, cl, bb, spin=2, K=K, precision=precision, flags=fl.FLINTS_SPIN2_AUGMENTED)
    out = torch.empty((npix, 2), dtype=torch.float64, device="cuda")
    var = torch.empty(npix, dtype=torch.float64, device="cuda")
    plan.lens_full(torch.from_numpy(m).cuda(), torch.from_numpy(defl).cuda(), out, var)
    torch.cuda.synchronize()
    v = to_host(out)
    sigma = float(np.sqrt(np.mean(P.real ** 2 + P.imag ** 2)))
    assert parity_metric(v[:, 0] + 1j * v[:, 1], ref.value, sigma) <= TOL[precision]
    assert parity_metric(to_host(var), ref.variance, x0) <= TOL[precision]
    assert plan.stats()["failed"] == 0


def test_augmented_flag_needs_spin2(fl, torch):
    with pytest.raises(fl.FlintsError):
        fl.Plan(16, wl.cl_tt(32, 20.0), spin=0, K=16, flags=fl.FLINTS_SPIN2_AUGMENTED)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spin2_rotation_to_target_frame(fl, torch, precision):
    # FLINTS_ROTATE_TO_TARGET: P returned in the frame at n (parallel transport back
    # along the deflection), against the oracle's rotated output
    nside, lmax, K = 32, 64, 32
    cl = wl.cl_ee(lmax, 50.0)
    P = sht.synth_map(nside, lmax, wl.draw_alm(cl, 44), spin=2)
    m = np.ascontiguousarray(np.stack([P.real, P.imag], axis=1))
    npix = hp.npix(nside)
    defl = wl.random_deflection(npix, 45) * 20
    tab, x0, _, _ = oracle_table(cl, None, 2, K, nside)
    ref = kr.lens(nside, K, 2, m, defl, np.arange(npix), tab, x0, rotate=True)
    plain = kr.lens(nside, K, 2, m, defl, np.arange(npix), tab, x0)
    sigma = float(np.sqrt(np.mean(P.real ** 2 + P.imag ** 2)))
    assert parity_metric(ref.value, plain.value, sigma) > 1e-4  # the rotation is not negligible here
    plan = fl.Plan(nside, cl, spin=2, K=K, precision=precision, flags=fl.FLINTS_ROTATE_TO_TARGET)
    out = torch.empty((npix, 2), dtype=torch.float64, device="cuda")
    plan.lens_full(torch.from_numpy(m).cuda(), torch.from_numpy(defl).cuda(), out)
    torch.cuda.synchronize()
    v = to_host(out)
    assert parity_metric(v[:, 0] + 1j * v[:, 1], ref.value, sigma) <= TOL[precision]
    with pytest.raises(fl.FlintsError):
        fl.Plan(nside, wl.cl_tt(lmax, 50.0), spin=0, K=K, flags=fl.FLINTS_ROTATE_TO_TARGET)


def _deflection_field(nside, lmax, seed):
    phi = wl.draw_alm(wl.cl_phiphi(lmax), seed)
    ell = np.arange(lmax + 1)
    cle = wl.cl_phiphi(lmax) * ell * (ell + 1)
    return cle, np.ascontiguousarray(sht.synth_map(nside, lmax, phi, gradient=True))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("K,rotate", [(16, False), (32, False), (48, False), (32, True)])
def test_spin1_deflection_parity(fl, torch, precision, K, rotate):
    # spin 1: a deflection field d = grad phi (P = d_theta + i d_phi) lensed by another
    nside, lmax = 32, 64
    cle, m = _deflection_field(nside, lmax, 55)
    npix = hp.npix(nside)
    defl = wl.random_deflection(npix, 56) * 8
    tab, x0, _, _ = oracle_table(cle, None, 1, K, nside)
    ref = kr.lens(nside, K, 1, m, defl, np.arange(npix), tab, x0, rotate=rotate)
    flags = fl.FLINTS_ROTATE_TO_TARGET if rotate else 0
    plan = fl.Plan(nside, cle, spin=1, K=K, precision=precision, flags=flags)
    out = torch.empty((npix, 2), dtype=torch.float64, device="cuda")
    var = torch.empty(npix, dtype=torch.float64, device="cuda")
    plan.lens_full(torch.from_numpy(m).cuda(), torch.from_numpy(defl).cuda(), out, var)
    torch.cuda.synchronize()
    v = to_host(out)
    sigma = float(np.sqrt(np.mean(np.sum(m ** 2, axis=1))))
    assert parity_metric(v[:, 0] + 1j * v[:, 1], ref.value, sigma) <= TOL[precision]
    assert parity_metric(to_host(var), ref.variance, x0) <= TOL[precision]
    assert plan.stats()["failed"] == 0


@pytest.mark.parametrize("K", [16, 24, 48])
def test_spin0_all_stencil_sizes(fl, torch, K):
    nside, lmax = 32, 64
    cl = wl.cl_tt(lmax, 50.0)
    alm = wl.draw_alm(cl, 51)
    m = sht.synth_map(nside, lmax, alm)
    defl = wl.random_deflection(hp.npix(nside), 52) * 8
    tab, x0, _, _ = oracle_table(cl, None, 0, K, nside)
    ref = kr.lens(nside, K, 0, m, defl, np.arange(hp.npix(nside)), tab, x0)
    for precision in ("fp64", "mixed"):
        plan = fl.Plan(nside, cl, spin=0, K=K, precision=precision)
        out = torch.empty(hp.npix(nside), dtype=torch.float64, device="cuda")
        plan.lens_full(torch.from_numpy(m).cuda(), torch.from_numpy(defl).cuda(), out)
        torch.cuda.synchronize()
        assert parity_metric(to_host(out), ref.value, float(np.std(m))) <= TOL[precision]


@pytest.mark.parametrize("spin", [0, 2])
def test_mixed_fp64_fallback_path(fl, torch, c1_inputs, spin):
    """The FP64 fallback of the mixed path (taken when the double-float factor
    meets a non-positive pivot) rebuilds its geometry from the double-float
    copies; forcing it on every point checks that path against the oracle."""
    if spin == 0:
        W, cl, alm, m, defl, ref = c1_inputs
        nside, K, bb, sigma, x0 = W.nside, W.K, None, float(np.std(m)), None
    else:
        nside, K, lmax = 32, 32, 64
        cl = wl.cl_ee(lmax, 50.0)
        bb = 0.2 * cl
        P = sht.synth_map(nside, lmax, wl.draw_alm(cl, 61), spin=2, blm=wl.draw_alm(bb, 62))
        m = np.ascontiguousarray(np.stack([P.real, P.imag], axis=1))
        defl = wl.random_deflection(hp.npix(nside), 63) * 8
        tab, x0, _, _ = oracle_table(cl, bb, 2, K, nside)
        ref = kr.lens(nside, K, 2, m, defl, np.arange(hp.npix(nside)), tab, x0)
        sigma = float(np.sqrt(np.mean(P.real ** 2 + P.imag ** 2)))
    npix = hp.npix(nside)
    plan = fl.Plan(nside, cl, bb, spin=spin, K=K, precision="mixed", flags=fl.FLINTS_FORCE_FALLBACK)
    out = torch.empty((npix,) if spin == 0 else (npix, 2), dtype=torch.float64, device="cuda")
    var = torch.empty(npix, dtype=torch.float64, device="cuda")
    status = torch.empty(npix, dtype=torch.uint8, device="cuda")
    plan.lens(torch.from_numpy(m).cuda(), torch.from_numpy(defl).cuda(), out, var, status)
    torch.cuda.synchronize()
    v = to_host(out)
    if spin == 2:
        v = v[:, 0] + 1j * v[:, 1]
    # FP64 arithmetic on geometry carried to ~2^-48: well inside the mixed tolerance
    assert parity_metric(v, ref.value, sigma) <= 1e-8
    assert parity_metric(to_host(var), ref.variance, plan.info().xi0) <= 1e-8
    st = to_host(status)
    assert np.all(st & fl.ST_FALLBACK) and not np.any(st & fl.ST_FAILED)
    assert plan.stats()["fallback"] == npix


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("spin", [0, 2])
def test_supersampling_parity(fl, torch, precision, spin):
    # Sec. 2.6: an Nside 32 map predicted at every Nside 64 pixel centre, and a
    # ragged range of an Nside 80 grid (not a power-of-two multiple)
    nside, lmax, K = 32, 64, 32
    if spin == 0:
        cl, bb = wl.cl_tt(lmax, 50.0), None
        m = sht.synth_map(nside, lmax, wl.draw_alm(cl, 81))
        sigma = float(np.std(m))
    else:
        cl = wl.cl_ee(lmax, 50.0)
        bb = 0.3 * cl
        P = sht.synth_map(nside, lmax, wl.draw_alm(cl, 82), spin=2, blm=wl.draw_alm(bb, 83))
        m = np.ascontiguousarray(np.stack([P.real, P.imag], axis=1))
        sigma = float(np.sqrt(np.mean(P.real ** 2 + P.imag ** 2)))
    tab, x0, _, _ = oracle_table(cl, bb, spin, K, nside)
    plan = fl.Plan(nside, cl, bb, spin=spin, K=K, precision=precision)
    md = torch.from_numpy(m).cuda()
    for nout, first, count in [(64, 0, hp.npix(64)), (80, 12345, 4321), (64, 5, 0)]:
        var = torch.empty(count, dtype=torch.float64, device="cuda")
        st = torch.empty(count, dtype=torch.uint8, device="cuda")
        out, var, st = plan.supersample(md, nout, var=var, status=st, first=first, count=count)
        torch.cuda.synchronize()
        if count == 0:
            continue
        ref = kr.supersample(nside, nout, K, spin, m, np.arange(first, first + count), tab, x0)
        v = to_host(out)
        if spin == 2:
            v = v[:, 0] + 1j * v[:, 1]
        # the centres of the finer grid sit symmetrically between source pixels, so the
        # K-th place of a stencil is often an exact tie: such targets are checked against
        # the oracle's estimate on each valid K-nearest set
        bad = unexplained_mismatches(nside, K, spin, m, ref.target, v, to_host(var), ref, tab, x0, sigma,
                                     TOL[precision])
        assert bad == [], f"{len(bad)} targets differ from the oracle beyond ties"
        assert not np.any(to_host(st) & fl.ST_FAILED)


def test_wrong_spin_entry_point_is_an_error(fl, torch):
    plan = fl.Plan(16, wl.cl_tt(32, 20.0), spin=0, K=16)
    z = torch.zeros((hp.npix(16), 2), dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FlintsError):
        fl.api._check(fl.api._lib.flints_lens_spin2(plan._h, z.data_ptr(), z.data_ptr(), z.data_ptr(), None, None))


# ------------------------------------------------------ non-finite inputs
@pytest.mark.parametrize("spin", [0, 2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonfinite_deflections_are_flagged_not_ignored(fl, torch, spin, precision):
    """A NaN or infinite deflection is not a zero deflection: the point gets
    FLINTS_ST_INPUT | FLINTS_ST_FAILED and NaN outputs, the counters count it as
    failed, and every other point is unchanged (oracle parity)."""
    nside, lmax, K = 16, 32, 16
    npix = hp.npix(nside)
    cl = wl.cl_tt(lmax, 24.0) if spin == 0 else wl.cl_ee(lmax, 24.0)
    m = sht.synth_map(nside, lmax, wl.draw_alm(cl, 41), spin=spin)
    if spin == 2:
        m = np.stack([m.real, m.imag], axis=1)
    m = np.ascontiguousarray(m)
    defl = wl.random_deflection(npix, 42) * 4
    bad = np.array([0, 5, 77, npix // 2, npix - 1])
    defl_bad = defl.copy()
    defl_bad[bad[0], 0] = np.nan
    defl_bad[bad[1], 1] = np.inf
    defl_bad[bad[2]] = [-np.inf, 0.0]
    defl_bad[bad[3], 0] = np.nan
    defl_bad[bad[3], 1] = np.nan
    defl_bad[bad[4], 1] = -np.nan
    plan = fl.Plan(nside, cl, spin=spin, K=K, precision=precision)
    plan.reset_stats()
    out, var, st = plan.lens(torch.from_numpy(m).cuda(), torch.from_numpy(defl_bad).cuda(),
                             var=torch.empty(npix, dtype=torch.float64, device="cuda"),
                             status=torch.empty(npix, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    o, v, s = to_host(out), to_host(var), to_host(st)
    if spin == 2:
        o = o[:, 0] + 1j * o[:, 1]
    assert np.all(s[bad] == fl.ST_INPUT | fl.ST_FAILED)
    assert np.all(np.isnan(o[bad])) and np.all(np.isnan(v[bad]))
    good = np.setdiff1d(np.arange(npix), bad)
    assert np.all(s[good] & (fl.ST_INPUT | fl.ST_FAILED) == 0)
    assert plan.stats()["failed"] == bad.size
    tab, x0, _, _ = oracle_table(cl, None, spin, K, nside)
    ref = kr.lens(nside, K, spin, m, defl[good], good, tab, x0)
    sigma = float(np.sqrt(np.mean(np.abs(ref.value) ** 2)))
    assert parity_metric(o[good], ref.value, sigma) <= TOL[precision]
    assert parity_metric(v[good], ref.variance, x0) <= TOL[precision]
    plan.close()


def test_nonfinite_deflections_on_the_tabulated_route(fl, torch):
    """The same rule on the tabulated-inverse route (9-pixel stencil, FP64 and mixed)."""
    nside, lmax = 16, 32
    npix = hp.npix(nside)
    cl = wl.cl_tt(lmax, 24.0)
    m = torch.from_numpy(sht.synth_map(nside, lmax, wl.draw_alm(cl, 43))).cuda()
    defl = wl.random_deflection(npix, 44) * 4
    bad = np.array([3, 100, npix - 2])
    defl_bad = defl.copy()
    defl_bad[bad[0], 0] = np.nan
    defl_bad[bad[1], 1] = np.inf
    defl_bad[bad[2]] = np.nan
    for precision in ("fp64", "mixed"):
        plan = fl.PaperPlan(nside, cl, 1, precision)
        st = torch.empty(npix, dtype=torch.uint8, device="cuda")
        out, var = plan.lens(m, torch.from_numpy(defl_bad).cuda(), status=st)
        ref, _ = plan.lens(m, torch.from_numpy(defl).cuda())
        torch.cuda.synchronize()
        o, s, r = to_host(out), to_host(st), to_host(ref)
        assert np.all(s[bad] & (fl.ST_INPUT | fl.ST_FAILED) == fl.ST_INPUT | fl.ST_FAILED), precision
        assert np.all(np.isnan(o[bad])) and np.all(np.isnan(to_host(var)[bad])), precision
        good = np.setdiff1d(np.arange(npix), bad)
        assert np.all(s[good] & fl.ST_INPUT == 0)
        np.testing.assert_array_equal(o[good], r[good])
        plan.close()


def test_many_calls_of_one_plan_in_flight(fl, torch):
    """A plan's calls take its slots in turn (tile queue and job table): 100 calls
    issued back to back on two streams, without synchronising, wrap the 64 slots and
    give the same results as the calls made one at a time."""
    nside, lmax, K = 16, 32, 16
    npix = hp.npix(nside)
    cl = wl.cl_tt(lmax, 24.0)
    m = torch.from_numpy(sht.synth_map(nside, lmax, wl.draw_alm(cl, 51))).cuda()
    defl = torch.from_numpy(wl.random_deflection(npix, 52) * 4).cuda()
    plan = fl.Plan(nside, cl, spin=0, K=K, precision="mixed")
    n, size = 100, 96
    firsts = [(37 * i) % (npix - size) for i in range(n)]
    ref = []
    for f in firsts:
        o, _, _ = plan.lens(m, defl[f:f + size], first=f, count=size)
        torch.cuda.synchronize()
        ref.append(to_host(o))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [torch.full((size,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(n)]
    torch.cuda.synchronize()
    for i, f in enumerate(firsts):
        plan.lens(m, defl[f:f + size], out=outs[i], first=f, count=size, stream=streams[i & 1])
    torch.cuda.synchronize()
    for i in range(n):
        np.testing.assert_array_equal(to_host(outs[i]), ref[i])
    plan.close()
