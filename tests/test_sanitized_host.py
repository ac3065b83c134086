"""The library's CUDA sources under the sanitizers (tests/host_compile.SANITIZE).

First the address sanitizer with the bounds, shift and signed-overflow checks,
through the host emulation of
tests/cuda_host.py with device allocations and dynamic shared memory of exactly the
requested size and filled with 0xff bytes (device memory is not cleared): an
access past a buffer, a static shared array's row or the requested dynamic shared
memory, a read of memory nobody wrote that changes a result, or a plan whose
allocations flints_free does not return, fails these tests (any sanitizer finding
ends the run with an error).  A GPU would report such an access as a fault, or
not at all.  One script per C API (K-nearest with batches and the no-allocation
call, the tabulated route, the synthesis), results against the oracle.  Then the
thread sanitizer over the same kernels, as the race check (a report fails the
run)."""
import numpy as np
import pytest

import workloads as wl
from oracle import faces as fc
from oracle import healpix as hp
from oracle import kriging as kr
from oracle import sht
from oracle import xi
from tests import cuda_host as ch
from tests import host_compile as hc
from tests import test_api_host as A
from tests import test_paper_host as P
from tests import test_synth_host as S


@pytest.fixture(scope="module")
def builds(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    from concurrent.futures import ThreadPoolExecutor

    d = tmp_path_factory.mktemp("sanitized")
    jobs = {"api": (A.FILES, A.DRIVER),
            "paper": (["common.cuh", "lens.cuh", "paper_geom.cuh", "xi_table.cu", "paper.cu"], P.DRIVER),
            "synth": (["common.cuh", "synth.cu"], S.DRIVER)}
    with ThreadPoolExecutor(2 * len(jobs)) as pool:  # six compiler processes at once
        fut = {(k, san): pool.submit(ch.build, d, f"{k}_{san}", files, drv, san)
               for k, (files, drv) in jobs.items() for san in ("address", "thread")}
        out = {key: f.result() for key, f in fut.items()}
    return {k: out[(k, "address")] for k in jobs} | {"tsan_" + k: out[(k, "thread")] for k in jobs}


def test_k_nearest_api_under_the_sanitizers(builds):
    nside, lmax = 8, 16
    npix = hp.npix(nside)
    pix = np.arange(40, 140)
    cases = [(0, 16, 0, 0), (2, 32, 1, 0), (2, 24, 0, 1), (0, 48, 1, 4)]  # spin, K, precision, flags
    s = A.Session(builds["api"])
    refs = []
    for k, (spin, K, prec, flags) in enumerate(cases, start=1):
        cl, bb, m, sigma = A._sky(spin, nside, lmax, 30 + k)
        if flags & 1:
            bb = 0.3 * cl
        defl = wl.random_deflection(npix, 40 + k, rms=0.5 * np.sqrt(4 * np.pi / npix))[pix]
        weight = np.abs(cl) + (np.abs(bb) if bb is not None else 0.0)
        t_max, n = xi.grid_rule(weight, K, nside)
        if spin == 0:
            tp, x0 = xi.spin0_table(cl, t_max, n)
            tm = None
        else:
            tp, tm, x0 = xi.spin2_tables(cl, bb, t_max, n)
        ref = kr.lens(nside, K, spin, m, defl, pix, tp, x0, f_minus=tm if flags & 1 else None)
        refs.append((ref, sigma, x0, prec, flags))
        s.plan(k, nside, cl, bb, spin, K, prec, flags)
        s.map(k, nside, np.arange(npix), m)
        s.lens(k, pix[0], pix.size, k, defl)
    d1 = wl.random_deflection(npix, 99, rms=0.5 * np.sqrt(4 * np.pi / npix))
    s.batch([(1, 0, 100, 1, d1[:100]), (2, 700, 68, 2, d1[700:768])], obj=(2, 5))
    s.stencil(1, 0, 64, d1[:64])
    s.super(2, 16, 5, 100, 2)
    cl, _, _, _ = A._sky(2, nside, lmax, 32)
    s.noalloc(nside, cl, None, 2, 32, 1, 10, 100, 2, d1[10:110])
    s.reject(1, 2, 3)
    s.nreject()
    s.table(2, 0)
    s.table(3, 1)  # xi- of the augmented plan, into host buffers of exactly n + 1 values
    res = s.run()
    for k, (ref, sigma, x0, prec, flags) in enumerate(refs):
        st, v, var = res[3 * k + 2]
        tol = 1e-9 if prec == 0 else 1e-6
        ref_v = ref.value if np.iscomplexobj(ref.value) else ref.value + 0j
        assert np.all(st & 8 == 0)
        assert np.max(np.abs(v - ref_v)) <= tol * sigma, k
        if flags & 4:  # FLINTS_NO_VARIANCE: the buffer is left as it was
            assert np.all(np.isnan(var))
        else:
            assert np.max(np.abs(var - ref.variance)) <= tol * x0, k
    # the later calls ran to completion with their results (their values are checked
    # against the oracle by the unsanitized tests)
    assert [len(r[0]) for r in res[12]] == [100, 68] and len(res[13][0]) == 64 and len(res[14][0]) == 100
    assert len(res[15][0]) == 100
    assert res[16][-1] == "untouched 1" and res[17][-1] == "untouched 1"
    assert res[18][0][0] == 1.0 and res[19][0][0] == 0.0  # xi+(0)/xi+(0), xi-(0)


def test_tabulated_route_under_the_sanitizers(builds):
    nside, lmax = 8, 16
    npix = hp.npix(nside)
    for spin, y, prec, flags in [(0, 1, 0, 0), (0, 2, 1, 0), (2, 1, 1, 0), (2, 2, 0, 1)]:
        cl = wl.cl_tt(lmax, 0.7 * lmax) if spin == 0 else wl.cl_ee(lmax, 0.7 * lmax)
        bb = None if spin == 0 else 0.3 * cl
        if spin == 0:
            m = sht.synth_map(nside, lmax, wl.draw_alm(cl, 50 + y))
            sigma = float(np.std(m))
        else:
            Pm = sht.synth_map(nside, lmax, wl.draw_alm(cl, 50 + y), spin=2, blm=wl.draw_alm(bb, 60 + y))
            m = np.stack([Pm.real, Pm.imag], axis=1)
            sigma = float(np.sqrt(np.mean(np.abs(Pm) ** 2)))
        defl = wl.random_deflection(npix, 70 + y, rms=0.5 * np.sqrt(4 * np.pi / npix))
        t_max, n = fc.paper_grid_rule(cl, nside, y, bb)
        if spin == 0:
            tp, x0 = xi.spin0_table(cl, t_max, n)
            tm = None
        else:
            tp, tm, x0 = xi.spin2_tables(cl, bb, t_max, n)
        rv, rs2, _, _ = fc.paper_lens(nside, y, m, defl, np.arange(npix), tp, x0, classes=True, spin=spin,
                                      f_minus=tm if flags else None)
        head = f"lens {nside} {lmax} {y} {spin} {prec} {flags} {0 if bb is None else 1} "
        body = " ".join(x.hex() for x in cl) + ("" if bb is None else " " + " ".join(x.hex() for x in bb))
        body += " " + " ".join(float(x).hex() for x in np.ravel(m)) + " " + " ".join(
            float(x).hex() for x in np.ravel(defl))
        lines = hc.run(builds["paper"], head + body + "\n").splitlines()
        assert lines[0] == "0", lines[:2]
        rows = [ln.split() for ln in lines[1:]]
        v = np.array([float.fromhex(r[1]) for r in rows])
        if spin:
            v = v + 1j * np.array([float.fromhex(r[3]) for r in rows])
        s2 = np.array([float.fromhex(r[2]) for r in rows])
        tol = 1e-9 if prec == 0 else 1e-6
        assert np.max(np.abs(v - rv)) <= tol * sigma and np.max(np.abs(s2 - rs2)) <= tol * x0, (spin, y, prec)
    out = hc.run(builds["paper"], "reject 8 16 " + " ".join(x.hex() for x in wl.cl_tt(16, 12.0)) + "\n")
    assert out.splitlines()[-1] == "untouched 1 points 0"


def test_synthesis_under_the_sanitizers(builds):
    def flat(a):
        return " ".join(float(x).hex() for x in np.stack([a.real, a.imag], -1).ravel())

    for nside, lmax, prec in [(8, 16, 0), (4, 300, 1)]:
        cl = wl.cl_ee(lmax, 0.7 * lmax)
        e, b = wl.draw_alm(cl, 80 + nside), wl.draw_alm(0.4 * cl, 81 + nside)
        lines = hc.run(builds["synth"], f"synth {nside} {lmax} 2 {prec} 1 {flat(e)} {flat(b)}\n").splitlines()
        assert lines[0] == "0"
        got = np.array([float.fromhex(t) for t in lines[1:]])
        got = got[0::2] + 1j * got[1::2]
        ref = sht.synth_map(nside, lmax, e, spin=2, blm=b)
        assert np.max(np.abs(got - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)) <= (1e-10, 1e-9)[prec]
    assert hc.run(builds["synth"], "reject\n").splitlines()[-1] == "untouched 1"


def test_rare_kernel_branches_under_the_sanitizers(builds):
    """The branches the workloads never take, under the sanitizers: spin-1 plans
    (oracle parity), indefinite stencil covariances (the nugget steps, FP64 failures
    and the mixed kernel's FP64 fallback) and non-finite deflections inside a tile."""
    nside, lmax = 8, 16
    npix = hp.npix(nside)
    first, count = 200, 120
    defl = wl.random_deflection(count, 91) * 8
    pix = np.arange(first, first + count)
    ell = np.arange(lmax + 1.0)
    cl1 = ell * (ell + 1) * wl.cl_phiphi(lmax)
    g = sht.synth_map(nside, lmax, wl.draw_alm(wl.cl_phiphi(lmax), 92), gradient=True)
    t1, n1 = xi.grid_rule(np.abs(cl1), 16, nside)
    tab1, _, x01 = xi.spin1_tables(cl1, None, t1, n1)
    ref1 = kr.lens(nside, 16, 1, g, defl, pix, tab1, x01)
    cl = wl.cl_tt(lmax, 11.0)
    cl[lmax] = -0.0043 * cl[2]  # S + 1.49e-8 I indefinite on some stencils
    m = sht.synth_map(nside, lmax, wl.draw_alm(np.abs(cl), 95))
    d_all = wl.random_deflection(npix, 5) * 8
    d_bad = d_all[:96].copy()
    d_bad[[3, 40, 41], 0] = np.nan
    s = A.Session(builds["api"])
    s.plan(1, nside, cl1, None, 1, 16, 1)  # spin 1, mixed
    s.map(1, nside, np.arange(npix), g)
    s.lens(1, first, count, 1, defl)
    s.plan(2, nside, cl, None, 0, 16, 0)
    s.plan(3, nside, cl, None, 0, 16, 1)
    s.map(2, nside, np.arange(npix), m)
    s.lens(2, 0, npix, 2, d_all)
    s.lens(3, 0, npix, 2, d_all)
    s.lens(3, 0, 96, 2, d_bad)
    res = s.run()
    st, v, var = res[2]
    sigma = float(np.sqrt(np.mean(np.sum(g ** 2, 1))))
    assert np.all(st == 0)
    assert np.max(np.abs(v - ref1.value)) <= 1e-6 * sigma and np.max(np.abs(var - ref1.variance)) <= 1e-6 * x01
    st64, stmx = res[6][0], res[7][0]
    assert np.any(st64 & 1) and np.any(st64 & 8)  # nugget steps taken, and failures
    assert np.array_equal(stmx & (1 | 8), st64 & (1 | 8)) and np.all(stmx[st64 & 1 != 0] & 2)
    stb, vb, _ = res[8]
    assert np.all(stb[[3, 40, 41]] == 32 | 8) and np.all(np.isnan(vb[[3, 40, 41]].real))
    # the other points of those tiles as in the run with finite deflections (NaN where that
    # run failed too)
    np.testing.assert_array_equal(np.delete(vb, [3, 40, 41]), np.delete(res[7][1][:96], [3, 40, 41]))


# ------------------------------------------------------------ data races
def _paper_line(nside, lmax, y, spin, prec, flags, seed):
    npix = hp.npix(nside)
    cl = wl.cl_tt(lmax, 0.7 * lmax) if spin == 0 else wl.cl_ee(lmax, 0.7 * lmax)
    bb = None if spin == 0 else 0.3 * cl
    m = np.random.default_rng(seed).normal(size=npix if spin == 0 else (npix, 2))
    defl = wl.random_deflection(npix, seed + 1, rms=0.5 * np.sqrt(4 * np.pi / npix))
    head = f"lens {nside} {lmax} {y} {spin} {prec} {flags} {0 if bb is None else 1} "
    body = " ".join(x.hex() for x in cl) + ("" if bb is None else " " + " ".join(x.hex() for x in bb))
    return head + body + " " + " ".join(float(x).hex() for x in np.ravel(m)) + " " + " ".join(
        float(x).hex() for x in np.ravel(defl)) + "\n"


def test_no_data_races_in_the_kernels(builds):
    """The thread sanitizer over the emulated blocks (compute-sanitizer's race check
    is not available here): every kernel of the three C APIs -- the lens kernels of
    spin 0, 1, 2 and the augmented estimator, FP64 and mixed, the persistent class
    and batch kernels, the stencil and supersampling modes, the no-allocation call,
    the tabulated route's class-factor and apply kernels, the xi and synthesis
    kernels -- runs without two threads touching the same word, one writing, with
    no barrier between them (a report fails the run).  Removing one __syncwarp of
    the augmented apply kernel is reported."""
    nside, lmax = 8, 16
    npix = hp.npix(nside)
    s = A.Session(builds["tsan_api"])
    plans = [(0, 16, 0, 0), (2, 32, 1, 0), (2, 24, 0, 1), (1, 16, 1, 0), (0, 48, 0, 0)]  # the three factor forms
    for k, (spin, K, prec, flags) in enumerate(plans, 1):
        cl, bb, m, _ = A._sky(0 if spin == 0 else 2, nside, lmax, 20 + k)
        s.plan(k, nside, cl, 0.3 * cl if flags & 1 else bb, spin, K, prec, flags)
        s.map(k, nside, np.arange(npix), m)
        d = wl.random_deflection(npix, 30 + k, rms=0.5 * np.sqrt(4 * np.pi / npix))
        s.lens(k, 5, 40, k, d[5:45])
    d = wl.random_deflection(npix, 40, rms=0.5 * np.sqrt(4 * np.pi / npix))
    s.batch([(1, 0, 40, 1, d[:40]), (2, 300, 40, 2, d[300:340])], obj=(2, 4))
    s.stencil(2, 0, 32, d[:32])
    s.super(1, 16, 7, 40, 1)
    cl, _, _, _ = A._sky(2, nside, lmax, 41)
    s.noalloc(nside, cl, None, 2, 16, 1, 0, 40, 2, d[:40])
    res = s.run()
    assert [len(res[3 * k + 2][0]) for k in range(len(plans))] == [40] * len(plans)
    for spin, y, prec, flags in [(0, 1, 0, 0), (0, 2, 1, 0), (2, 1, 0, 1)]:
        assert hc.run(builds["tsan_paper"], _paper_line(4, 8, y, spin, prec, flags, 50 + y)).startswith("0\n")
    cl = wl.cl_ee(300, 210.0)
    alm = wl.draw_alm(cl, 60)
    flat = " ".join(float(x).hex() for x in np.stack([alm.real, alm.imag], -1).ravel())
    assert hc.run(builds["tsan_synth"], f"synth 4 300 2 1 1 {flat} {flat}\n").startswith("0\n")
