"""The seeded input generators (workloads/) follow the recipe they state: the
analytic spectra, the normalisation of the lensing potential to a 2.5 arcmin
rms deflection, Gaussian a_lm with the variance C_l, per-pixel deflections,
the batched and serving mixes, and the storage-free hashed maps."""
import math

import numpy as np
import pytest

import workloads as wl


def test_spectra_closed_forms():
    cl = wl.cl_tt(4096, 2500.0)
    assert cl[0] == cl[1] == 0.0
    for ell in (2, 10, 1000, 4096):
        assert cl[ell] == pytest.approx(1e3 / (ell * (ell + 1)) * math.exp(-(ell / 2500.0) ** 2), rel=1e-15)
    np.testing.assert_array_equal(wl.cl_ee(4096, 2500.0), 0.05 * cl)
    ee, bb = wl.C3.cl()
    assert np.all(bb == 0.0) and ee.size == 4097
    tt, none = wl.C1.cl()
    assert none is None and tt[100] == pytest.approx(1e3 / (100 * 101) * math.exp(-1.0), rel=1e-15)


@pytest.mark.parametrize("lmax", [128, 4096])
def test_lensing_potential_gives_the_stated_deflection_rms(lmax):
    c = wl.cl_phiphi(lmax)
    ell = np.arange(lmax + 1)
    assert c[0] == c[1] == 0.0
    assert c[3] / c[2] == pytest.approx((2 / 3) ** 4, rel=1e-14)  # proportional to l^-4
    power = np.sum((2 * ell + 1) / (4 * math.pi) * ell * (ell + 1) * c)
    assert math.sqrt(power) == pytest.approx(2.5 * math.pi / (180 * 60), rel=1e-13)


def test_alm_are_gaussian_with_variance_cl():
    lmax = 600
    cl = wl.cl_tt(lmax, 400.0)
    alm = wl.draw_alm(cl, 9)
    assert np.array_equal(alm, wl.draw_alm(cl, 9)) and not np.array_equal(alm, wl.draw_alm(cl, 10))
    assert np.all(np.triu(alm, 1) == 0) and np.all(alm[:, 0].imag == 0) and np.all(alm[:2] == 0)
    ell = np.arange(2, lmax + 1)
    # E|a_l0|^2 = C_l and E|a_lm|^2 = C_l for m > 0: the usual estimator is unbiased
    chat = (np.abs(alm[ell, 0]) ** 2 + 2 * np.sum(np.abs(alm[ell, 1:]) ** 2, axis=1)) / (2 * ell + 1)
    ratio = chat / cl[ell]
    sd = math.sqrt(np.mean(2.0 / (2 * ell + 1)) / ell.size)  # standard error of the mean ratio
    assert abs(np.mean(ratio) - 1.0) < 4 * sd
    # real and imaginary parts of m > 0 carry C_l/2 each
    re = np.concatenate([alm[l, 1:l + 1].real / math.sqrt(cl[l]) for l in ell])
    im = np.concatenate([alm[l, 1:l + 1].imag / math.sqrt(cl[l]) for l in ell])
    assert np.var(re) == pytest.approx(0.5, abs=0.01) and np.var(im) == pytest.approx(0.5, abs=0.01)


def test_deflections_and_pixel_samples():
    d = wl.random_deflection(200_000, 1)
    assert d.shape == (200_000, 2)
    assert math.sqrt(np.mean(np.sum(d ** 2, axis=1))) == pytest.approx(wl.DEFLECTION_RMS, rel=0.01)
    assert np.array_equal(d, wl.random_deflection(200_000, 1))
    p = wl.sample_pixels(12 * 64 * 64, 5000, 3)
    assert p.dtype == np.int64 and p.size == 5000 and np.all(np.diff(p) > 0)
    assert p[0] >= 0 and p[-1] < 12 * 64 * 64
    assert wl.sample_pixels(12, 100, 3).size == 12  # capped at the map size


def test_batched_mix():
    maps = wl.batched_maps(64)
    assert len(maps) == 64 and len({m.name for m in maps}) == 64
    assert {m.nside for m in maps} == {256, 512, 1024, 2048}
    assert {m.K for m in maps} == {16, 24, 32, 48} and {m.spin for m in maps} == {0, 2}
    for m in maps:
        assert m.lmax == min(2 * m.nside, 4096) and m.l_damp == pytest.approx(0.61 * m.lmax)
    assert [m.nside for m in wl.batched_maps(64)] == [m.nside for m in maps]  # seeded


def test_serving_stream():
    jobs = wl.job_stream(4000, rate_hz=5.0, seed=500)
    t = np.array([j.arrival_s for j in jobs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.mean(gaps) == pytest.approx(0.2, rel=0.06)  # Poisson: exponential gaps of mean 1/rate
    assert np.std(gaps) == pytest.approx(0.2, rel=0.08)
    for j in jobs:
        npix = 12 * j.nside * j.nside
        assert j.nside in (512, 1024, 2048, 4096) and j.spin in (0, 2) and j.K in (16, 32)
        assert 1e4 <= j.count <= min(npix, 1e8) and 0 <= j.first and j.first + j.count <= npix
    # counts log-uniform in [1e4, 1e8] before the cap: uncapped ones fill each decade alike
    big = [j for j in jobs if j.nside == 4096]  # Npix = 2.0e8 > 1e8: never capped
    dec = np.floor(np.log10([j.count for j in big]))
    share = np.bincount(dec.astype(int), minlength=9)[4:8] / len(big)
    assert np.all(np.abs(share - 0.25) < 0.05), share


def test_hashed_maps_are_storage_free_and_standard_normal():
    idx = np.arange(1_000_000, dtype=np.int64) * 197 + 12345
    v = wl.hashed_normal(idx, 6)
    assert abs(np.mean(v)) < 0.005 and np.std(v) == pytest.approx(1.0, abs=0.005)
    np.testing.assert_array_equal(wl.hashed_normal(idx[::7], 6), v[::7])  # any subset, same values
    two = wl.hashed_normal(idx[:1000], 6, 2)
    assert two.shape == (1000, 2) and abs(np.corrcoef(two[:, 0], two[:, 1])[0, 1]) < 0.1
    m = wl.HashedMap(12 * 4096 * 4096, 6, 2)
    np.testing.assert_array_equal(m[idx[:10]], two[:10])
    np.testing.assert_array_equal(m[idx[:10], 1], two[:10, 1])
    assert not np.array_equal(wl.hashed_normal(idx[:100], 7), v[:100])
