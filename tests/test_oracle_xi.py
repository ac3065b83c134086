"""Pins of the oracle's correlation functions (Eq. correlation_func, Eq. spins_correl,
Appendix B) against closed forms, scipy special functions and identities."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import xi
from tests.wigner_ref import wigner_d
import workloads as wl

RNG = np.random.default_rng(1234)


def test_wigner_reference_small_cases():
    b = np.linspace(0.1, 3.0, 7)
    c, s = np.cos(b), np.sin(b)
    # textbook d^1 and d^2 entries
    np.testing.assert_allclose(wigner_d(1, 1, 0, b), -s / math.sqrt(2), rtol=0, atol=1e-15)
    np.testing.assert_allclose(wigner_d(1, 0, 1, b), s / math.sqrt(2), rtol=0, atol=1e-15)
    np.testing.assert_allclose(wigner_d(1, 1, 1, b), (1 + c) / 2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(wigner_d(2, 2, 2, b), ((1 + c) / 2) ** 2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(wigner_d(2, 2, -2, b), ((1 - c) / 2) ** 2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(wigner_d(2, 0, 0, b), (3 * c * c - 1) / 2, rtol=0, atol=1e-15)


def test_xi0_at_zero_is_spectrum_sum():
    # P_l(1) = 1 so xi(0) = sum (2l+1) C_l / 4 pi (Eq. correlation_func at cos = 1)
    cl = wl.cl_tt(128, 100.0)
    ell = np.arange(129)
    expect = np.sum((2 * ell + 1) * cl) / (4 * math.pi)
    got = xi.xi0_direct(cl, np.zeros(1))[0]
    assert abs(got - expect) <= 1e-14 * expect


@pytest.mark.parametrize("ell", [0, 1, 2, 3, 7, 40, 200])
def test_xi0_single_multipole_is_legendre(ell):
    cl = np.zeros(ell + 1)
    cl[ell] = 1.0
    t = np.concatenate([[0.0, 1e-9, 1e-6], RNG.uniform(0, 4, 20)])
    got, dgot = xi.xi0_direct(cl, t, deriv=True)
    x = 1 - t / 2
    ref = (2 * ell + 1) / (4 * math.pi) * eval_legendre(ell, x)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * (2 * ell + 1))
    # derivative against a central difference in t
    h = 1e-6
    fd = (xi.xi0_direct(cl, t[3:] + h) - xi.xi0_direct(cl, t[3:] - h)) / (2 * h)
    np.testing.assert_allclose(dgot[3:], fd, rtol=1e-5, atol=1e-7 * (2 * ell + 1) * (ell + 1) ** 2)
    # closed-form slope at t = 0: d/dt P_l(1 - t/2) = -l(l+1)/4
    assert abs(dgot[0] - (-(2 * ell + 1) / (4 * math.pi) * ell * (ell + 1) / 4)) <= 1e-12 * max(1, ell * ell * ell)


def test_xi0_small_angle_no_cancellation():
    # near t = 0 the u-form recurrence must agree with an exact series of P_l(1-u):
    # P_l(1-u) = 1 - l(l+1)/2 u + (l-1)l(l+1)(l+2)/16 u^2 - ...
    ell = 4000
    cl = np.zeros(ell + 1)
    cl[ell] = 1.0
    u = 1e-12
    got = xi.xi0_direct(cl, np.array([2 * u]))[0] * 4 * math.pi / (2 * ell + 1)
    series = 1 - ell * (ell + 1) / 2 * u + (ell - 1) * ell * (ell + 1) * (ell + 2) / 16 * u * u
    assert abs(got - series) < 1e-15


def test_delta_columns_unitary_and_symmetric():
    L = 60
    for m2 in (0, 1, 2):
        D = xi.delta_column(L, m2)
        for ell in range(m2, L + 1):
            col = D[ell, L - ell: L + ell + 1]
            assert abs(np.sum(col * col) - 1.0) < 1e-13  # rows of a unitary matrix
            # Delta^l_{-u,m2} = (-1)^{l+m2} Delta^l_{u,m2}
            np.testing.assert_allclose(col[::-1], (-1) ** (ell + m2) * col, rtol=0, atol=1e-14)


@pytest.mark.parametrize("m1,m2", [(0, 0), (1, 1), (1, -1), (2, 2), (2, -2)])
def test_appendix_b_route_matches_jacobi(m1, m2):
    L = 40
    beta = np.concatenate([[0.0, 1e-4], RNG.uniform(0, math.pi, 9)])
    d = xi.wigner_d_fourier(L, m1, m2, beta)
    for ell in range(max(abs(m1), abs(m2)), L + 1):
        np.testing.assert_allclose(d[ell], wigner_d(ell, m1, m2, beta), rtol=0, atol=2e-13)  # about 2.5e-15 l: 1e-13 at l = 40 near b = 0, pi


@pytest.mark.parametrize("ell", [2, 3, 10, 37])
def test_xi2_single_multipole(ell):
    cl = np.zeros(ell + 1)
    cl[ell] = 1.0
    t = np.concatenate([[0.0, 1e-8], RNG.uniform(0, 4, 10)])
    beta = 2 * np.arcsin(np.sqrt(t) / 2)
    xp, xm, dxp, dxm = xi.xi2_direct(cl, None, t, deriv=True)
    w = (2 * ell + 1) / (4 * math.pi)
    np.testing.assert_allclose(xp, w * wigner_d(ell, 2, 2, beta), rtol=0, atol=1e-14 * (2 * ell + 1))
    np.testing.assert_allclose(xm, w * wigner_d(ell, 2, -2, beta), rtol=0, atol=1e-14 * (2 * ell + 1))
    h = 1e-7
    tt = t[2:]
    fdp = (xi.xi2_direct(cl, None, tt + h)[0] - xi.xi2_direct(cl, None, tt - h)[0]) / (2 * h)
    np.testing.assert_allclose(dxp[2:], fdp, rtol=1e-5, atol=1e-6 * w * ell * ell)
    # closed-form slope at 0: d^l_22 ~ 1 - (l(l+1) - 4) b^2 / 4 and t ~ b^2
    assert abs(dxp[0] - (-w * (ell * (ell + 1) - 4) / 4)) < 1e-10 * w * ell * ell


@pytest.mark.parametrize("ell", [1, 2, 7, 31])
def test_xi1_single_multipole(ell):
    # spin 1: xi+ = (2l+1)/4pi d^l_{11}, xi- = (2l+1)/4pi d^l_{1,-1} (Jacobi closed forms)
    cl = np.zeros(ell + 1)
    cl[ell] = 1.0
    t = np.concatenate([[0.0, 1e-8], RNG.uniform(0, 4, 10)])
    beta = 2 * np.arcsin(np.sqrt(t) / 2)
    xp, xm, dxp, dxm = xi.xi1_direct(cl, None, t, deriv=True)
    w = (2 * ell + 1) / (4 * math.pi)
    np.testing.assert_allclose(xp, w * wigner_d(ell, 1, 1, beta), rtol=0, atol=1e-14 * (2 * ell + 1))
    np.testing.assert_allclose(xm, w * wigner_d(ell, 1, -1, beta), rtol=0, atol=1e-14 * (2 * ell + 1))
    h = 1e-7
    tt = t[2:]
    fdm = (xi.xi1_direct(cl, None, tt + h)[1] - xi.xi1_direct(cl, None, tt - h)[1]) / (2 * h)
    np.testing.assert_allclose(dxm[2:], fdm, rtol=1e-5, atol=1e-6 * w * ell * ell)
    # closed-form slope at 0: d^l_11 ~ 1 - (l(l+1) - 1) b^2 / 4 and t ~ b^2
    assert abs(dxp[0] - (-w * (ell * (ell + 1) - 1) / 4)) < 1e-10 * w * max(ell * ell, 1)


def test_xi1_zero_lag():
    cl = wl.cl_phiphi(200) * np.arange(201) * np.arange(1, 202)  # deflection E spectrum l(l+1) C^phiphi
    xp, xm = xi.xi1_direct(cl, None, np.zeros(1))
    ell = np.arange(201)
    assert abs(xp[0] - np.sum((2 * ell + 1) * cl) / (4 * math.pi)) < 1e-13 * xp[0]
    assert abs(xm[0]) < 1e-14 * xp[0]  # d^l_{1,-1}(0) = 0
    # the deflection variance is the 2.5 arcmin rms of the workloads
    assert abs(math.sqrt(xp[0]) - wl.DEFLECTION_RMS) < 1e-3 * wl.DEFLECTION_RMS


def test_xi2_zero_lag():
    cl = wl.cl_ee(300, 180.0)
    bb = 0.3 * cl
    xp, xm = xi.xi2_direct(cl, bb, np.zeros(1))
    ell = np.arange(301)
    assert abs(xp[0] - np.sum((2 * ell + 1) * (cl + bb)) / (4 * math.pi)) < 1e-13 * xp[0]
    assert abs(xm[0]) < 1e-14 * xp[0]  # d^l_{2,-2}(0) = 0


def test_hermite_table_reproduces_cubics():
    a, b, c, d = 0.3, -1.7, 2.2, -0.9
    n, tmax = 17, 2.5
    nodes = np.arange(n + 1) * tmax / n
    tab = xi.HermiteTable(tmax, n, a + b * nodes + c * nodes ** 2 + d * nodes ** 3,
                          b + 2 * c * nodes + 3 * d * nodes ** 2)
    t = RNG.uniform(0, tmax, 200)
    np.testing.assert_allclose(tab(t), a + b * t + c * t ** 2 + d * t ** 3, rtol=0, atol=1e-13)


def test_table_accuracy_c1_spectrum():
    cl = wl.cl_tt(128, 100.0)
    tmax = 4 * (1.35 * math.sqrt(16 / 3.0) / 64) ** 2
    tab, x0 = xi.spin0_table(cl, tmax, 256)  # a quarter of the grid rule's intervals
    t = RNG.uniform(0, tmax, 500)
    # cubic Hermite error h^4/384 max|f''''| at 256 intervals: measured 5.2e-10
    np.testing.assert_allclose(tab(t), xi.xi0_direct(cl, t) / x0, rtol=0, atol=1e-9)
    assert tab.f[0] == 1.0


@pytest.mark.parametrize("name,cl,K,nside", [
    ("c1", wl.cl_tt(128, 100.0), 16, 64),
    ("c2", wl.cl_tt(4096, 2500.0), 32, 2048),
    ("c3", wl.cl_ee(4096, 2500.0), 32, 4096),
])
def test_grid_rule_meets_tolerance(name, cl, K, nside):
    t_max, n = xi.grid_rule(cl, K, nside)
    assert n & (n - 1) == 0 and 64 <= n <= 65536
    t = np.linspace(0, t_max, 301)[1:]
    t = t - 0.37 * t_max / n  # off-node points
    if name == "c3":
        tp, _, _ = xi.spin2_tables(cl, None, t_max, n)
        ref = xi.xi2_direct(cl, None, t)[0] / xi.xi2_direct(cl, None, np.zeros(1))[0][0]
        np.testing.assert_allclose(tp(t), ref, rtol=0, atol=1e-10)
    else:
        tab, x0 = xi.spin0_table(cl, t_max, n)
        np.testing.assert_allclose(tab(t), xi.xi0_direct(cl, t) / x0, rtol=0, atol=1e-10)
