"""Pins of the oracle's kriging estimator (Secs. 2.1, 2.2, 2.4, 3.1) against closed
forms, library special cases, brute force and the paper's exact benchmark."""
import math

import numpy as np
import pytest

from oracle import healpix as hp
from oracle import kriging as kr
from oracle import sht
from oracle import xi
from tests.wigner_ref import wigner_d
import workloads as wl

RNG = np.random.default_rng(77)


# ------------------------------------------------------------ displacement
def test_displacement_geodesic():
    nside = 32
    pix = RNG.integers(0, hp.npix(nside), 300)
    defl = RNG.normal(size=(300, 2)) * 3e-3
    defl[:5] = 0.0
    n = hp.pix2vec(nside, pix)
    n2 = kr.displace(nside, pix, defl)
    assert np.array_equal(n2[:5], n[:5])  # zero deflection leaves the centre in place
    np.testing.assert_allclose(np.linalg.norm(n2, axis=1), 1.0, rtol=0, atol=4.5e-16)  # 2 ulp
    # geodesic length equals |d|
    ang = 2 * np.arcsin(np.linalg.norm(n2 - n, axis=1) / 2)
    np.testing.assert_allclose(ang, np.hypot(defl[:, 0], defl[:, 1]), rtol=1e-12, atol=1e-18)
    # initial direction is (d_theta, d_phi) in the local basis
    e_th, e_ph = kr.local_basis(n)
    a = np.sum((n2 - n) * e_th, axis=1)
    b = np.sum((n2 - n) * e_ph, axis=1)
    dl = np.hypot(defl[5:, 0], defl[5:, 1])
    np.testing.assert_allclose(a[5:] / np.hypot(a[5:], b[5:]), defl[5:, 0] / dl, rtol=0, atol=1e-6)
    np.testing.assert_allclose(b[5:] / np.hypot(a[5:], b[5:]), defl[5:, 1] / dl, rtol=0, atol=1e-6)


# ---------------------------------------------------------- linear algebra
def test_cholesky_and_solve_against_numpy():
    P, K = 5, 12
    X = RNG.normal(size=(P, K, K)) + 1j * RNG.normal(size=(P, K, K))
    A = X @ np.conj(np.swapaxes(X, 1, 2)) + K * np.eye(K)
    L, ok = kr.cholesky_batched(A)
    assert ok.all()
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=0, atol=1e-12)
    b = RNG.normal(size=(P, K)) + 1j * RNG.normal(size=(P, K))
    z = kr.forward_solve(L, b)
    np.testing.assert_allclose(np.einsum("pij,pj->pi", L, z), b, rtol=0, atol=1e-12)


def test_nugget_rule_for_indefinite_matrix():
    K = 6
    Q, _ = np.linalg.qr(RNG.normal(size=(K, K)))
    lam = np.array([-3e-6, 1e-9, 0.1, 0.5, 1.0, 2.0])
    S = (Q * lam) @ Q.T
    L, nug = kr.factor_with_nugget(S[None])
    # n = -lambda_min + epsilon (Sec. 2.4), up to the extra epsilon steps rounding may need
    assert 3e-6 + kr.EPS_NUGGET - 1e-12 <= nug[0] <= 3e-6 + 3 * kr.EPS_NUGGET
    np.testing.assert_allclose(L[0] @ L[0].T, S + nug[0] * np.eye(K), rtol=0, atol=1e-14)
    # a positive-definite matrix takes n = epsilon
    _, nug = kr.factor_with_nugget(((Q * np.abs(lam)) @ Q.T + 1e-3 * np.eye(K))[None])
    assert nug[0] == kr.EPS_NUGGET


# ------------------------------------------------------------------ spin 0
@pytest.fixture(scope="module")
def c1_table():
    cl = wl.cl_tt(128, 100.0)
    tmax = 4 * (2.0 * math.sqrt(16 / 3.0) / 64) ** 2
    tab, x0 = xi.spin0_table(cl, tmax, 512)
    return cl, tab, x0


def test_pixel_centre_returns_pixel_value(c1_table):
    # At a pixel centre c = S e_q, so with A = S + n I:
    #   value - y_q = -n (A^-1 y)_q   and   variance = xi(0) n (1 - n (A^-1)_qq)   (closed forms)
    cl, tab, x0 = c1_table
    nside, K = 64, 16
    y = wl.white_map(hp.npix(nside), 1, 11)
    pix = RNG.integers(0, hp.npix(nside), 200)
    res = kr.lens(nside, K, 0, y, np.zeros((200, 2)), pix, tab, x0)
    assert np.all(res.stencil[:, 0] == pix)
    assert np.all(res.variance <= kr.EPS_NUGGET * x0 * (1 + 1e-9))
    assert np.all(res.variance >= 0)
    for p in range(0, 200, 10):
        X = hp.pix2vec(nside, res.stencil[p])
        A = tab(np.sum((X[:, None] - X[None]) ** 2, axis=-1)) + kr.EPS_NUGGET * np.eye(K)
        Ainv = np.linalg.inv(A)
        gap = -kr.EPS_NUGGET * (Ainv @ y[res.stencil[p]])[0]
        assert abs((res.value[p] - y[pix[p]]) - gap) < 1e-6 * abs(gap) + 1e-12
        var = x0 * kr.EPS_NUGGET * (1 - kr.EPS_NUGGET * Ainv[0, 0])
        assert abs(res.variance[p] - var) < 1e-6 * var


def test_weights_match_dense_solve(c1_table):
    cl, tab, x0 = c1_table
    nside, K = 64, 16
    y = wl.white_map(hp.npix(nside), 1, 12)
    pix = RNG.integers(0, hp.npix(nside), 50)
    defl = wl.random_deflection(50, 13) * 5
    res = kr.lens(nside, K, 0, y, defl, pix, tab, x0)
    for p in range(50):
        X = hp.pix2vec(nside, res.stencil[p])
        S = tab(np.sum((X[:, None] - X[None]) ** 2, axis=-1)) + kr.EPS_NUGGET * np.eye(K)
        c = tab(np.sum((X - res.target[p]) ** 2, axis=-1))
        w = np.linalg.solve(S, c)
        assert abs(w @ y[res.stencil[p]] - res.value[p]) < 1e-9 * np.abs(y).max() * np.abs(w).sum()
        assert abs(x0 * (1 - c @ w) - res.variance[p]) < 1e-10 * x0


def test_monopole_limit_weights_sum_to_one():
    # simple kriging does not reproduce constants, but a large monopole C_0 drives the
    # weights towards the ordinary-kriging limit sum w = 1 as O(1/C_0)
    nside, K = 64, 16
    base = wl.cl_tt(128, 100.0)
    tmax = 4 * (2.0 * math.sqrt(16 / 3.0) / 64) ** 2
    pix = RNG.integers(0, hp.npix(nside), 20)
    defl = wl.random_deflection(20, 14) * 5
    gaps = []
    for M in (1e2, 1e4):
        cl = base.copy()
        cl[0] = M * np.sum((2 * np.arange(129) + 1) * base) / (4 * math.pi) * 4 * math.pi
        tab, x0 = xi.spin0_table(cl, tmax, 512)
        ones = np.ones(hp.npix(nside))
        res = kr.lens(nside, K, 0, ones, defl, pix, tab, x0)
        gaps.append(np.max(np.abs(1 - res.value)))
    assert gaps[1] < gaps[0] / 30


# --------------------------------------------------- spin 2 phase convention
def _sY2(ell, m, v):
    th = np.arctan2(np.hypot(v[:, 0], v[:, 1]), v[:, 2])
    ph = np.arctan2(v[:, 1], v[:, 0])
    # Appendix A: sY_lm = (-1)^s sqrt((2l+1)/4pi) e^{i m phi} d^l_{m,-s}(theta), s = 2
    return math.sqrt((2 * ell + 1) / (4 * math.pi)) * np.exp(1j * m * ph) * wigner_d(ell, m, -2, th)


@pytest.mark.parametrize("ell", [2, 3, 5, 8])
def test_spin2_pair_phase_by_addition_theorem(ell):
    a = RNG.normal(size=(40, 3))
    a /= np.linalg.norm(a, axis=1)[:, None]
    b = a + RNG.normal(size=(40, 3)) * 0.3
    b /= np.linalg.norm(b, axis=1)[:, None]
    corr = sum(_sY2(ell, m, a) * np.conj(_sY2(ell, m, b)) for m in range(-ell, ell + 1))
    beta = 2 * np.arcsin(np.linalg.norm(a - b, axis=1) / 2)
    model = (2 * ell + 1) / (4 * math.pi) * wigner_d(ell, 2, 2, beta) * kr.pair_phase(a, b)
    np.testing.assert_allclose(corr, model, rtol=0, atol=1e-13)


def test_spin2_synthesis_matches_harmonics():
    lmax = 6
    v = RNG.normal(size=(15, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    for ell in range(2, lmax + 1):
        for m in range(0, ell + 1):
            E = np.zeros((lmax + 1, lmax + 1), complex)
            E[ell, m] = 0.7 - 0.2j
            got = sht.synth_points(lmax, E, v, spin=2)
            a = -E[ell, m]  # a_{2,lm} = -(E + iB)
            ref = a * _sY2(ell, m, v)
            if m > 0:
                ref = ref + (-(-1) ** m * np.conj(E[ell, m])) * _sY2(ell, -m, v)
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


def test_spin2_frame_covariance():
    # rotating the local frame of every pixel (P_q -> e^{2i psi_q} P_q, covariances
    # rotated alike) leaves the estimate unchanged
    K = 10
    Q, _ = np.linalg.qr(RNG.normal(size=(K, K)) + 1j * RNG.normal(size=(K, K)))
    C = (Q * np.linspace(1e-6, 3, K)) @ np.conj(Q.T)
    c = RNG.normal(size=K) + 1j * RNG.normal(size=K)
    y = RNG.normal(size=K) + 1j * RNG.normal(size=K)
    psi = np.exp(2j * RNG.uniform(0, np.pi, K))

    def est(C, c, y):
        L, _ = kr.factor_with_nugget(C[None])
        zc = kr.forward_solve(L, np.conj(c)[None])[0]
        zy = kr.forward_solve(L, y[None])[0]
        return np.sum(np.conj(zc) * zy)

    v0 = est(C, c, y)
    v1 = est(psi[:, None] * C * np.conj(psi)[None, :], c * np.conj(psi), psi * y)
    assert abs(v0 - v1) < 1e-10 * abs(v0)


# -------------------------------------------- exact benchmark on C1 (spin 0)
@pytest.fixture(scope="module")
def c1_lensed():
    W = wl.C1
    cl, _ = W.cl()
    alm = wl.draw_alm(cl, W.seed_map)
    phi_alm = wl.draw_alm(wl.cl_phiphi(W.lmax), W.seed_phi)
    tmap = sht.synth_map(W.nside, W.lmax, alm)
    defl = sht.synth_map(W.nside, W.lmax, phi_alm, gradient=True)
    pix = np.arange(W.npix)
    tmax = 4 * (2.0 * math.sqrt(W.K / 3.0) / W.nside) ** 2 * 1.5
    tab, x0 = xi.spin0_table(cl, tmax, 1024)
    res = kr.lens(W.nside, W.K, 0, tmap, defl, pix, tab, x0)
    truth = sht.synth_points(W.lmax, alm, res.target)
    return tmap, defl, res, truth, x0


def test_c1_deflection_rms(c1_lensed):
    _, defl, _, _, _ = c1_lensed
    rms = math.sqrt(np.mean(np.sum(defl ** 2, axis=1)))
    assert 0.7 * wl.DEFLECTION_RMS < rms < 1.3 * wl.DEFLECTION_RMS


def test_c1_error_statistics_match_predicted_variance(c1_lensed):
    # Sec. 3.2 / Fig. cmb_exp_error: measured error / predicted sigma ~ N(0, 1)
    tmap, _, res, truth, _ = c1_lensed
    r = (res.value - truth) / np.sqrt(res.variance)
    assert abs(np.mean(r)) < 0.05
    assert 0.9 < np.std(r) < 1.1
    rel = np.sqrt(np.mean((res.value - truth) ** 2) / np.mean(truth ** 2))
    assert rel < 0.2


def test_spin2_error_statistics_match_predicted_variance():
    # spin-2 exact benchmark on an Nside 64 sky: Q/U kriged with the Hermitian
    # xi+ covariance and parallel-transport phases; |error| / sigma ~ unit complex Gaussian
    nside, lmax, K = 64, 128, 16
    cl = wl.cl_ee(lmax, 100.0)
    alm = wl.draw_alm(cl, 21)
    P = sht.synth_map(nside, lmax, alm, spin=2)
    qu = np.stack([P.real, P.imag], axis=1)
    pix = wl.sample_pixels(hp.npix(nside), 4000, 22)
    defl = wl.random_deflection(pix.size, 23)
    tmax = 4 * (2.0 * math.sqrt(K / 3.0) / nside) ** 2 * 1.5
    tp, tm, x0 = xi.spin2_tables(cl, None, tmax, 1024)
    res = kr.lens(nside, K, 2, qu, defl, pix, tp, x0)
    truth = sht.synth_points(lmax, alm, res.target, spin=2)
    r = np.abs(res.value - truth) ** 2 / res.variance
    assert 0.85 < np.mean(r) < 1.15  # E|P - P_hat|^2 = sigma^2 for a circular Gaussian
    rel = np.sqrt(np.mean(np.abs(res.value - truth) ** 2) / np.mean(np.abs(truth) ** 2))
    assert rel < 0.2


@pytest.mark.parametrize("spin", [1, 2])
def test_spin2_pair_phase_factorises_through_the_target(spin):
    # The pair phase equals conj(phase(n', a)) phase(n', b) exp(-isE), E the spherical excess
    # of the triangle (n', a, b): tan(E/2) = n'.(a x b) / (1 + n'.a + a.b + b.n')
    # (Van Oosterom-Strackee).  The CUDA path assembles spin-s covariances this way.
    n = RNG.normal(size=(500, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    for scale in (1e-3, 3e-2, 0.3):
        a = n + RNG.normal(size=(500, 3)) * scale
        a /= np.linalg.norm(a, axis=1)[:, None]
        b = n + RNG.normal(size=(500, 3)) * scale
        b /= np.linalg.norm(b, axis=1)[:, None]
        triple = np.einsum("pi,pi->p", n, np.cross(a, b))
        den = 1 + np.sum(n * a, 1) + np.sum(a * b, 1) + np.sum(b * n, 1)
        x = triple / den
        g = ((1 - 1j * x) ** 2 / (1 + x * x)) ** spin  # exp(-isE) with E = 2 atan(x)
        got = np.conj(kr.pair_phase(n, a, spin)) * kr.pair_phase(n, b, spin) * g
        np.testing.assert_allclose(got, kr.pair_phase(a, b, spin), rtol=0, atol=1e-12)


# ------------------------------------------------- supersampling (Sec. 2.6)
def test_supersampling_error_statistics():
    # An Nside 32 map band-limited at lmax 64 predicted at every Nside 64 pixel
    # centre (Table 1's experiment, scaled down): the targets are the finer grid's
    # centres and measured error / predicted sigma ~ N(0, 1) against the harmonic sum.
    nside, lmax, K = 32, 64, 16
    cl = wl.cl_tt(lmax, 50.0)
    alm = wl.draw_alm(cl, 71)
    m = sht.synth_map(nside, lmax, alm)
    pix = np.arange(hp.npix(2 * nside))
    tmax = 4 * (2.0 * math.sqrt(K / 3.0) / nside) ** 2 * 1.5
    tab, x0 = xi.spin0_table(cl, tmax, 1024)
    res = kr.supersample(nside, 2 * nside, K, 0, m, pix, tab, x0)
    np.testing.assert_array_equal(res.target, hp.pix2vec(2 * nside, pix))
    truth = sht.synth_points(lmax, alm, res.target)
    r = (res.value - truth) / np.sqrt(res.variance)
    assert abs(np.mean(r)) < 0.05
    assert 0.9 < np.std(r) < 1.1
    # predicted precision (Table 1's column: sqrt(mean sigma^2) / sigma_map) matches the measured one
    pred = math.sqrt(np.mean(res.variance)) / np.std(m)
    meas = math.sqrt(np.mean((res.value - truth) ** 2)) / np.std(m)
    assert 0.85 < meas / pred < 1.15


# ------------------------------------- rotation to the target frame (Sec. 3.1)
def _rodrigues(v, axis, ang):
    k = axis / np.linalg.norm(axis, axis=-1, keepdims=True)
    c, s = np.cos(ang)[..., None], np.sin(ang)[..., None]
    return v * c + np.cross(k, v) * s + k * np.sum(k * v, axis=-1, keepdims=True) * (1 - c)


def test_transport_phase_matches_rotation_along_the_geodesic():
    # Parallel transport along a great circle is the rotation about that circle's
    # axis taking n' to n.  A polarisation of orientation psi at n' (from e_theta
    # towards e_phi, P = |P| exp(2i psi)) arrives at n with orientation chi; the
    # oracle's rotation must give exp(2i chi) = exp(2i psi) pair_phase(n, n').
    n = RNG.normal(size=(400, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    for scale in (1e-4, 3e-3, 0.2):
        defl = RNG.normal(size=(400, 2)) * scale
        e_th, e_ph = kr.local_basis(n)
        dl = np.linalg.norm(defl, axis=1)
        npr = np.cos(dl)[:, None] * n + (np.sinc(dl / np.pi)[:, None]) * (defl[:, :1] * e_th + defl[:, 1:] * e_ph)
        psi = RNG.uniform(0, np.pi, 400)
        et2, ep2 = kr.local_basis(npr)
        u = np.cos(psi)[:, None] * et2 + np.sin(psi)[:, None] * ep2
        ang = np.arccos(np.clip(np.sum(n * npr, axis=1), -1, 1))
        ut = _rodrigues(u, np.cross(npr, n), ang)
        chi = np.arctan2(np.sum(ut * e_ph, axis=1), np.sum(ut * e_th, axis=1))
        got = np.exp(2j * psi) * kr.pair_phase(n, npr)
        np.testing.assert_allclose(got, np.exp(2j * chi), rtol=0, atol=1e-10)


def test_transport_along_a_meridian_keeps_the_frame():
    # a deflection along e_theta moves along the meridian: e_theta is transported
    # onto e_theta, so the rotation is the identity
    nside = 16
    pix = np.arange(hp.npix(nside))
    defl = np.zeros((pix.size, 2))
    defl[:, 0] = RNG.normal(size=pix.size) * 1e-2
    tv = kr.displace(nside, pix, defl)
    np.testing.assert_allclose(kr.pair_phase(hp.pix2vec(nside, pix), tv), 1.0, rtol=0, atol=1e-12)


# ----------------------------------------- augmented (widely linear) spin 2
def _sY(s, ell, m, v):
    th = np.arctan2(np.hypot(v[:, 0], v[:, 1]), v[:, 2])
    ph = np.arctan2(v[:, 1], v[:, 0])
    # Appendix A: sY_lm = (-1)^s sqrt((2l+1)/4pi) e^{i m phi} d^l_{m,-s}(theta)
    return (-1) ** s * math.sqrt((2 * ell + 1) / (4 * math.pi)) * np.exp(1j * m * ph) * wigner_d(ell, m, -s, th)


@pytest.mark.parametrize("ell", [2, 3, 5, 8])
def test_spin2_pseudo_phase_by_addition_theorem(ell):
    # <P_a P_b> = sum_l (C^EE - C^BB) sum_m 2Y_lm(a) (-2Y_lm(b))^* (P = -sum (E + iB) 2Y with
    # real E, B fields); for one l this must equal (2l+1)/4pi d^l_{2,-2}(beta) pseudo_phase(a, b)
    a = RNG.normal(size=(40, 3))
    a /= np.linalg.norm(a, axis=1)[:, None]
    b = a + RNG.normal(size=(40, 3)) * 0.3
    b /= np.linalg.norm(b, axis=1)[:, None]
    corr = sum(_sY(2, ell, m, a) * np.conj(_sY(-2, ell, m, b)) for m in range(-ell, ell + 1))
    beta = 2 * np.arcsin(np.linalg.norm(a - b, axis=1) / 2)
    model = (2 * ell + 1) / (4 * math.pi) * wigner_d(ell, 2, -2, beta) * kr.pseudo_phase(a, b)
    np.testing.assert_allclose(corr, model, rtol=0, atol=1e-13)


def _aug_inputs(n_pts, K, spread, seed):
    rng = np.random.default_rng(seed)
    t = rng.normal(size=(n_pts, 3))
    t /= np.linalg.norm(t, axis=1)[:, None]
    X = t[:, None, :] + rng.normal(size=(n_pts, K, 3)) * spread
    X /= np.linalg.norm(X, axis=2)[:, :, None]
    y = rng.normal(size=(n_pts, K)) + 1j * rng.normal(size=(n_pts, K))
    return t, X, y


def test_augmented_real_form_matches_complex_augmented_solve():
    # library special case: the widely linear estimator written in the complex augmented
    # form z = (P, P^*), R = [[G, C], [C^*, G^*]], w = R^-1 E[z P_0^*], solved by numpy,
    # against the oracle's 2K x 2K real form (nugget n on the diagonal of G in both)
    lmax, K = 40, 6
    cl = wl.cl_ee(lmax, 30.0)
    bb = 0.3 * cl
    nodes_t = 0.2
    fp, fm, x0 = xi.spin2_tables(cl, bb, nodes_t, 2048)
    t, X, y = _aug_inputs(30, K, 0.05, 5)
    T = np.sum((X[:, :, None, :] - X[:, None, :, :]) ** 2, axis=-1)
    t0 = np.sum((t[:, None, :] - X) ** 2, axis=-1)
    S = fp(T.reshape(-1)).reshape(T.shape)
    val, var, nug = kr._estimate_augmented(X, t, y, S, fp(t0), fm, T, t0, x0, kr.EPS_NUGGET)
    for p in range(t.shape[0]):
        G = np.empty((K, K), complex)
        C = np.empty((K, K), complex)
        for i in range(K):
            for j in range(K):
                if i == j:
                    G[i, j], C[i, j] = 1.0 + nug[p], 0.0
                else:
                    G[i, j] = fp(np.array([T[p, i, j]]))[0] * kr.pair_phase(X[p, i], X[p, j])
                    C[i, j] = fm(np.array([T[p, i, j]]))[0] * kr.pseudo_phase(X[p, i], X[p, j])
        g0 = fp(t0[p]) * kr.pair_phase(X[p], np.broadcast_to(t[p], X[p].shape))
        c0 = fm(t0[p]) * kr.pseudo_phase(X[p], np.broadcast_to(t[p], X[p].shape))
        R = np.block([[G, C], [np.conj(C), np.conj(G)]])
        pv = np.concatenate([g0, np.conj(c0)])
        w = np.linalg.solve(R, pv)
        z = np.concatenate([y[p], np.conj(y[p])])
        assert abs(np.vdot(w, z) - val[p]) < 1e-9 * max(1.0, abs(val[p]))
        assert abs(x0 * (1.0 - np.vdot(pv, w).real) - var[p]) < 1e-9 * x0


def test_augmented_equals_hermitian_without_xi_minus():
    # C^BB = C^EE makes xi- vanish: the augmented estimator reduces to the paper's
    # Hermitian one (same nugget rule, the real form of G + nI has G's spectrum)
    nside, lmax, K = 32, 64, 16
    cl = wl.cl_ee(lmax, 50.0)
    P = sht.synth_map(nside, lmax, wl.draw_alm(cl, 31), spin=2, blm=wl.draw_alm(cl, 32))
    qu = np.stack([P.real, P.imag], axis=1)
    pix = wl.sample_pixels(hp.npix(nside), 500, 33)
    defl = wl.random_deflection(pix.size, 34) * 4
    tmax = 4 * (2.0 * math.sqrt(K / 3.0) / nside) ** 2 * 1.5
    tp, tm, x0 = xi.spin2_tables(cl, cl, tmax, 1024)
    assert np.max(np.abs(tm.f)) < 1e-15
    herm = kr.lens(nside, K, 2, qu, defl, pix, tp, x0)
    aug = kr.lens(nside, K, 2, qu, defl, pix, tp, x0, f_minus=tm)
    scale = np.sqrt(np.mean(np.abs(herm.value) ** 2))
    assert np.max(np.abs(aug.value - herm.value)) < 1e-12 * scale
    assert np.max(np.abs(aug.variance - herm.variance)) < 1e-12 * x0


def test_augmented_error_statistics_with_pure_e_modes():
    # B = 0 (xi- = xi+ at l >> 1 scales): the augmented estimator is the exact Gaussian
    # conditional, its errors match its predicted variance and beat the Hermitian one
    nside, lmax, K = 64, 128, 16
    cl = wl.cl_ee(lmax, 100.0)
    alm = wl.draw_alm(cl, 21)
    P = sht.synth_map(nside, lmax, alm, spin=2)
    qu = np.stack([P.real, P.imag], axis=1)
    pix = wl.sample_pixels(hp.npix(nside), 4000, 22)
    defl = wl.random_deflection(pix.size, 23)
    tmax = 4 * (2.0 * math.sqrt(K / 3.0) / nside) ** 2 * 1.5
    tp, tm, x0 = xi.spin2_tables(cl, None, tmax, 1024)
    herm = kr.lens(nside, K, 2, qu, defl, pix, tp, x0)
    aug = kr.lens(nside, K, 2, qu, defl, pix, tp, x0, f_minus=tm)
    truth = sht.synth_points(lmax, alm, aug.target, spin=2)
    r = np.abs(aug.value - truth) ** 2 / aug.variance
    assert 0.85 < np.mean(r) < 1.15
    e_aug = np.mean(np.abs(aug.value - truth) ** 2)
    e_herm = np.mean(np.abs(herm.value - truth) ** 2)
    assert e_aug < 0.9 * e_herm
    assert np.all(aug.variance <= herm.variance * (1 + 1e-9))


# ------------------------------------------------------------------ spin 1
@pytest.mark.parametrize("ell", [1, 2, 5, 8])
def test_spin1_phases_by_addition_theorem(ell):
    # <P_a P_b^*> and <P_a P_b> of a spin-1 field from the 1Y harmonics of Appendix A;
    # the odd spin makes the direction-of-travel pi visible
    a = RNG.normal(size=(40, 3))
    a /= np.linalg.norm(a, axis=1)[:, None]
    b = a + RNG.normal(size=(40, 3)) * 0.3
    b /= np.linalg.norm(b, axis=1)[:, None]
    beta = 2 * np.arcsin(np.linalg.norm(a - b, axis=1) / 2)
    w = (2 * ell + 1) / (4 * math.pi)
    herm = sum(_sY(1, ell, m, a) * np.conj(_sY(1, ell, m, b)) for m in range(-ell, ell + 1))
    np.testing.assert_allclose(herm, w * wigner_d(ell, 1, 1, beta) * kr.pair_phase(a, b, 1), rtol=0, atol=1e-13)
    pseudo = sum(_sY(1, ell, m, a) * np.conj(_sY(-1, ell, m, b)) for m in range(-ell, ell + 1))
    np.testing.assert_allclose(pseudo, w * wigner_d(ell, 1, -1, beta) * kr.pseudo_phase(a, b, 1), rtol=0, atol=1e-13)


@pytest.mark.parametrize("spin", [1, 2])
def test_pseudo_covariance_of_real_fields(spin):
    # with real E, B fields (a_{l,-m} = (-1)^m a_lm^*) and P = -sum (E + iB)_lm sY_lm,
    # <P_a P_b> = sum_l (C^E - C^B) sum_m (-1)^m sY_lm(a) sY_l,-m(b); the augmented
    # estimator models it as (-1)^s xi-(beta) pseudo_phase(a, b)
    a = RNG.normal(size=(30, 3))
    a /= np.linalg.norm(a, axis=1)[:, None]
    b = a + RNG.normal(size=(30, 3)) * 0.3
    b /= np.linalg.norm(b, axis=1)[:, None]
    beta = 2 * np.arcsin(np.linalg.norm(a - b, axis=1) / 2)
    for ell in (2, 3, 6):
        corr = sum((-1) ** m * _sY(spin, ell, m, a) * _sY(spin, ell, -m, b) for m in range(-ell, ell + 1))
        model = (-1) ** spin * (2 * ell + 1) / (4 * math.pi) * wigner_d(ell, spin, -spin, beta) \
            * kr.pseudo_phase(a, b, spin)
        np.testing.assert_allclose(corr, model, rtol=0, atol=1e-13)


def test_spin1_deflection_field_exact_benchmark():
    # the deflection d = grad phi is a spin-1 field P = d_theta + i d_phi with
    # C^E = l(l+1) C^phiphi, C^B = 0: kriged from its pixel values at displaced
    # directions it must match the harmonic gradient there, errors ~ predicted sigma
    nside, lmax, K = 64, 128, 16
    phi = wl.draw_alm(wl.cl_phiphi(lmax), 24)
    ell = np.arange(lmax + 1)
    cle = wl.cl_phiphi(lmax) * ell * (ell + 1)
    dmap = sht.synth_map(nside, lmax, phi, gradient=True)
    pix = wl.sample_pixels(hp.npix(nside), 3000, 25)
    defl = wl.random_deflection(pix.size, 26) * 2
    tmax = 4 * (2.0 * math.sqrt(K / 3.0) / nside) ** 2 * 1.5
    tp, tm, x0 = xi.spin1_tables(cle, None, tmax, 1024)
    res = kr.lens(nside, K, 1, dmap, defl, pix, tp, x0)
    gth, gph = sht.synth_gradient_points(lmax, phi, res.target)
    truth = gth + 1j * gph
    r = np.abs(res.value - truth) ** 2 / res.variance
    assert 0.85 < np.mean(r) < 1.15
    rel = math.sqrt(np.mean(np.abs(res.value - truth) ** 2) / np.mean(np.abs(truth) ** 2))
    assert rel < 0.05
    aug = kr.lens(nside, K, 1, dmap, defl, pix, tp, x0, f_minus=tm)
    assert np.mean(np.abs(aug.value - truth) ** 2) < np.mean(np.abs(res.value - truth) ** 2)


# ------------------------------------------- symmetries of the HEALPix grid
def _quarter_turn(nside):
    """RING index of every pixel's image under the rotation by pi/2 about the z axis
    (ring i holds 4 nq pixels, so pixel j goes to pixel j + nq of the same ring)."""
    ring, j = hp.pix2ring(nside, np.arange(hp.npix(nside)))
    first, n_in, _, _, _, nq = hp.ring_info(nside, ring)
    return first + (j + nq) % n_in


def _mirror(nside):
    """RING index of every pixel's image under z -> -z (ring i -> ring 4 Nside - i, same
    position in the ring)."""
    ring, j = hp.pix2ring(nside, np.arange(hp.npix(nside)))
    return hp.ring_info(nside, 4 * nside - ring)[0] + j


@pytest.mark.parametrize("spin", [0, 2])
def test_lens_commutes_with_the_grid_symmetries(spin):
    """The whole estimator (displacement, K-nearest stencil, phases, factor) is covariant
    under the symmetries of the grid.  A quarter turn about z carries every local frame
    (e_theta, e_phi) along, so maps, deflections and outputs move with their pixels
    unchanged.  The mirror z -> -z turns e_theta into -e_theta (keeping e_phi): the
    deflection's theta component changes sign, and a spin-2 P = Q + iU measured from
    e_theta towards e_phi becomes conj(P) (angle chi -> pi - chi).  Catches mistakes
    that break these symmetries: a phase or frame sign lost in one hemisphere, a
    displacement or index slip confined to one cap or one quarter of the rings."""
    nside, lmax, K = 16, 40, 16
    npix = hp.npix(nside)
    cl = wl.cl_tt(lmax, 30.0) if spin == 0 else wl.cl_ee(lmax, 30.0)
    m = sht.synth_map(nside, lmax, wl.draw_alm(cl, 41), spin=spin)
    defl = np.random.default_rng(42).normal(scale=0.03, size=(npix, 2))  # about half a pixel
    t_max, n = xi.grid_rule(np.abs(cl), K, nside)
    tab, x0 = xi.spin0_table(cl, t_max, n) if spin == 0 else xi.spin2_tables(cl, None, t_max, n)[::2]
    qu = m if spin == 0 else np.stack([m.real, m.imag], axis=1)
    pix = np.arange(npix)
    base = kr.lens(nside, K, spin, qu, defl, pix, tab, x0)
    sigma = np.sqrt(np.mean(np.abs(m) ** 2))

    rot = _quarter_turn(nside)
    v = hp.pix2vec(nside, pix)
    np.testing.assert_allclose(hp.pix2vec(nside, rot), np.stack([-v[:, 1], v[:, 0], v[:, 2]], 1), rtol=0, atol=1e-15)
    qu_r, defl_r = np.empty_like(qu), np.empty_like(defl)
    qu_r[rot], defl_r[rot] = qu, defl
    r = kr.lens(nside, K, spin, qu_r, defl_r, pix, tab, x0)
    assert np.max(np.abs(r.value[rot] - base.value)) <= 1e-10 * sigma
    assert np.max(np.abs(r.variance[rot] - base.variance)) <= 1e-10 * x0

    mir = _mirror(nside)
    np.testing.assert_array_equal(hp.pix2vec(nside, mir), v * np.array([1.0, 1.0, -1.0]))
    qu_m, defl_m = np.empty_like(qu), np.empty_like(defl)
    qu_m[mir] = qu if spin == 0 else qu * np.array([1.0, -1.0])
    defl_m[mir] = defl * np.array([-1.0, 1.0])
    r = kr.lens(nside, K, spin, qu_m, defl_m, pix, tab, x0)
    want = base.value if spin == 0 else np.conj(base.value)
    assert np.max(np.abs(r.value[mir] - want)) <= 1e-10 * sigma
    assert np.max(np.abs(r.variance[mir] - base.variance)) <= 1e-10 * x0
