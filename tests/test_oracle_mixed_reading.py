"""Why the mixed path runs its factor in double-float rather than as a single-
precision Cholesky factor corrected by FP64 iterative refinement.

On the Nside 4096 spin-2 workload (K = 32 nearest pixels, lmax 4096, the
nugget 1.49e-8 of Sec. 2.4) the normalised covariance S + nI of a stencil has
eigenvalues down to the nugget (those of S reach 1e-12), so its condition
number is about 2e9 and kappa * u_32 is about 100: rounded to FP32 the
matrix is not positive definite, and a factor that exists only after a
diagonal shift is too poor a preconditioner for refinement to reach the 1e-6
tolerance of the mixed path in a bounded number of steps.  These are properties of the covariance the paper builds
(Eqs. fundamental_variance, spins_correl), checked here with the oracle on
seeded stencils of that workload.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
from oracle import kriging as kr
from oracle import xi

W = wl.C3
P = 8  # stencils sampled


@pytest.fixture(scope="module")
def systems():
    cl, bb = W.cl()
    t_max, n = xi.grid_rule(cl + bb, W.K, W.nside)
    f_plus, _, x0 = xi.spin2_tables(cl, bb, t_max, n)
    pix = wl.sample_pixels(W.npix, P, 11)
    d = np.random.default_rng(3).normal(size=(P, 2)) * wl.DEFLECTION_RMS / np.sqrt(2)
    tv = kr.displace(W.nside, pix, d)
    idx, _ = kr.knn(W.nside, tv, W.K)
    X = hp.pix2vec(W.nside, idx)
    S = f_plus(kr._chord2(X[:, :, None, :], X[:, None, :, :]))
    S = S * kr.pair_phase(X[:, :, None, :], X[:, None, :, :], 2)
    S[:, np.arange(W.K), np.arange(W.K)] = 1.0
    A = S + kr.EPS_NUGGET * np.eye(W.K)
    c = f_plus(kr._chord2(tv[:, None, :], X)) * kr.pair_phase(np.broadcast_to(tv[:, None, :], X.shape), X, 2)
    b = np.conj(c)
    # a realisation of the field on the stencil: y = L g with L L^H = A
    g = np.random.default_rng(4).normal(size=(P, W.K, 2)) @ np.array([1.0, 1j]) / np.sqrt(2)
    y = np.einsum("pij,pj->pi", np.linalg.cholesky(A), g)
    return S, A, b, y


def test_covariance_is_too_ill_conditioned_for_an_fp32_factor(systems):
    S, A, _, _ = systems
    lam = np.linalg.eigvalsh(A)
    cond = lam[:, -1] / lam[:, 0]
    assert np.all(cond > 1e8) and np.all(cond * 2.0 ** -24 > 1.0)
    _, ok = kr.cholesky_batched(A.astype(np.complex64))
    assert not ok.any()  # S + nI rounded to FP32 is not positive definite on any stencil


def test_fp64_refinement_of_a_shifted_fp32_factor_stalls_above_the_tolerance(systems):
    S, A, b, y = systems
    w_exact = np.linalg.solve(A, b[..., None])[..., 0]
    v_exact = np.einsum("pi,pi->p", np.conj(w_exact), y)
    L32, ok = kr.cholesky_batched((S + 1e-6 * np.eye(W.K)).astype(np.complex64))
    assert ok.all()  # the smallest shift tried that makes every FP32 factor exist
    errs = []
    for p in range(P):
        L = L32[p].astype(np.complex128)
        w = np.zeros(W.K, complex)
        for _ in range(30):  # residual in FP64, correction through the FP32 factor
            r = (b[p] - A[p] @ w).astype(np.complex64).astype(np.complex128)
            w = w + np.linalg.solve(L.conj().T, np.linalg.solve(L, r))
        errs.append(abs(np.vdot(w, y[p]) - v_exact[p]))
    # values are in units of the field's standard deviation: every stencil is still
    # above the mixed path's 1e-6 tolerance after 30 refinement steps, each an FP64
    # K^2 matvec (measured: 7e-6 to 4e-5)
    assert min(errs) > 1e-6, errs
