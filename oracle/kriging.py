"""Plain FP64 kriging interpolator on the HEALPix sphere: the CPU oracle.

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path.

For every target pixel p (RING index) the oracle performs the steps of the
method in the paper's order:

1. Displaced direction (Sec. 3.1, lensed-direction equation): with |d| the
   length of the deflection (d_theta, d_phi) in the local basis (e_theta,
   e_phi) at the pixel centre n,
       n' = cos|d| n + sin|d| (d_theta e_theta + d_phi e_phi) / |d|.
2. Stencil: the K pixel centres nearest to n' in chord distance
   t = |n' - n_q|^2, ties broken by the lower RING index.  The search scans a
   ring window and proves the result exact by comparing the K-th distance with
   a lower bound for every pixel outside the window; points where the proof
   fails are searched again in a larger window.
3. Covariances (Eqs. fundamental_variance, v_spins): S_ij = xi(t_ij)/xi(0)
   between stencil pixels, c_i = xi(t(n', n_i))/xi(0) to the target.  Spin s
   (1: a deflection, 2: Q/U) uses the Hermitian <P_i P_j^*> =
   xi+(t_ij) exp(is(a_ij - a_ji - pi)) with a_ij the angle at n_i, measured from
   e_theta towards e_phi, of the geodesic towards n_j.
4. Cholesky (Sec. 2.4) of S + n I with the nugget n = epsilon = 1.49e-8 when
   that factorisation has only positive pivots, and otherwise the paper's rule
   n = -lambda_min + epsilon (lambda_min the lowest eigenvalue of S).
5. Conditional mean and variance (Eqs. best_temperature_field, gaussvar,
   major_eq, gaussvar_pol): with L L^H = S + n I, z_c = L^{-1} conj(c),
   z_y = L^{-1} y,
       value = z_c^H z_y,   variance = xi(0) (1 - |z_c|^2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import healpix as hp

EPS_NUGGET = 1.49e-8  # square root of the double-precision machine epsilon (Sec. 2.4)


# ------------------------------------------------------------- geometry
def local_basis(v: np.ndarray):
    """(e_theta, e_phi) at unit vectors v (..., 3); undefined exactly at the poles."""
    x, y, z = v[..., 0], v[..., 1], v[..., 2]
    s = np.sqrt(x * x + y * y)
    cphi = np.where(s > 0, x / np.where(s > 0, s, 1.0), 1.0)
    sphi = np.where(s > 0, y / np.where(s > 0, s, 1.0), 0.0)
    e_th = np.stack([z * cphi, z * sphi, -s], axis=-1)
    e_ph = np.stack([-sphi, cphi, np.zeros_like(s)], axis=-1)
    return e_th, e_ph


def displace(nside: int, pix: np.ndarray, defl: np.ndarray) -> np.ndarray:
    """Displaced unit vectors n' for target pixels ``pix`` with deflections ``defl`` (n, 2)."""
    z, s, phi = hp.pix2ang(nside, pix)
    cphi, sphi = np.cos(phi), np.sin(phi)
    n = np.stack([s * cphi, s * sphi, z], axis=-1)
    e_th = np.stack([z * cphi, z * sphi, -s], axis=-1)
    e_ph = np.stack([-sphi, cphi, np.zeros_like(s)], axis=-1)
    dth = defl[:, 0]
    dph = defl[:, 1]
    dl = np.sqrt(dth * dth + dph * dph)
    sinc = np.sinc(dl / np.pi)  # sin|d| / |d|, equal to 1 at |d| = 0
    return (np.cos(dl)[:, None] * n
            + (sinc * dth)[:, None] * e_th
            + (sinc * dph)[:, None] * e_ph)


def _chord2(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    d = a - b
    return np.sum(d * d, axis=-1)


def knn(nside: int, targets: np.ndarray, K: int, R: int | None = None, W: int | None = None):
    """Exact K nearest RING pixels to each unit vector in ``targets`` (P, 3).

    Returns (indices (P, K) int64, squared chords (P, K)) sorted by (chord^2, index).
    """
    targets = np.asarray(targets, dtype=np.float64)
    P = targets.shape[0]
    N = int(nside)
    rho = math.sqrt(K / 3.0)  # radius of a cap holding K pixels, in units of 1/Nside
    if R is None:
        R = int(math.ceil(2.0 * rho / 0.6)) + 1
    if W is None:
        W = int(math.ceil(2.0 * rho / 1.1)) + 1
    idx_out = np.empty((P, K), dtype=np.int64)
    key_out = np.empty((P, K))
    todo = np.arange(P)
    while todo.size:
        ok, idx, key = _knn_window(N, targets[todo], K, R, W)
        idx_out[todo[ok]] = idx[ok]
        key_out[todo[ok]] = key[ok]
        todo = todo[~ok]
        R, W = 2 * R, 2 * W
        if R > 4 * N and W > 4 * N:
            # the window covers the whole sphere: brute force
            allpix = np.arange(hp.npix(N))
            vv = hp.pix2vec(N, allpix)
            for p in todo:
                kk = _chord2(targets[p][None, :], vv)
                order = np.lexsort((allpix, kk))[:K]
                idx_out[p] = allpix[order]
                key_out[p] = kk[order]
            break
    return idx_out, key_out


def _knn_window(N: int, tv: np.ndarray, K: int, R: int, W: int):
    P = tv.shape[0]
    z = np.clip(tv[:, 2], -1.0, 1.0)
    ic = hp.ring_above(N, z)  # ring just north of (or at) the target latitude
    ic = np.clip(ic, 1, 4 * N - 1)
    offs = np.arange(-R, R + 2)  # rings ic-R .. ic+R+1
    rings = ic[:, None] + offs[None, :]
    rvalid = (rings >= 1) & (rings <= 4 * N - 1)
    rr = np.clip(rings, 1, 4 * N - 1)
    first, n_in, zr, sr, f, nq = hp.ring_info(N, rr)
    phi_t = np.arctan2(tv[:, 1], tv[:, 0]) % (2.0 * np.pi)
    jc = np.floor(phi_t[:, None] * (2.0 * nq) / np.pi - f + 0.5).astype(np.int64) % n_in
    m = np.arange(-W, W + 1)
    nw = 2 * W + 1
    small = n_in <= nw  # whole ring fits in the window
    j = np.where(small[..., None], np.arange(nw)[None, None, :],
                 (jc[..., None] + m[None, None, :]) % n_in[..., None])
    cvalid = rvalid[..., None] & np.where(small[..., None], np.arange(nw)[None, None, :] < n_in[..., None], True)
    pix = first[..., None] + j
    pix = np.where(cvalid, pix, 0)
    vv = hp.pix2vec(N, pix.reshape(-1)).reshape(P, -1, 3)
    key = _chord2(tv[:, None, :], vv)
    cv = cvalid.reshape(P, -1)
    key = np.where(cv, key, np.inf)
    pflat = pix.reshape(P, -1)
    order = np.lexsort((pflat, key), axis=-1)[:, :K]
    kidx = np.take_along_axis(pflat, order, axis=1)
    kkey = np.take_along_axis(key, order, axis=1)
    # lower bound for every pixel outside the window
    st = np.sqrt(np.maximum(tv[:, 0] ** 2 + tv[:, 1] ** 2, 0.0))
    lb = np.full(P, np.inf)
    for side in (0, -1):
        r_out = rings[:, 0] - 1 if side == 0 else rings[:, -1] + 1
        inside = (r_out >= 1) & (r_out <= 4 * N - 1)
        _, _, zo, so, _, _ = hp.ring_info(N, np.clip(r_out, 1, 4 * N - 1))
        b = (z - zo) ** 2 + (st - so) ** 2
        lb = np.where(inside, np.minimum(lb, b), lb)
    # excluded pixels of each window ring: the nearest ones are W+1 steps from jc
    for dm in (-(W + 1), W + 1):
        jo = (jc + dm) % n_in
        po = first + jo
        vo = hp.pix2vec(N, np.where(rvalid & ~small, po, 0).reshape(-1)).reshape(P, -1, 3)
        ko = _chord2(tv[:, None, :], vo)
        ko = np.where(rvalid & ~small, ko, np.inf)
        lb = np.minimum(lb, ko.min(axis=1))
    ok = np.isfinite(kkey[:, -1]) & (kkey[:, -1] < lb)
    return ok, kidx, kkey


# ------------------------------------------------------------ linear algebra
def cholesky_batched(A: np.ndarray):
    """Cholesky L L^H = A for a batch (P, K, K) of Hermitian matrices.

    Returns (L, ok) where ok[p] is False if a pivot was not positive.
    """
    P, K, _ = A.shape
    L = np.zeros_like(A)
    ok = np.ones(P, dtype=bool)
    for j in range(K):
        d = A[:, j, j].real - np.sum(np.abs(L[:, j, :j]) ** 2, axis=1)
        ok &= d > 0
        ljj = np.sqrt(np.where(d > 0, d, 1.0))
        L[:, j, j] = ljj
        if j + 1 < K:
            s = A[:, j + 1:, j] - np.einsum("pik,pk->pi", L[:, j + 1:, :j], np.conj(L[:, j, :j]))
            L[:, j + 1:, j] = s / ljj[:, None]
    return L, ok


def forward_solve(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve L z = b for lower-triangular L (P, K, K) and right-hand sides b (P, K)."""
    P, K, _ = L.shape
    z = np.zeros(b.shape, dtype=np.result_type(L, b))
    for j in range(K):
        z[:, j] = (b[:, j] - np.einsum("pk,pk->p", L[:, j, :j], z[:, :j])) / L[:, j, j]
    return z


def factor_with_nugget(S: np.ndarray, eps: float = EPS_NUGGET):
    """Cholesky of S + n I with the nugget rule of Sec. 2.4; returns (L, n per point)."""
    P, K, _ = S.shape
    eye = np.eye(K)
    nug = np.full(P, eps)
    L, ok = cholesky_batched(S + eps * eye)
    bad = np.nonzero(~ok)[0]
    if bad.size:
        lam = np.linalg.eigvalsh(S[bad])[:, 0]
        nb = np.where(lam < 0, -lam, 0.0) + eps
        for _ in range(60):
            Lb, okb = cholesky_batched(S[bad] + nb[:, None, None] * eye)
            if okb.all():
                break
            nb = np.where(okb, nb, nb + eps)  # rounding can leave the shifted matrix indefinite
        L[bad] = Lb
        nug[bad] = nb
    return L, nug


# -------------------------------------------------------------- estimator
@dataclass
class Result:
    value: np.ndarray      # (P,) float (spin 0) or complex Q + iU (spin 2)
    variance: np.ndarray   # (P,)
    stencil: np.ndarray    # (P, K) RING indices
    keys: np.ndarray       # (P, K) squared chords to n'
    nugget: np.ndarray     # (P,)
    target: np.ndarray     # (P, 3) displaced unit vectors


def phase_s(va: np.ndarray, vb: np.ndarray, spin: int) -> np.ndarray:
    """exp(i s a_ab) where a_ab is the angle at va, from e_theta towards e_phi, of the
    tangent direction towards vb (the projection of vb - va on the tangent plane)."""
    e_th, e_ph = local_basis(va)
    d = vb - va
    A = np.sum(d * e_th, axis=-1)
    B = np.sum(d * e_ph, axis=-1)
    w = A + 1j * B
    with np.errstate(invalid="ignore", divide="ignore"):  # a point paired with itself has no direction
        return (w / np.abs(w)) ** spin


def phase2(va: np.ndarray, vb: np.ndarray) -> np.ndarray:
    """exp(2i a_ab) (spin 2)."""
    return phase_s(va, vb, 2)


def pair_phase(va: np.ndarray, vb: np.ndarray, spin: int = 2) -> np.ndarray:
    """Phase of <P(va) P(vb)^*> relative to xi+: exp(i s (a_ab - a_ba - pi)), both
    frames referred to the geodesic's direction of travel from va to vb (at vb
    that direction is a_ba + pi; the pi matters for odd s only).

    Coincident points (zero separation) correlate with no rotation: V_ii = 1
    in Eq. v_spins."""
    ph = (-1.0) ** spin * phase_s(va, vb, spin) * np.conj(phase_s(vb, va, spin))
    return np.where(np.isfinite(ph), ph, 1.0 + 0.0j)


def pseudo_phase(va: np.ndarray, vb: np.ndarray, spin: int = 2) -> np.ndarray:
    """Phase of the pseudo-covariance <P(va) P(vb)> relative to xi-:
    exp(i s (a_ab + a_ba + pi)) (the same direction-of-travel convention).

    Coincident points have xi-(0) = 0; their phase is set to 0."""
    ph = (-1.0) ** spin * phase_s(va, vb, spin) * phase_s(vb, va, spin)
    return np.where(np.isfinite(ph), ph, 0.0 + 0.0j)


def real_form(G: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Twice the covariance of the real vector (Q_1..Q_K, U_1..U_K) against
    (Q_1..Q_M, U_1..U_M), from the Hermitian covariance G = <P P^H> and the
    pseudo-covariance C = <P P^T> of P = Q + iU (blocks (..., K, M) -> (..., 2K, 2M)):
        2<Q Q> = Re(G + C),  2<Q U> = Im(C - G),  2<U Q> = Im(G + C),  2<U U> = Re(G - C)."""
    top = np.concatenate([(G + C).real, (C - G).imag], axis=-1)
    bot = np.concatenate([(G + C).imag, (G - C).real], axis=-1)
    return np.concatenate([top, bot], axis=-2)


def _estimate_augmented(X, targets, y, S, c, f_minus, T, t0, xi_zero, eps, spin=2):
    """Widely linear (augmented) spin-2 estimate: the Gaussian conditional mean of
    (Q, U) at the target given (Q_i, U_i), using both xi+ (through <P P^*>) and xi-
    (through <P P>), as a 2K x 2K real system."""
    K = X.shape[1]
    # <P_a P_b> of real E and B fields carries (-1)^s relative to the harmonic sum
    # sum_m sY(a) (-sY(b))^* = (2l+1)/(4 pi) d^l_{s,-s} pseudo_phase(a, b)
    sgn = (-1.0) ** spin
    G = S * pair_phase(X[:, :, None, :], X[:, None, :, :], spin)
    G[:, np.arange(K), np.arange(K)] = 1.0
    C = sgn * f_minus(T.reshape(-1)).reshape(T.shape) * pseudo_phase(X[:, :, None, :], X[:, None, :, :], spin)
    C[:, np.arange(K), np.arange(K)] = 0.0
    tb = np.broadcast_to(targets[:, None, :], X.shape)
    g0 = c * pair_phase(X, tb, spin)            # <P_i P_0^*> / xi+(0)
    c0 = sgn * f_minus(t0) * pseudo_phase(X, tb, spin)  # <P_i P_0> / xi+(0)
    A = real_form(G, C)
    B = real_form(g0[:, :, None], c0[:, :, None])  # (batch, 2K, 2): columns for Q_0 and U_0
    L, nug = factor_with_nugget(A, eps)
    ZQ = forward_solve(L, B[:, :, 0])
    ZU = forward_solve(L, B[:, :, 1])
    zx = forward_solve(L, np.concatenate([y.real, y.imag], axis=1))
    val = np.sum(ZQ * zx, axis=1) + 1j * np.sum(ZU * zx, axis=1)
    var = xi_zero * (1.0 - 0.5 * (np.sum(ZQ * ZQ, axis=1) + np.sum(ZU * ZU, axis=1)))
    return val, var, nug


def estimate(nside: int, spin: int, maps: np.ndarray, targets: np.ndarray, idx: np.ndarray,
             f_plus, xi_zero: float, eps: float = EPS_NUGGET, f_minus=None):
    """Steps 3-5 on a given stencil ``idx`` (B, K): (values, variances, nuggets).

    ``f_minus`` (spin 1, 2): xi-/xi+(0); when given, the augmented estimator is used."""
    K = idx.shape[1]
    X = hp.pix2vec(nside, idx)  # (B, K, 3)
    T = _chord2(X[:, :, None, :], X[:, None, :, :])
    S = f_plus(T.reshape(-1)).reshape(T.shape)
    t0 = _chord2(targets[:, None, :], X)
    c = f_plus(t0)
    if spin != 0 and f_minus is not None:
        y = maps[idx, 0] + 1j * maps[idx, 1]
        return _estimate_augmented(X, targets, y, S, c, f_minus, T, t0, xi_zero, eps, spin)
    if spin == 0:
        y = maps[idx]
        L, nug = factor_with_nugget(S, eps)
        zc = forward_solve(L, c)
        zy = forward_solve(L, y)
        return np.sum(zc * zy, axis=1), xi_zero * (1.0 - np.sum(zc * zc, axis=1)), nug
    Ph = pair_phase(X[:, :, None, :], X[:, None, :, :], spin)
    C = S * Ph
    C[:, np.arange(K), np.arange(K)] = 1.0
    c0 = c * pair_phase(np.broadcast_to(targets[:, None, :], X.shape), X, spin)
    y = maps[idx, 0] + 1j * maps[idx, 1]
    L, nug = factor_with_nugget(C, eps)
    zc = forward_solve(L, np.conj(c0))
    zy = forward_solve(L, y)
    return np.sum(np.conj(zc) * zy, axis=1), xi_zero * (1.0 - np.sum(np.abs(zc) ** 2, axis=1)), nug


def interpolate(nside: int, K: int, spin: int, maps: np.ndarray, targets: np.ndarray,
                f_plus, xi_zero: float, eps: float = EPS_NUGGET, batch: int = 4096, f_minus=None) -> Result:
    """Kriging at unit vectors ``targets`` (P, 3) from a RING map.

    ``maps``: (Npix,) real for spin 0; (Npix, 2) real and imaginary parts for spin 1
    ((d_theta, d_phi) of a deflection) and spin 2 (Q, U).
    ``f_plus``: callable t -> xi(t)/xi(0) (spin 0) or xi+(t)/xi+(0) (spin 2),
    either an ``xi.HermiteTable`` (tabulated mode) or a direct evaluation.
    ``f_minus`` (spin 2, optional): xi-(t)/xi+(0); selects the augmented estimator.
    """
    P = targets.shape[0]
    vals = np.empty(P, dtype=np.float64 if spin == 0 else np.complex128)
    var = np.empty(P)
    sten = np.empty((P, K), dtype=np.int64)
    keys = np.empty((P, K))
    nugs = np.empty(P)
    for b0 in range(0, P, batch):
        tv = targets[b0:b0 + batch]
        idx, key = knn(nside, tv, K)
        v, s2, nug = estimate(nside, spin, maps, tv, idx, f_plus, xi_zero, eps, f_minus)
        vals[b0:b0 + batch] = v
        var[b0:b0 + batch] = s2
        sten[b0:b0 + batch] = idx
        keys[b0:b0 + batch] = key
        nugs[b0:b0 + batch] = nug
    return Result(vals, var, sten, keys, nugs, targets)


def lens(nside: int, K: int, spin: int, maps: np.ndarray, defl: np.ndarray, pix: np.ndarray,
         f_plus, xi_zero: float, eps: float = EPS_NUGGET, rotate: bool = False, f_minus=None) -> Result:
    """Lensed values at target pixels ``pix`` (Born remap T(n + d(n)), Sec. 3.1).

    ``rotate`` (spin 2): return P in the frame at the target pixel n rather than at
    the displaced direction n', i.e. P(n') parallel-transported back along the
    geodesic from n' to n, which multiplies it by pair_phase(n, n')."""
    pix = np.asarray(pix, dtype=np.int64)
    tv = displace(nside, pix, np.asarray(defl, dtype=np.float64))
    res = interpolate(nside, K, spin, maps, tv, f_plus, xi_zero, eps, f_minus=f_minus)
    if rotate and spin != 0:
        res.value = res.value * pair_phase(hp.pix2vec(nside, pix), tv, spin)
    return res


def supersample(nside: int, nside_out: int, K: int, spin: int, maps: np.ndarray, pix_out: np.ndarray,
                f_plus, xi_zero: float, eps: float = EPS_NUGGET) -> Result:
    """Values at the centres of pixels ``pix_out`` of a finer Nside_out grid (Sec. 2.6):
    the same estimator with undisplaced targets."""
    tv = hp.pix2vec(nside_out, np.asarray(pix_out, dtype=np.int64))
    return interpolate(nside, K, spin, maps, tv, f_plus, xi_zero, eps)
