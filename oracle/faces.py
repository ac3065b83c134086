"""HEALPix base-face geometry for the paper's pixel-centred stencil (Sec. 2.3):
face coordinates of RING pixels, the continuous face projection, point
location, vertex-sharing neighbours and the 9 * 4^(y-1) stencil.

Test infrastructure (oracle): only tests/, the smoke check and the CPU-baseline
leg of the benchmark use it; it shares no code with the CUDA path.

Faces.  The sphere is divided into 12 base faces; face f holds the pixels
(f, ix, iy), 0 <= ix, iy < N.  Face f has ring coordinate jrll[f] and azimuth
coordinate jpll[f] (in units of N rings and pi/4):
    jrll = 2 2 2 2 3 3 3 3 4 4 4 4,   jpll = 1 3 5 7 0 2 4 6 1 3 5 7.
A point with face coordinates (X, Y) in [0, 1]^2 (pixel centres at
((ix + 1/2)/N, (iy + 1/2)/N)) lies on ring coordinate rho = jrll - X - Y and
    rho < 1:      z = 1 - rho^2/3,           phi = (pi/4)(jpll + (X - Y)/rho)
    1 <= rho <= 3: z = (2 - rho) 2/3,        phi = (pi/4)(jpll + X - Y)
    rho > 3:      z = -(1 - (4 - rho)^2/3),  phi = (pi/4)(jpll + (X - Y)/(4 - rho)),
the HEALPix projection, which at pixel centres gives the RING centres
(ring i = N rho, position j from phi).  Pixel vertices are the images of the
integer face coordinates.

Stencil (Sec. 2.3, "neighbors()" extended with the NESTED hierarchy): at level
y the direction's pixel at Nside_c = Nside / 2^(y-1) and the pixels of that
grid sharing a vertex with it (8, or 7 at the 24 pixels next to the vertices
where three faces meet), each replaced by its 4^(y-1) sub-pixels at Nside:
9 * 4^(y-1) (or 8 * 4^(y-1)) RING pixels.  The paper's "pixelization at
Nside/y" is read as Nside / 2^(y-1), the only grid whose pixels hold
4^(y-1) pixels each.
"""
from __future__ import annotations

import math

import numpy as np

from . import healpix as hp
from . import kriging as kr
from . import xi

JRLL = np.array([2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4])
JPLL = np.array([1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7])


def _ring_params(N: int, i):
    """(nr, kshift) of rings i (1-based)."""
    i = np.asarray(i, dtype=np.int64)
    nr = np.where(i < N, i, np.where(i > 3 * N, 4 * N - i, N))
    ks = np.where((i >= N) & (i <= 3 * N), (i - N) & 1, 0)
    return nr, ks


def xyf2ring(N: int, ix, iy, f):
    """RING index of pixel (f, ix, iy)."""
    ix, iy, f = (np.asarray(a, dtype=np.int64) for a in (ix, iy, f))
    jr = JRLL[f] * N - ix - iy - 1
    nr, ks = _ring_params(N, jr)
    jp = (JPLL[f] * nr + ix - iy + 1 + ks) // 2
    jp = np.where(jp > 4 * nr, jp - 4 * nr, jp)
    jp = np.where(jp < 1, jp + 4 * nr, jp)
    first = np.where(jr < N, 2 * jr * (jr - 1),
                     np.where(jr <= 3 * N, 2 * N * (N - 1) + 4 * N * (jr - N), 12 * N * N - 2 * nr * (nr + 1)))
    return first + jp - 1


def ring2xyf(N: int, pix):
    """(ix, iy, f) of RING pixels, by trying the 12 faces: on face f the ring and
    position fix ix + iy and (ix - iy mod 8 nr); the face is the one where both
    coordinates fall in [0, N)."""
    pix = np.asarray(pix, dtype=np.int64)
    i = hp.pix2ring(N, pix)[0]
    first = hp.ring_info(N, i)[0]
    jp = pix - first + 1
    nr, ks = _ring_params(N, i)
    out_ix = np.full(pix.shape, -1, dtype=np.int64)
    out_iy = np.full(pix.shape, -1, dtype=np.int64)
    out_f = np.full(pix.shape, -1, dtype=np.int64)
    for f in range(12):
        s = JRLL[f] * N - 1 - i
        d = 2 * jp - 1 - ks - JPLL[f] * nr
        d = (d + 4 * nr) % (8 * nr) - 4 * nr  # representative in [-4 nr, 4 nr)
        ok = ((s + d) % 2 == 0)
        ix = (s + d) // 2
        iy = (s - d) // 2
        ok &= (ix >= 0) & (ix < N) & (iy >= 0) & (iy < N)
        ok &= out_f < 0
        out_ix = np.where(ok, ix, out_ix)
        out_iy = np.where(ok, iy, out_iy)
        out_f = np.where(ok, f, out_f)
    assert np.all(out_f >= 0), "RING pixel without a face"
    return out_ix, out_iy, out_f


def face2vec(X, Y, f):
    """Unit vectors of face coordinates (X, Y) on faces f (the projection above)."""
    X, Y = np.asarray(X, dtype=np.float64), np.asarray(Y, dtype=np.float64)
    f = np.asarray(f, dtype=np.int64)
    rho = JRLL[f] - X - Y
    north, south = rho < 1.0, rho > 3.0
    rn = np.where(north, rho, np.where(south, 4.0 - rho, 1.0))
    z = np.where(north, 1.0 - rho * rho / 3.0,
                 np.where(south, -(1.0 - (4.0 - rho) ** 2 / 3.0), (2.0 - rho) * 2.0 / 3.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(north | south, np.where(rn > 0, (X - Y) / np.where(rn > 0, rn, 1.0), 0.0), X - Y)
    phi = 0.25 * math.pi * (JPLL[f] + t)
    s = np.sqrt(np.maximum(0.0, (1.0 - z) * (1.0 + z)))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=-1)


def vertices(N: int, pix):
    """(n, 4, 3) vertices of RING pixels: images of the integer face coordinates."""
    ix, iy, f = ring2xyf(N, pix)
    corners = [(0, 0), (1, 0), (0, 1), (1, 1)]
    return np.stack([face2vec((ix + a) / N, (iy + b) / N, f) for a, b in corners], axis=-2)


def vec2pix(N: int, v):
    """RING pixel containing each unit vector: the face and (X, Y) that the
    projection maps onto it (inverse of face2vec), then (ix, iy) = floor(N X, N Y)."""
    v = np.asarray(v, dtype=np.float64)
    z = v[..., 2]
    phi = np.arctan2(v[..., 1], v[..., 0]) % (2.0 * math.pi)
    a = phi / (0.25 * math.pi)  # azimuth in units of pi/4, [0, 8)
    best_f = np.full(z.shape, -1, dtype=np.int64)
    bx = np.zeros(z.shape)
    by = np.zeros(z.shape)
    for f in range(12):
        if JRLL[f] == 2:
            rho = np.where(z > 2.0 / 3.0, np.sqrt(3.0 * (1.0 - z)), 2.0 - 1.5 * z)
            scale = np.where(z > 2.0 / 3.0, rho, 1.0)
        elif JRLL[f] == 4:
            rho = np.where(z < -2.0 / 3.0, 4.0 - np.sqrt(3.0 * (1.0 + z)), 2.0 - 1.5 * z)
            scale = np.where(z < -2.0 / 3.0, 4.0 - rho, 1.0)
        else:
            rho = 2.0 - 1.5 * z
            scale = np.ones_like(z)
        da = (a - JPLL[f] + 4.0) % 8.0 - 4.0  # azimuth offset from the face centre, [-4, 4)
        d = da * scale
        s = JRLL[f] - rho
        X = 0.5 * (s + d)
        Y = 0.5 * (s - d)
        ok = (X >= 0) & (X <= 1) & (Y >= 0) & (Y <= 1) & (best_f < 0)
        best_f = np.where(ok, f, best_f)
        bx = np.where(ok, X, bx)
        by = np.where(ok, Y, by)
    assert np.all(best_f >= 0), "direction outside every face"
    ix = np.minimum((bx * N).astype(np.int64), N - 1)
    iy = np.minimum((by * N).astype(np.int64), N - 1)
    return xyf2ring(N, ix, iy, best_f)


def neighbours(N: int, pix, tol: float = 1e-9):
    """Pixels sharing at least one vertex with each RING pixel, sorted by RING
    index, padded with -1 to 8 columns."""
    pix = np.atleast_1d(np.asarray(pix, dtype=np.int64))
    cand, _ = kr.knn(N, hp.pix2vec(N, pix), min(25, hp.npix(N)))
    vp = vertices(N, pix)                                   # (n, 4, 3)
    vc = vertices(N, cand.ravel()).reshape(cand.shape + (4, 3))  # (n, c, 4, 3)
    dist = np.linalg.norm(vp[:, None, :, None, :] - vc[:, :, None, :, :], axis=-1)
    share = np.any(dist < tol / N, axis=(2, 3)) & (cand != pix[:, None])
    out = np.full((pix.size, 8), -1, dtype=np.int64)
    for r in range(pix.size):
        nb = np.sort(cand[r][share[r]])
        assert nb.size <= 8, "more than 8 vertex neighbours"
        out[r, :nb.size] = nb
    return out


def children(N_c: int, pix_c, level: int):
    """RING indices (at N_c * 2^level) of the 4^level sub-pixels of RING pixels at
    N_c, in face-coordinate order (x fastest)."""
    ix, iy, f = ring2xyf(N_c, pix_c)
    k = 1 << level
    a, b = np.meshgrid(np.arange(k), np.arange(k), indexing="xy")
    a, b = a.ravel(), b.ravel()
    return xyf2ring(N_c * k, ix[..., None] * k + a, iy[..., None] * k + b, f[..., None])


def stencil(N: int, targets, y: int):
    """The paper's stencil of unit vectors ``targets`` at level y: (n, 9 * 4^(y-1))
    RING indices at N, -1 where the direction's pixel has 7 neighbours.  Order:
    the direction's pixel, then its neighbours by RING index, each expanded to
    its sub-pixels in face-coordinate order."""
    N_c = N >> (y - 1)
    assert N_c << (y - 1) == N and N_c >= 1, "Nside must be divisible by 2^(y-1)"
    c = vec2pix(N_c, targets)
    nb = neighbours(N_c, c)
    coarse = np.concatenate([c[:, None], nb], axis=1)  # (n, 9)
    k = 1 << (2 * (y - 1))
    out = np.full((coarse.shape[0], 9 * k), -1, dtype=np.int64)
    valid = coarse >= 0
    ch = children(N_c, np.where(valid, coarse, 0), y - 1)  # (n, 9, k)
    ch = np.where(valid[..., None], ch, -1)
    out[:] = ch.reshape(coarse.shape[0], 9 * k)
    return out


# ------------------------------------------------- correlation table domain
PAPER_CHORD_BOUND = 7.0  # chords within a level-y stencil, and to its targets, in units of 1/Nside_c


def paper_grid_rule(cl: np.ndarray, nside: int, y: int, cl_bb: np.ndarray | None = None):
    """Domain and size of the correlation table for the level-y stencil: every
    chord between members of a stencil, and from a target in the central coarse
    pixel to them, is below 7 / Nside_c (Nside_c = Nside / 2^(y-1); the bound
    found by adding the centre-to-centre chords of the coarse pixels and the
    radii of the pixels grows from 4.7 at Nside_c = 2 to 6.3 at 64 and
    converges below 6.5), so t_max = (7 / Nside_c)^2, at most 4 (the antipodal
    chord^2, reached only for Nside_c <= 3); the interval count
    follows the error rule of xi.grid_rule (spin 2: weights |C^EE| + |C^BB|).
    Returns (t_max, n)."""
    n_c = nside >> (y - 1)
    t_max = min((PAPER_CHORD_BOUND / n_c) ** 2, 4.0)  # 4: the chord^2 of antipodal points
    w = np.abs(cl) if cl_bb is None else np.abs(cl) + np.abs(cl_bb)
    return t_max, xi.table_size(w, t_max)


# ------------------------------------------------- estimator with tabulated S^-1
def inverse_estimate(nside: int, maps: np.ndarray, targets: np.ndarray, idx: np.ndarray, f_plus, xi_zero: float,
                     eps: float = kr.EPS_NUGGET):
    """Spin-0 estimate on stencils ``idx`` (-1 = absent member) the way Sec. 2.4
    forms it: L from the Cholesky of S + n I (nugget rule of Sec. 2.4), L^-1 by
    direct inversion, S^-1 = L^-T L^-1 (the tabulated matrix), then the weights
    w = S^-1 c, value = w . y and variance = xi(0) (1 - c . w).  Returns
    (values, variances, nuggets)."""
    P = targets.shape[0]
    val = np.empty(P)
    var = np.empty(P)
    nug = np.empty(P)
    counts = np.sum(idx >= 0, axis=1)
    for K in np.unique(counts):
        rows = np.nonzero(counts == K)[0]
        st = np.stack([r[r >= 0] for r in idx[rows]])  # members in stencil order
        X = hp.pix2vec(nside, st)
        T = np.sum((X[:, :, None, :] - X[:, None, :, :]) ** 2, axis=-1)
        S = f_plus(T.reshape(-1)).reshape(T.shape)
        L, n = kr.factor_with_nugget(S, eps)
        eye = np.broadcast_to(np.eye(K), L.shape)
        Linv = np.stack([kr.forward_solve(L, eye[:, :, k]) for k in range(K)], axis=2)  # L^-1 e_k as columns
        Sinv = np.einsum("pki,pkj->pij", Linv, Linv)
        c = f_plus(np.sum((targets[rows][:, None, :] - X) ** 2, axis=-1))
        w = np.einsum("pij,pj->pi", Sinv, c)
        val[rows] = np.sum(w * maps[st], axis=1)
        var[rows] = xi_zero * (1.0 - np.sum(c * w, axis=1))
        nug[rows] = n
    return val, var, nug


# ------------------------------------------------- inverse per class of central pixels
def class_representative(n_c: int, pix_c):
    """Representative of each central pixel's symmetry class (Sec. 2.4: S^-1 is
    tabulated once for stencils that the symmetries of the grid map onto each
    other), with the map of the pixel's stencil onto the representative's:
    (rep, mirror, dphi), a member v going to R_z(dphi) M v, M the reflection
    z -> -z when mirror is set.

    The grid is invariant under z -> -z (ring i -> 4 Nc - i, same position j),
    under rotations by pi/2 about the polar axis (j -> j + nq) and, on the rings
    of the equatorial belt, under the rotation by one pixel.  A pixel whose
    stencil lies wholly inside the belt (folded ring Nc + 3 .. 2 Nc: the
    members' rings stay within Nc + 1 .. 3 Nc - 1) is congruent to the first
    pixel of its folded ring; any other to the pixel j mod nq of its folded ring."""
    pix_c = np.asarray(pix_c, dtype=np.int64)
    ring, j = hp.pix2ring(n_c, pix_c)
    mirror = ring > 2 * n_c
    fr = np.where(mirror, 4 * n_c - ring, ring)
    first, _, _, _, _, nq = hp.ring_info(n_c, fr)
    jr = np.where(fr >= n_c + 3, 0, j % nq)
    dphi = (jr - j) * (np.pi / 2.0) / nq
    return first + jr, mirror, dphi


def to_class_frame(v: np.ndarray, mirror, dphi) -> np.ndarray:
    """Apply the class map (reflection, then rotation about the polar axis) to
    vectors v (..., K, 3) of stencils whose maps are given per stencil."""
    mirror = np.asarray(mirror)[..., None]
    c, s = np.cos(dphi)[..., None], np.sin(dphi)[..., None]
    x, y, z = v[..., 0], v[..., 1], np.where(mirror, -v[..., 2], v[..., 2])
    return np.stack([c * x - s * y, s * x + c * y, z], axis=-1)


def stencil_ordered(nside: int, y: int, pix_c) -> list:
    """Members of the level-y stencils of coarse pixels ``pix_c`` in the order
    that makes congruent stencils list corresponding members at the same place:
    sorted by (s r, dphi), r the member's ring, s = +1 for a central pixel in the
    northern half (ring <= 2 Nside_c) and -1 in the southern, dphi the member's
    azimuth minus the central pixel's, wrapped to (-pi, pi], compared exactly
    (fractions of a quarter turn).  Rotations about the polar axis keep r and
    dphi; the reflection z -> -z keeps dphi and maps s r to s r - 4 Nside."""
    from fractions import Fraction

    n_c = nside >> (y - 1)
    pix_c = np.atleast_1d(np.asarray(pix_c, dtype=np.int64))
    idx = stencil(nside, hp.pix2vec(n_c, pix_c), y)
    ring_c, j_c = hp.pix2ring(n_c, pix_c)
    _, _, _, _, f_c, nq_c = hp.ring_info(n_c, ring_c)
    out = []
    for k in range(pix_c.size):
        mem = idx[k][idx[k] >= 0]
        r, j = hp.pix2ring(nside, mem)
        _, _, _, _, f, nq = hp.ring_info(nside, r)
        sgn = 1 if ring_c[k] <= 2 * n_c else -1
        u_c = Fraction(int(2 * j_c[k] + round(2 * f_c[k])), int(2 * nq_c[k]))
        keys = []
        for a in range(mem.size):
            du = Fraction(int(2 * j[a] + round(2 * f[a])), int(2 * nq[a])) - u_c
            while du > 2:
                du -= 4
            while du <= -2:
                du += 4
            keys.append((sgn * int(r[a]), du, int(mem[a])))
        keys.sort()
        out.append(np.array([m for _, _, m in keys], dtype=np.int64))
    return out


def class_covariance(nside: int, members: np.ndarray, f_plus, spin: int = 0) -> np.ndarray:
    """Member-member covariance of one stencil (members in order): spin 0
    xi(t_ij)/xi(0); spin 2 xi+(t_ij)/xi+(0) exp(2i(a_ij - a_ji)) (Eqs. v_spins,
    spins_correl), unit diagonal."""
    X = hp.pix2vec(nside, members)
    K = members.size
    S = f_plus(np.sum((X[:, None, :] - X[None, :, :]) ** 2, axis=-1).reshape(-1)).reshape(K, K)
    if spin == 0:
        return S
    C = S * kr.pair_phase(X[:, None, :], X[None, :, :], spin)
    C[np.arange(K), np.arange(K)] = 1.0
    return C


def class_covariance_aug(nside: int, members: np.ndarray, f_plus, f_minus, spin: int = 2) -> np.ndarray:
    """The augmented (widely linear) member covariance of one stencil: the real
    2K x 2K form (kriging.real_form) of the Hermitian part G (class_covariance)
    and the pseudo-covariance C_ij = (-1)^s xi-(t_ij)/xi+(0) exp(is(a_ij + a_ji
    + pi)) (zero diagonal) of P = Q + iU, in the order (Q_1..Q_K, U_1..U_K)."""
    X = hp.pix2vec(nside, members)
    K = members.size
    G = class_covariance(nside, members, f_plus, spin)
    T = np.sum((X[:, None, :] - X[None, :, :]) ** 2, axis=-1)
    C = (-1.0) ** spin * f_minus(T.reshape(-1)).reshape(K, K) * kr.pseudo_phase(X[:, None, :], X[None, :, :], spin)
    C[np.arange(K), np.arange(K)] = 0.0
    return kr.real_form(G, C)


def class_estimate(nside: int, y: int, maps: np.ndarray, targets: np.ndarray, f_plus, xi_zero: float,
                   eps: float = kr.EPS_NUGGET, spin: int = 0, f_minus=None):
    """Estimate with the inverse tabulated per class (Sec. 2.4): for each class
    the representative's S + n I is factored (nugget rule of Sec. 2.4) and
    L^-1 found by direct inversion from the representative's own member
    positions; a target in coarse pixel c uses that L^-1 with c's members
    matched to the representative's (the member nearest to R_z(dphi) M v), its
    own covariances c_i and data: z_c = L^-1 conj(c), z_y = L^-1 y, value
    conj(z_c) . z_y (= c^H S^-1 y), variance xi(0) (1 - |z_c|^2).  (The same
    estimator as w = S^-1 c with S^-1 = L^-H L^-1 formed explicitly, but
    without that product's loss of a factor cond(S).)

    Spin 2 (maps (Npix, 2) = Q, U): c_i = xi+(t_i)/xi+(0) exp(2i(a_0i - a_i0));
    rotations about the polar axis carry the local frames along and leave the
    member-member phases unchanged, the reflection z -> -z turns every angle a
    into pi - a and conjugates them, so a mirrored class uses conj(L^-1).

    Augmented (``f_minus`` given, spin 1, 2): the class factor is that of the
    real 2K x 2K form A of (G, C) (class_covariance_aug); conjugating G and C
    flips the sign of U, A -> D A D with D = diag(I, -I), so a mirrored class
    uses D L^-1 D; per target the columns B of (<P_i P_0^*>, <P_i P_0>) and the
    data (Q_i, U_i) give Z_Q, Z_U = L^-1 B and z_x = L^-1 x, the value
    (Z_Q . z_x, Z_U . z_x) and the variance xi+(0) (1 - (|Z_Q|^2 + |Z_U|^2)/2).
    Returns (values, variances, stencils)."""
    n_c = nside >> (y - 1)
    cpix = vec2pix(n_c, targets)
    idx = stencil(nside, targets, y)
    rep, mirror, dphi = class_representative(n_c, cpix)
    P = targets.shape[0]
    val = np.empty(P, dtype=np.float64 if spin == 0 else np.complex128)
    var = np.empty(P)
    for r in np.unique(rep):
        rows = np.nonzero(rep == r)[0]
        ridx = stencil(nside, hp.pix2vec(n_c, np.array([r])), y)[0]
        ridx = ridx[ridx >= 0]
        K = ridx.size
        Xr = hp.pix2vec(nside, ridx)
        aug = spin != 0 and f_minus is not None
        A = class_covariance_aug(nside, ridx, f_plus, f_minus, spin) if aug else class_covariance(nside, ridx, f_plus,
                                                                                                  spin)
        L, _ = kr.factor_with_nugget(A[None], eps)
        eye = np.eye(A.shape[0], dtype=L.dtype)[None]
        Linv = np.stack([kr.forward_solve(L, eye[:, :, k]) for k in range(A.shape[0])], axis=2)[0]
        mem = np.stack([row[row >= 0] for row in idx[rows]])  # (n, K): every pixel of a class has K members
        X = hp.pix2vec(nside, mem)
        U = to_class_frame(X, mirror[rows], dphi[rows])
        d = np.linalg.norm(U[:, :, None, :] - Xr[None, None, :, :], axis=-1)
        perm = np.argmin(d, axis=2)  # member a of c <-> member perm[a] of the representative
        assert np.max(np.min(d, axis=2)) < 1e-9 / nside, "stencil not congruent to its class representative"
        assert np.all(np.sort(perm, axis=1) == np.arange(K)), "class map is not a bijection of the members"
        tgt = targets[rows][:, None, :]
        t0 = np.sum((tgt - X) ** 2, axis=-1)
        c = f_plus(t0)
        if aug:
            tb = np.broadcast_to(tgt, X.shape)
            sgn = (-1.0) ** spin
            g0 = c * kr.pair_phase(X, tb, spin)  # <P_i P_0^*> / xi+(0)
            c0 = sgn * f_minus(t0) * kr.pseudo_phase(X, tb, spin)  # <P_i P_0> / xi+(0)
            B = kr.real_form(g0[:, :, None], c0[:, :, None])  # (n, 2K, 2) in c's member order
            xv = np.concatenate([maps[mem, 0], maps[mem, 1]], axis=1)
            ar = np.arange(rows.size)[:, None]
            pos = np.concatenate([perm, K + perm], axis=1)  # c's 2K slots in the representative's order
            B_r = np.empty_like(B)
            x_r = np.empty_like(xv)
            B_r[ar, pos] = B
            x_r[ar, pos] = xv
            dsig = np.concatenate([np.ones(K), -np.ones(K)])
            Lm = Linv * np.outer(dsig, dsig)  # D L^-1 D
            Li = np.where(mirror[rows][:, None, None], Lm[None], Linv[None])
            ZQ = np.einsum("pij,pj->pi", Li, B_r[:, :, 0])
            ZU = np.einsum("pij,pj->pi", Li, B_r[:, :, 1])
            zx = np.einsum("pij,pj->pi", Li, x_r)
            val[rows] = np.sum(ZQ * zx, axis=1) + 1j * np.sum(ZU * zx, axis=1)
            var[rows] = xi_zero * (1.0 - 0.5 * (np.sum(ZQ * ZQ, axis=1) + np.sum(ZU * ZU, axis=1)))
            continue
        if spin == 0:
            yv = maps[mem]
        else:
            c = c * kr.pair_phase(np.broadcast_to(tgt, X.shape), X, spin)
            yv = maps[mem, 0] + 1j * maps[mem, 1]
        ar = np.arange(rows.size)[:, None]
        c_r = np.empty_like(c)
        y_r = np.empty_like(yv)
        c_r[ar, perm] = c  # in the representative's member order
        y_r[ar, perm] = yv
        Li = np.where(mirror[rows][:, None, None], np.conj(Linv)[None], Linv[None]) if spin != 0 else Linv[None]
        zc = np.einsum("pij,pj->pi", Li, np.conj(c_r))
        zy = np.einsum("pij,pj->pi", Li, y_r)
        val[rows] = np.sum(np.conj(zc) * zy, axis=1) if spin != 0 else np.sum(zc * zy, axis=1)
        var[rows] = xi_zero * (1.0 - np.sum(np.abs(zc) ** 2, axis=1))
    return val, var, idx


def paper_lens(nside: int, y: int, maps: np.ndarray, defl: np.ndarray, pix: np.ndarray, f_plus, xi_zero: float,
               classes: bool = False, spin: int = 0, f_minus=None):
    """Lensed values with the paper's stencil at level y (Secs. 2.3-2.5);
    ``classes``: the inverse per class of central pixels (class_estimate)
    instead of S^-1 per target (spin 0 only)."""
    tv = kr.displace(nside, np.asarray(pix, dtype=np.int64), np.asarray(defl, dtype=np.float64))
    if classes:
        v, s2, idx = class_estimate(nside, y, maps, tv, f_plus, xi_zero, spin=spin, f_minus=f_minus)
        return v, s2, idx, tv
    assert spin == 0, "the per-target S^-1 route is spin 0"
    idx = stencil(nside, tv, y)
    v, s2, n = inverse_estimate(nside, maps, tv, idx, f_plus, xi_zero)
    return v, s2, idx, tv


def paper_supersample(nside: int, nside_out: int, y: int, maps: np.ndarray, pix_out: np.ndarray, f_plus,
                      xi_zero: float, classes: bool = False, spin: int = 0):
    """Supersampling (Sec. 2.6) with the paper's stencil at level y."""
    tv = hp.pix2vec(nside_out, np.asarray(pix_out, dtype=np.int64))
    if classes:
        v, s2, idx = class_estimate(nside, y, maps, tv, f_plus, xi_zero, spin=spin)
        return v, s2, idx, tv
    assert spin == 0, "the per-target S^-1 route is spin 0"
    idx = stencil(nside, tv, y)
    v, s2, n = inverse_estimate(nside, maps, tv, idx, f_plus, xi_zero)
    return v, s2, idx, tv
