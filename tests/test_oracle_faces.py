"""Pins of the oracle's face geometry and the paper's pixel-centred stencil with
tabulated S^-1 (Secs. 2.3-2.5) against the independent RING geometry, round
trips, the topology of the HEALPix grid, the solve route of the estimator and
the exact harmonic sum."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import faces as fc
from oracle import healpix as hp
from oracle import kriging as kr
from oracle import sht
from oracle import xi

RNG = np.random.default_rng(2010)


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16])
def test_face_coordinates_round_trip_and_centres(N):
    pix = np.arange(hp.npix(N))
    ix, iy, f = fc.ring2xyf(N, pix)
    assert np.array_equal(fc.xyf2ring(N, ix, iy, f), pix)
    # the projection of the face-coordinate centres is the RING geometry's centre
    v = fc.face2vec((ix + 0.5) / N, (iy + 0.5) / N, f)
    assert np.max(np.abs(v - hp.pix2vec(N, pix))) < 2e-15


@pytest.mark.parametrize("N", [2, 8, 64])
def test_point_location_inverts_the_projection(N):
    # random interior points of random pixels map back to their pixel
    n = 4000
    f = RNG.integers(0, 12, n)
    ix, iy = RNG.integers(0, N, n), RNG.integers(0, N, n)
    X = (ix + RNG.uniform(0.02, 0.98, n)) / N
    Y = (iy + RNG.uniform(0.02, 0.98, n)) / N
    v = fc.face2vec(X, Y, f)
    assert np.array_equal(fc.vec2pix(N, v), fc.xyf2ring(N, ix, iy, f))
    pix = np.arange(hp.npix(min(N, 16)))
    assert np.array_equal(fc.vec2pix(min(N, 16), hp.pix2vec(min(N, 16), pix)), pix)


@pytest.mark.parametrize("N", [2, 4, 8])
def test_vertex_neighbours_topology(N):
    # every pixel has 8 vertex neighbours except the 24 next to the 8 vertices
    # where three base faces meet (7); the relation is symmetric
    npx = hp.npix(N)
    nb = fc.neighbours(N, np.arange(npx))
    cnt = np.sum(nb >= 0, axis=1)
    assert np.sum(cnt == 7) == 24 and np.sum(cnt == 8) == npx - 24
    for p in range(npx):
        for q in nb[p][nb[p] >= 0]:
            assert p in nb[q]
    # neighbours are close: within 2.5 pixel sizes
    d = np.linalg.norm(hp.pix2vec(N, np.where(nb >= 0, nb, 0)) - hp.pix2vec(N, np.arange(npx))[:, None], axis=-1)
    assert np.max(np.where(nb >= 0, d, 0.0)) < 2.5 * math.sqrt(4 * math.pi / npx)


@pytest.mark.parametrize("y", [1, 2])
def test_stencil_structure(y):
    N = 32
    tv = hp.pix2vec(N, RNG.integers(0, hp.npix(N), 500))
    tv = kr.displace(N, RNG.integers(0, hp.npix(N), 500), wl.random_deflection(500, 3) * 10)
    st = fc.stencil(N, tv, y)
    k = 4 ** (y - 1)
    assert st.shape == (500, 9 * k)
    for s in st:
        m = s[s >= 0]
        assert m.size in (8 * k, 9 * k) and np.unique(m).size == m.size
    # the first block holds the pixels of the direction's pixel at Nside / 2^(y-1)
    c = fc.vec2pix(N >> (y - 1), tv)
    assert np.array_equal(np.sort(st[:, :k], axis=1), np.sort(fc.children(N >> (y - 1), c, y - 1), axis=1))
    if y == 1:
        assert np.array_equal(st[:, 0], fc.vec2pix(N, tv))


@pytest.mark.parametrize("y,tol", [(1, 1e-10), (2, 1e-7)])
def test_inverse_route_matches_solve_and_exact_benchmark(y, tol):
    # the tabulated-inverse estimate equals the Cholesky-solve estimate on the same
    # stencil (to the inverse's conditioning), and its errors match its predicted
    # variance against the harmonic sum
    nside, lmax = 64, 128
    cl = wl.cl_tt(lmax, 100.0)
    alm = wl.draw_alm(cl, 5)
    m = sht.synth_map(nside, lmax, alm)
    pix = wl.sample_pixels(hp.npix(nside), 2000, 6)
    defl = wl.random_deflection(pix.size, 7)
    tmax = 4 * (3.0 * math.sqrt(9 * 4 ** (y - 1) / 3.0) / nside) ** 2 * 2
    tab, x0 = xi.spin0_table(cl, tmax, 2048)
    v, s2, idx, tv = fc.paper_lens(nside, y, m, defl, pix, tab, x0)
    full = np.sum(idx >= 0, axis=1) == idx.shape[1]
    ve, se, _ = kr.estimate(nside, 0, m, tv[full], idx[full], tab, x0)
    assert np.max(np.abs(ve - v[full])) <= tol * np.std(m)
    assert np.max(np.abs(se - s2[full])) <= tol * x0
    truth = sht.synth_points(lmax, alm, tv)
    r = (v - truth) ** 2 / s2
    if y == 1:
        assert 0.85 < np.mean(r) < 1.15
    else:  # the 1.49e-8 nugget bounds the predicted variance from below
        assert 0.5 < np.mean(r) < 1.15


def _chord_signature(nside, members):
    """Sorted pairwise chords of a stencil: invariant under rotations and reflections."""
    X = hp.pix2vec(nside, members)
    d = np.linalg.norm(X[:, None] - X[None], axis=-1)
    return np.sort(d[np.triu_indices(members.size, 1)])


@pytest.mark.parametrize("n_c,y", [(1, 1), (2, 1), (4, 1), (8, 1), (16, 1), (4, 2), (8, 2)])
def test_class_representatives_are_congruent(n_c, y):
    # the symmetry classes of S^-1 tabulation (Sec. 2.4): every coarse pixel's stencil
    # maps member by member onto its representative's, the representatives lie in
    # the northern hemisphere's first quarter (or first pixel of a belt ring), and
    # stencils of one class have the same pairwise chords (a congruence invariant
    # computed without the class map)
    nside = n_c << (y - 1)
    cen = np.arange(hp.npix(n_c))
    rep, mirror, dphi = fc.class_representative(n_c, cen)
    ring, j = hp.pix2ring(n_c, rep)
    assert np.all(ring <= 2 * n_c) and np.all(j < np.maximum(hp.ring_info(n_c, ring)[5], 1))
    assert np.array_equal(rep[rep], rep)  # a representative represents itself
    idx = fc.stencil(nside, hp.pix2vec(n_c, cen), y)
    ridx = fc.stencil(nside, hp.pix2vec(n_c, rep), y)
    for c in cen:
        m, r = idx[c][idx[c] >= 0], ridx[c][ridx[c] >= 0]
        assert m.size == r.size
        U = fc.to_class_frame(hp.pix2vec(nside, m), mirror[c], dphi[c])
        d = np.linalg.norm(U[:, None] - hp.pix2vec(nside, r)[None], axis=-1)
        assert np.max(np.min(d, axis=1)) < 1e-12 and np.unique(np.argmin(d, axis=1)).size == m.size
        assert np.max(np.abs(_chord_signature(nside, m) - _chord_signature(nside, r))) < 1e-12
    # class count: rings 1 .. min(Nc + 2, 2 Nc) by quarter-ring positions, one per deeper belt ring
    n_cls = sum(min(i, n_c) for i in range(1, min(n_c + 2, 2 * n_c) + 1)) + max(0, n_c - 2)
    assert np.unique(rep).size == n_cls


@pytest.mark.parametrize("nside,lmax,y,tol_inv", [(8, 16, 1, 1e-11), (16, 32, 2, 1e-7), (2, 12, 2, 1e-11)])
def test_class_route_matches_per_target_routes(nside, lmax, y, tol_inv):
    # L^-1 tabulated from the class representative's geometry gives the Cholesky
    # solve on each target's own stencil to rounding (1e-10), and the literal
    # S^-1 = L^-T L^-1 route to that route's own error (an explicit inverse loses
    # a factor cond(S) ~ 1e8 at y = 2)
    cl = wl.cl_tt(lmax, 0.7 * lmax)
    t_max, n = fc.paper_grid_rule(cl, nside, y)
    tab, x0 = xi.spin0_table(cl, t_max, n)
    m = sht.synth_map(nside, lmax, wl.draw_alm(cl, 3))
    pix = np.arange(hp.npix(nside))
    defl = wl.random_deflection(pix.size, 4, rms=0.5 * math.sqrt(4 * math.pi / hp.npix(nside)))
    v, s2, idx, tv = fc.paper_lens(nside, y, m, defl, pix, tab, x0)
    vc, s2c, idxc, _ = fc.paper_lens(nside, y, m, defl, pix, tab, x0, classes=True)
    assert np.array_equal(idx, idxc)
    assert np.max(np.abs(vc - v)) <= tol_inv * np.std(m)
    assert np.max(np.abs(s2c - s2)) <= tol_inv * x0
    cnt = np.sum(idx >= 0, axis=1)
    for k in np.unique(cnt):
        rows = np.nonzero(cnt == k)[0]
        st = np.stack([r[r >= 0] for r in idx[rows]])
        ve, se, _ = kr.estimate(nside, 0, m, tv[rows], st, tab, x0)
        assert np.max(np.abs(vc[rows] - ve)) <= 1e-10 * np.std(m)
        assert np.max(np.abs(s2c[rows] - se)) <= 1e-10 * x0


@pytest.mark.parametrize("n_c,y", [(1, 1), (4, 1), (8, 1), (4, 2)])
def test_member_order_is_kept_by_the_symmetries(n_c, y):
    # in the ordering rule, every stencil of a class lists its members so that the
    # chord matrices coincide (what lets one tabulated factor serve the class)
    nside = n_c << (y - 1)
    cen = np.arange(hp.npix(n_c))
    rep = fc.class_representative(n_c, cen)[0]
    ordered = fc.stencil_ordered(nside, y, cen)
    for c in cen:
        m, r = ordered[c], ordered[rep[c]]
        assert np.array_equal(np.sort(m), np.sort(fc.stencil(nside, hp.pix2vec(n_c, np.array([c])), y)[0][
            fc.stencil(nside, hp.pix2vec(n_c, np.array([c])), y)[0] >= 0]))
        X, Y = hp.pix2vec(nside, m), hp.pix2vec(nside, r)
        T = np.sum((X[:, None] - X[None]) ** 2, axis=-1)
        Tr = np.sum((Y[:, None] - Y[None]) ** 2, axis=-1)
        assert np.max(np.abs(T - Tr)) <= 1e-13 * np.max(Tr)


@pytest.mark.parametrize("spin", [1, 2])
@pytest.mark.parametrize("n_c,y", [(2, 1), (4, 1), (8, 1), (4, 2)])
def test_spin2_class_covariance_rotates_and_conjugates(n_c, y, spin):
    # the spin-2 member-member covariance of every stencil, taken to its class
    # representative's member order, equals the representative's (rotation about the
    # polar axis: frames turn with the sphere) or its complex conjugate (reflection
    # z -> -z: every angle a becomes pi - a) -- what lets one L^-1, or its
    # conjugate, serve a class
    nside = n_c << (y - 1)
    lmax = 3 * nside
    cl = wl.cl_ee(lmax, 0.7 * lmax)
    t_max, n = fc.paper_grid_rule(cl, nside, y, 0.3 * cl)
    tables = xi.spin2_tables if spin == 2 else xi.spin1_tables
    tab, _, _ = tables(cl, 0.3 * cl, t_max, n)
    cen = np.arange(hp.npix(n_c))
    rep, mirror, dphi = fc.class_representative(n_c, cen)
    ordered = fc.stencil_ordered(nside, y, cen)
    reps = {}
    for c in cen:
        m = ordered[c]
        C = fc.class_covariance(nside, m, tab, spin)
        r = int(rep[c])
        if r not in reps:
            reps[r] = fc.class_covariance(nside, ordered[r], tab, spin)
        ref = np.conj(reps[r]) if mirror[c] else reps[r]
        assert np.max(np.abs(C - ref)) < 1e-12, f"coarse pixel {c}"
    assert np.any(mirror) and not np.all(mirror)


@pytest.mark.parametrize("spin", [1, 2])
@pytest.mark.parametrize("nside,lmax,y", [(8, 16, 1), (16, 32, 2)])
def test_spin2_class_route_matches_per_target_solve(nside, lmax, y, spin):
    cl = wl.cl_ee(lmax, 0.7 * lmax)
    bb = 0.3 * cl
    t_max, n = fc.paper_grid_rule(cl, nside, y, bb)
    tab, _, x0 = (xi.spin2_tables if spin == 2 else xi.spin1_tables)(cl, bb, t_max, n)
    P = sht.synth_map(nside, lmax, wl.draw_alm(cl, 3), spin=spin, blm=wl.draw_alm(bb, 4))
    m = np.ascontiguousarray(np.stack([P.real, P.imag], axis=1))
    pix = np.arange(hp.npix(nside))
    defl = wl.random_deflection(pix.size, 5, rms=0.5 * math.sqrt(4 * math.pi / hp.npix(nside)))
    v, s2, idx, tv = fc.paper_lens(nside, y, m, defl, pix, tab, x0, classes=True, spin=spin)
    sigma = math.sqrt(np.mean(np.abs(P) ** 2))
    cnt = np.sum(idx >= 0, axis=1)
    for k in np.unique(cnt):
        rows = np.nonzero(cnt == k)[0]
        st = np.stack([r[r >= 0] for r in idx[rows]])
        ve, se, _ = kr.estimate(nside, spin, m, tv[rows], st, tab, x0)
        # the class route factors the representative's covariance, whose member
        # positions differ from the target's own by rounding; at y = 2 the
        # spin-1 covariance's conditioning turns that into up to 3e-10
        tol = 1e-10 if y == 1 else 1e-9
        assert np.max(np.abs(v[rows] - ve)) <= tol * sigma
        assert np.max(np.abs(s2[rows] - se)) <= tol * x0


@pytest.mark.parametrize("n_c,y", [(4, 1), (8, 1), (4, 2)])
def test_augmented_class_covariance_and_route(n_c, y):
    # the augmented (xi+, xi-) member covariance of every stencil equals its class
    # representative's A (rotation) or D A D, D = diag(I, -I) (reflection: G, C
    # conjugate, U changes sign); the class route then matches the per-target
    # augmented solve
    nside = n_c << (y - 1)
    lmax = 3 * nside
    cl = wl.cl_ee(lmax, 0.7 * lmax)
    bb = 0.3 * cl
    t_max, n = fc.paper_grid_rule(cl, nside, y, bb)
    tp, tm, x0 = xi.spin2_tables(cl, bb, t_max, n)
    cen = np.arange(hp.npix(n_c))
    rep, mirror, _ = fc.class_representative(n_c, cen)
    ordered = fc.stencil_ordered(nside, y, cen)
    reps = {}
    for c in cen:
        A = fc.class_covariance_aug(nside, ordered[c], tp, tm, 2)
        r = int(rep[c])
        if r not in reps:
            reps[r] = fc.class_covariance_aug(nside, ordered[r], tp, tm, 2)
        k = ordered[c].size
        dsig = np.concatenate([np.ones(k), -np.ones(k)])
        ref = reps[r] * np.outer(dsig, dsig) if mirror[c] else reps[r]
        assert np.max(np.abs(A - ref)) < 1e-12, f"coarse pixel {c}"
    P = sht.synth_map(nside, lmax, wl.draw_alm(cl, 3), spin=2, blm=wl.draw_alm(bb, 4))
    m = np.ascontiguousarray(np.stack([P.real, P.imag], axis=1))
    pix = np.arange(hp.npix(nside))
    defl = wl.random_deflection(pix.size, 5, rms=0.5 * math.sqrt(4 * math.pi / hp.npix(nside)))
    v, s2, idx, tv = fc.paper_lens(nside, y, m, defl, pix, tp, x0, classes=True, spin=2, f_minus=tm)
    sigma = math.sqrt(np.mean(np.abs(P) ** 2))
    cnt = np.sum(idx >= 0, axis=1)
    for k in np.unique(cnt):
        rows = np.nonzero(cnt == k)[0]
        st = np.stack([r[r >= 0] for r in idx[rows]])
        ve, se, _ = kr.estimate(nside, 2, m, tv[rows], st, tp, x0, f_minus=tm)
        assert np.max(np.abs(v[rows] - ve)) <= 1e-10 * sigma
        assert np.max(np.abs(s2[rows] - se)) <= 1e-10 * x0
