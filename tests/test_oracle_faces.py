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
