"""Pins of the oracle's HEALPix RING geometry and exact K-nearest search."""

import numpy as np
import pytest

from oracle import healpix as hp
from oracle import kriging as kr


def test_nside1_base_pixels():
    # Nside = 1: three rings of four pixels at z = 2/3, 0, -2/3; the middle ring
    # starts at phi = 0, the others are offset by half a pixel (pi/4).
    z, s, phi = hp.pix2ang(1, np.arange(12))
    np.testing.assert_allclose(z, [2 / 3] * 4 + [0] * 4 + [-2 / 3] * 4, rtol=0, atol=1e-16)
    q = np.pi / 2
    np.testing.assert_allclose(phi, [q / 2 + k * q for k in range(4)] + [k * q for k in range(4)]
                               + [q / 2 + k * q for k in range(4)], rtol=0, atol=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 4, 16, 64])
def test_ring_layout(nside):
    npix = hp.npix(nside)
    pix = np.arange(npix)
    ring, j = hp.pix2ring(nside, pix)
    first, n_in, z, s, f, nq = hp.ring_info(nside, ring)
    assert np.all(first + j == pix) and np.all((j >= 0) & (j < n_in))
    counts = np.bincount(ring, minlength=4 * nside)[1:]
    r = np.arange(1, 4 * nside)
    expect = np.where(r < nside, 4 * r, np.where(r > 3 * nside, 4 * (4 * nside - r), 4 * nside))
    assert np.all(counts == expect)
    v = hp.pix2vec(nside, pix)
    assert np.abs(np.sum(v * v, axis=1) - 1).max() <= 1e-15
    # north-south mirror symmetry: pixel p and Npix-1-p have opposite z
    z2 = hp.pix2ang(nside, pix)[0]
    np.testing.assert_allclose(z2, -z2[::-1], rtol=0, atol=1e-16)
    # z strictly decreasing from ring to ring; mean z is zero (equal areas)
    zr = hp.ring_info(nside, r)[2]
    assert np.all(np.diff(zr) < 0)
    assert abs(np.mean(z2)) < 1e-15


@pytest.mark.parametrize("nside", [2, 8, 64])
def test_ring_above(nside):
    rng = np.random.default_rng(3)
    zz = np.concatenate([rng.uniform(-1, 1, 500), hp.ring_info(nside, np.arange(1, 4 * nside))[2]])
    i = hp.ring_above(nside, zz)
    zr = np.concatenate([[np.inf], hp.ring_info(nside, np.arange(1, 4 * nside))[2], [-np.inf]])
    assert np.all(zr[i] >= zz) and np.all(zr[i + 1] < zz)


def _brute_knn(nside, tv, K):
    allpix = np.arange(hp.npix(nside))
    vv = hp.pix2vec(nside, allpix)
    out = []
    for v in tv:
        key = np.sum((vv - v) ** 2, axis=1)
        out.append(allpix[np.lexsort((allpix, key))[:K]])
    return np.array(out)


@pytest.mark.parametrize("nside,K", [(1, 4), (4, 16), (8, 24), (16, 48), (64, 32)])
def test_knn_matches_brute_force(nside, K):
    rng = np.random.default_rng(nside * 100 + K)
    tv = rng.normal(size=(60, 3))
    tv /= np.linalg.norm(tv, axis=1)[:, None]
    # add points right next to the poles and on pixel centres
    tv = np.concatenate([tv, [[0, 0, 1.0]], [[1e-9, 0, -1.0]], hp.pix2vec(nside, np.arange(0, hp.npix(nside), 7))[:20]])
    tv /= np.linalg.norm(tv, axis=1)[:, None]
    idx, key = kr.knn(nside, tv, min(K, hp.npix(nside)))
    ref = _brute_knn(nside, tv, min(K, hp.npix(nside)))
    assert np.array_equal(idx, ref)
    assert np.all(np.diff(key, axis=1) >= 0)


def test_knn_large_nside_against_local_brute_force():
    nside, K = 4096, 32
    rng = np.random.default_rng(9)
    tv = rng.normal(size=(20, 3))
    tv /= np.linalg.norm(tv, axis=1)[:, None]
    idx, key = kr.knn(nside, tv, K)
    # brute force over every pixel of the 41 rings around the target latitude
    for v, row in zip(tv, idx):
        ic = int(hp.ring_above(nside, np.array([v[2]]))[0])
        rings = np.arange(max(1, ic - 20), min(4 * nside - 1, ic + 20) + 1)
        first, n_in = hp.ring_info(nside, rings)[:2]
        pix = np.concatenate([f + np.arange(n) for f, n in zip(first, n_in)])
        kk = np.sum((hp.pix2vec(nside, pix) - v) ** 2, axis=1)
        ref = pix[np.lexsort((pix, kk))[:K]]
        assert np.array_equal(row, ref)
