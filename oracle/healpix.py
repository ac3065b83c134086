"""HEALPix RING-ordering geometry for the CPU oracle (test infrastructure).

The oracle is test infrastructure: only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg use it.  It shares no code with the CUDA
path.

The paper interpolates maps on the HEALPix grid (Sec. 2.3, "Identifying
neighbors"); its RING ordering is the standard one of the HEALPix
pixelisation: Npix = 12 Nside^2 equal-area pixels on 4 Nside - 1
iso-latitude rings.

* North polar cap, ring i = 1 .. Nside-1: 4i pixels, z = 1 - i^2/(3 Nside^2),
  phi_j = (j + 1/2) pi / (2i), first pixel 2i(i-1).
* Equatorial belt, ring i = Nside .. 3 Nside: 4 Nside pixels,
  z = (4 Nside - 2i)/(3 Nside), phi_j = (j + f) pi/(2 Nside) with
  f = 1/2 when i + Nside is even and f = 0 otherwise,
  first pixel 2 Nside (Nside - 1) + 4 Nside (i - Nside).
* South polar cap mirrors the north cap: ring i = 4 Nside - i', 4i' pixels.

Positions are formed so that z and sin(theta) come from integer ratios and a
single square root: polar cap s = i sqrt(6 Nside^2 - i^2) / (3 Nside^2),
belt s = sqrt((2i - Nside)(7 Nside - 2i)) / (3 Nside).
"""
from __future__ import annotations

import numpy as np


def npix(nside: int) -> int:
    return 12 * nside * nside


def nring(nside: int) -> int:
    return 4 * nside - 1


def ring_info(nside: int, ring: np.ndarray):
    """Per ring (1-based index): (first pixel, pixels in ring, z, s, phase offset f, nq).

    Pixel j (0-based) of the ring sits at phi = (j + f) * pi / (2 nq), nq being
    the number of pixels per quarter ring.
    """
    ring = np.asarray(ring, dtype=np.int64)
    N = int(nside)
    north = ring < N
    south = ring > 3 * N
    belt = ~(north | south)
    ip = np.where(south, 4 * N - ring, ring)  # mirrored index for the caps
    nq = np.where(belt, N, ip)
    n_in = 4 * nq
    first = np.where(
        north,
        2 * ip * (ip - 1),
        np.where(belt, 2 * N * (N - 1) + 4 * N * (ring - N), 12 * N * N - 2 * ip * (ip + 1)),
    )
    three_n2 = 3.0 * N * N
    ipf = ip.astype(np.float64)
    rf = ring.astype(np.float64)
    with np.errstate(invalid="ignore"):  # each branch is only kept where it applies
        z_cap = (three_n2 - ipf * ipf) / three_n2
        s_cap = ipf * np.sqrt(6.0 * N * N - ipf * ipf) / three_n2
        z_belt = (4.0 * N - 2.0 * rf) / (3.0 * N)
        s_belt = np.sqrt((2.0 * rf - N) * (7.0 * N - 2.0 * rf)) / (3.0 * N)
    z = np.where(belt, z_belt, np.where(north, z_cap, -z_cap))
    s = np.where(belt, s_belt, s_cap)
    f = np.where(belt & ((ring + N) % 2 == 1), 0.0, 0.5)
    return first, n_in, z, s, f, nq


def pix2ring(nside: int, pix: np.ndarray):
    """RING pixel index -> (ring, index within ring), both int64 (ring is 1-based)."""
    pix = np.asarray(pix, dtype=np.int64)
    N = int(nside)
    ncap = 2 * N * (N - 1)
    np_ = 12 * N * N
    ring = np.empty_like(pix)
    north = pix < ncap
    south = pix >= np_ - ncap
    belt = ~(north | south)
    # north cap: largest i with 2i(i-1) <= p
    p = pix[north]
    i = ((1 + np.sqrt(1 + 2 * p.astype(np.float64))) // 2).astype(np.int64)
    i = np.where(2 * i * (i - 1) > p, i - 1, i)
    i = np.where(2 * (i + 1) * i <= p, i + 1, i)
    ring[north] = i
    # belt
    ring[belt] = (pix[belt] - ncap) // (4 * N) + N
    # south cap: mirrored pixel q = Npix-1-p lies in mirrored north ring
    q = np_ - 1 - pix[south]
    i = ((1 + np.sqrt(1 + 2 * q.astype(np.float64))) // 2).astype(np.int64)
    i = np.where(2 * i * (i - 1) > q, i - 1, i)
    i = np.where(2 * (i + 1) * i <= q, i + 1, i)
    ring[south] = 4 * N - i
    first = ring_info(N, ring)[0]
    return ring, pix - first


def pix2ang(nside: int, pix: np.ndarray):
    """RING pixel -> (z, s, phi) with z = cos(theta), s = sin(theta)."""
    ring, j = pix2ring(nside, pix)
    _, _, z, s, f, nq = ring_info(nside, ring)
    phi = (j + f) * np.pi / (2.0 * nq)
    return z, s, phi


def pix2vec(nside: int, pix: np.ndarray) -> np.ndarray:
    """RING pixel -> unit vector, shape (..., 3)."""
    z, s, phi = pix2ang(nside, pix)
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=-1)


def ring_above(nside: int, z: np.ndarray) -> np.ndarray:
    """Index of the last ring whose z is >= the given z (0 if none), int64.

    Inverse of the ring latitude rule: polar cap i = Nside sqrt(3(1-z)),
    belt i = Nside (2 - 3z/2); a final comparison against the exact ring z
    removes rounding at ring boundaries.
    """
    z = np.asarray(z, dtype=np.float64)
    N = int(nside)
    za = np.abs(z)
    i_belt = np.floor(N * (2.0 - 1.5 * z))
    i_n = np.floor(N * np.sqrt(np.maximum(3.0 * (1.0 - za), 0.0)))
    i_cap = np.where(z > 0, i_n, 4 * N - 1 - i_n)
    i = np.where(za <= 2.0 / 3.0, i_belt, i_cap).astype(np.int64)
    i = np.clip(i, 0, 4 * N - 1)
    for _ in range(2):
        zi = ring_info(N, np.clip(i, 1, 4 * N - 1))[2]
        i = np.where((i >= 1) & (zi < z), i - 1, i)
        zn = ring_info(N, np.clip(i + 1, 1, 4 * N - 1))[2]
        i = np.where((i + 1 <= 4 * N - 1) & (zn >= z), i + 1, i)
    return i
