"""Seeded synthetic inputs for the lensing remap.

This module only draws random numbers and evaluates the analytic input
spectra that define the workloads; it computes no step of the interpolation
method (no correlation function, no geometry, no kriging).  Both the CUDA
path (through its tests and ``bench.py``) and the CPU oracle take their inputs
from here, so neither side generates data for the other.

Workloads (all spectra are zero for l < 2):

* ``c1``: spin 0, Nside 64, lmax 128, C_l = 1e3/(l(l+1)) exp(-(l/100)^2),
  K = 16, FP64.
* ``c2``: spin 0, Nside 2048, lmax 4096, damping scale l = 2500, K = 32,
  FP64 and mixed.
* ``c3``: spin 2 (Q/U), Nside 4096, lmax 4096, C_l^EE = 0.05 x the C2 shape,
  C_l^BB = 0, K = 32, mixed and FP64.
* ``c4``: 64 independent maps, Nside in {256, 512, 1024, 2048},
  K in {16, 24, 32, 48}, spin in {0, 2}, lmax = min(2 Nside, 4096),
  damping at 0.61 lmax.
* ``c5``: Poisson stream of jobs, point count log-uniform in [1e4, 1e8]
  (capped at Npix), spin in {0, 2}, K in {16, 32}, Nside in
  {512, 1024, 2048, 4096}.

The lensing potential has C_l^phiphi proportional to l^-4 for l >= 2, scaled
so that the deflection d = grad(phi) has an rms of 2.5 arcmin:
sum_l (2l+1)/(4 pi) l(l+1) C_l^phiphi = (2.5 arcmin)^2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ARCMIN = math.pi / (180.0 * 60.0)
DEFLECTION_RMS = 2.5 * ARCMIN


def cl_tt(lmax: int, l_damp: float) -> np.ndarray:
    """Temperature spectrum C_l = 1e3/(l(l+1)) exp(-(l/l_damp)^2), l >= 2."""
    ell = np.arange(lmax + 1, dtype=np.float64)
    cl = np.zeros(lmax + 1)
    e = ell[2:]
    cl[2:] = 1e3 / (e * (e + 1.0)) * np.exp(-((e / l_damp) ** 2))
    return cl


def cl_ee(lmax: int, l_damp: float) -> np.ndarray:
    """E-mode spectrum: 0.05 x the temperature shape (B = 0)."""
    return 0.05 * cl_tt(lmax, l_damp)


def cl_phiphi(lmax: int, rms: float = DEFLECTION_RMS) -> np.ndarray:
    """Lensing potential spectrum proportional to l^-4 with a given deflection rms (rad)."""
    ell = np.arange(lmax + 1, dtype=np.float64)
    cl = np.zeros(lmax + 1)
    e = ell[2:]
    cl[2:] = e ** -4.0
    power = np.sum((2.0 * e + 1.0) / (4.0 * math.pi) * e * (e + 1.0) * cl[2:])
    return cl * (rms * rms / power)


def draw_alm(cl: np.ndarray, seed: int) -> np.ndarray:
    """Gaussian harmonic coefficients a_lm for m >= 0, shape (lmax+1, lmax+1) [l, m].

    m = 0: real N(0, C_l); m > 0: complex with independent N(0, C_l/2) real and
    imaginary parts.  Entries with m > l are zero.  Draw order: l-major, then m,
    real part before imaginary part, from numpy's PCG64(seed).
    """
    lmax = len(cl) - 1
    rng = np.random.Generator(np.random.PCG64(seed))
    alm = np.zeros((lmax + 1, lmax + 1), dtype=np.complex128)
    for ell in range(lmax + 1):
        g = rng.standard_normal(2 * ell + 1)
        sd = math.sqrt(cl[ell]) if cl[ell] > 0 else 0.0
        alm[ell, 0] = sd * g[0]
        if ell > 0:
            re = g[1::2]
            im = g[2::2]
            alm[ell, 1 : ell + 1] = (sd / math.sqrt(2.0)) * (re + 1j * im)
    return alm


def white_map(npix: int, ncomp: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """Seeded white-noise map values, shape (npix,) or (npix, ncomp)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (npix,) if ncomp == 1 else (npix, ncomp)
    return sigma * rng.standard_normal(shape)


def random_deflection(npix: int, seed: int, rms: float = DEFLECTION_RMS) -> np.ndarray:
    """Seeded per-pixel deflection (d_theta, d_phi) in radians, total rms ``rms``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rms / math.sqrt(2.0)) * rng.standard_normal((npix, 2))


def sample_pixels(npix: int, n: int, seed: int) -> np.ndarray:
    """Sorted, distinct, seeded pixel indices (int64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = min(n, npix)
    return np.sort(rng.choice(npix, size=n, replace=False)).astype(np.int64)


@dataclass(frozen=True)
class Workload:
    name: str
    spin: int
    nside: int
    lmax: int
    l_damp: float
    K: int
    seed_map: int
    seed_phi: int
    seed_sample: int

    @property
    def npix(self) -> int:
        return 12 * self.nside * self.nside

    def cl(self) -> tuple[np.ndarray, np.ndarray | None]:
        """(C_l, C_l^BB) for the workload: spin 0 -> (TT, None); spin 2 -> (EE, BB = 0)."""
        if self.spin == 0:
            return cl_tt(self.lmax, self.l_damp), None
        return cl_ee(self.lmax, self.l_damp), np.zeros(self.lmax + 1)


C1 = Workload("c1", 0, 64, 128, 100.0, 16, 1, 2, 0)
C2 = Workload("c2", 0, 2048, 4096, 2500.0, 32, 3, 4, 5)
C3 = Workload("c3", 2, 4096, 4096, 2500.0, 32, 6, 7, 8)


def batched_maps(n: int = 64, seed: int = 100) -> list[Workload]:
    """The 64-map batched workload: Nside, K and spin drawn uniformly, seed 100+i."""
    out = []
    for i in range(n):
        rng = np.random.Generator(np.random.PCG64(seed + i))
        nside = int(rng.choice([256, 512, 1024, 2048]))
        K = int(rng.choice([16, 24, 32, 48]))
        spin = int(rng.choice([0, 2]))
        lmax = min(2 * nside, 4096)
        out.append(Workload(f"c4_{i}", spin, nside, lmax, 0.61 * lmax, K, seed + i, 10_000 + seed + i, 0))
    return out


@dataclass(frozen=True)
class Job:
    arrival_s: float
    spin: int
    K: int
    nside: int
    first: int
    count: int


def job_stream(n_jobs: int, rate_hz: float, seed: int = 500, max_points: float = 1e8) -> list[Job]:
    """Serving workload: Poisson arrivals, log-uniform point counts in [1e4, max_points]
    (capped at Npix), spin in {0, 2}, K in {16, 32}, Nside in {512, 1024, 2048, 4096};
    each job is a contiguous RING pixel range of its map."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    jobs = []
    for _ in range(n_jobs):
        t += rng.exponential(1.0 / rate_hz)
        nside = int(rng.choice([512, 1024, 2048, 4096]))
        npix = 12 * nside * nside
        count = int(min(npix, round(10 ** rng.uniform(4.0, math.log10(max_points)))))
        first = int(rng.integers(0, npix - count + 1))
        jobs.append(Job(t, int(rng.choice([0, 2])), int(rng.choice([16, 32])), nside, first, count))
    return jobs


def hashed_normal(idx: np.ndarray, seed: int, ncomp: int = 1) -> np.ndarray:
    """Deterministic N(0,1)-like values per pixel index (SplitMix64 hash, Box-Muller),
    so that any subset of a huge map can be generated without materialising it."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):  # modular 64-bit arithmetic
        return _hashed(idx, seed, ncomp)


def _hashed(idx, seed, ncomp):
    out = []
    for c in range(ncomp):
        z = idx * np.uint64(2 * ncomp) + np.uint64(2 * c) + np.uint64(seed) * np.uint64(0x9E3779B97F4A7C15)
        u = []
        for k in range(2):
            x = z + np.uint64(k)
            x = (x + np.uint64(0x9E3779B97F4A7C15))
            x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            x = x ^ (x >> np.uint64(31))
            u.append(((x >> np.uint64(11)).astype(np.float64) + 0.5) / 9007199254740992.0)
        out.append(np.sqrt(-2.0 * np.log(u[0])) * np.cos(2.0 * math.pi * u[1]))
    return out[0] if ncomp == 1 else np.stack(out, axis=-1)


class HashedMap:
    """A map of ``hashed_normal`` values, indexable like a numpy array (no storage)."""

    def __init__(self, npix: int, seed: int, ncomp: int = 1):
        self.npix, self.seed, self.ncomp = npix, seed, ncomp

    def __getitem__(self, key):
        if isinstance(key, tuple):
            idx, comp = key
            return hashed_normal(idx, self.seed, self.ncomp)[..., comp]
        return hashed_normal(key, self.seed, self.ncomp)
