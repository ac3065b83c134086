"""Spherical-harmonic synthesis for the oracle: the paper's exact benchmark.

Test infrastructure (tests, smoke check, CPU-baseline leg of the benchmark).

Sec. 3.2 measures the interpolator against "the true lensed maps, obtained by
summing exactly the spherical harmonics at the position of interpolation".
This module does that sum, T(n) = sum_lm a_lm Y_lm(n) and, for spin 2,
P(n) = Q + iU = sum_lm a_{2,lm} 2Y_lm(n) with a_{2,lm} = -(E_lm + i B_lm),
using the harmonics of Appendix A.  The per-colatitude Wigner-d sums run in C
(``sht.c``, OpenMP over directions); the sum over m is done here, directly at
arbitrary directions, or by an FFT along each HEALPix ring to make test maps.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import healpix as hp

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "liboracle_sht.so")
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile ``sht.c`` with the host gcc (portable flags only)."""
    src = os.path.join(_HERE, "sht.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-D_DEFAULT_SOURCE", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_theta_coeffs.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp,
                                            ctypes.c_long, dp, dp, dp]
        lib.oracle_theta_coeffs.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def theta_coeffs(lmax: int, mode: int, alm: np.ndarray, blm: np.ndarray | None, theta: np.ndarray):
    """C wrapper: returns complex array (npts, 2, lmax+1) of per-colatitude sums (see sht.c)."""
    lib = _load()
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    er = np.ascontiguousarray(alm.real, dtype=np.float64)
    ei = np.ascontiguousarray(alm.imag, dtype=np.float64)
    br = bi = None
    if blm is not None:
        br = np.ascontiguousarray(blm.real, dtype=np.float64)
        bi = np.ascontiguousarray(blm.imag, dtype=np.float64)
    n = theta.size
    out_re = np.empty((n, 2, lmax + 1))
    out_im = np.empty((n, 2, lmax + 1))
    lib.oracle_theta_coeffs(lmax, mode, _ptr(er), _ptr(ei), _ptr(br), _ptr(bi), n, _ptr(theta),
                            _ptr(out_re), _ptr(out_im))
    return out_re + 1j * out_im


def _angles(vecs: np.ndarray):
    v = np.asarray(vecs, dtype=np.float64)
    theta = np.arctan2(np.sqrt(v[:, 0] ** 2 + v[:, 1] ** 2), v[:, 2])
    phi = np.arctan2(v[:, 1], v[:, 0])
    return theta, phi


def synth_points(lmax: int, alm: np.ndarray, vecs: np.ndarray, spin: int = 0,
                 blm: np.ndarray | None = None, chunk: int = 512) -> np.ndarray:
    """Field at unit vectors ``vecs`` (n, 3): real T for spin 0, complex Q + iU for spin 2."""
    theta, phi = _angles(vecs)
    n = theta.size
    out = np.empty(n, dtype=np.float64 if spin == 0 else np.complex128)
    m = np.arange(lmax + 1)
    for a in range(0, n, chunk):
        th, ph = theta[a:a + chunk], phi[a:a + chunk]
        F = theta_coeffs(lmax, 0 if spin == 0 else 2, alm, blm, th)
        E = np.exp(1j * np.outer(ph, m))
        if spin == 0:
            w = np.where(m == 0, 1.0, 2.0)
            out[a:a + chunk] = np.real(np.sum(w * F[:, 0, :] * E, axis=1))
        else:
            out[a:a + chunk] = np.sum(F[:, 0, :] * E, axis=1) + np.sum(F[:, 1, 1:] * np.conj(E[:, 1:]), axis=1)
    return out


def synth_gradient_points(lmax: int, alm: np.ndarray, vecs: np.ndarray, chunk: int = 512):
    """Gradient (d_theta, d_phi) = (dT/dtheta, dT/dphi / sin theta) of a spin-0 field."""
    theta, phi = _angles(vecs)
    n = theta.size
    dth = np.empty(n)
    dph = np.empty(n)
    m = np.arange(lmax + 1)
    w = np.where(m == 0, 1.0, 2.0)
    for a in range(0, n, chunk):
        th, ph = theta[a:a + chunk], phi[a:a + chunk]
        F = theta_coeffs(lmax, 1, alm, None, th)
        E = np.exp(1j * np.outer(ph, m))
        dth[a:a + chunk] = np.real(np.sum(w * F[:, 1, :] * E, axis=1))
        dph[a:a + chunk] = np.real(np.sum(w * 1j * m * F[:, 0, :] * E, axis=1)) / np.sin(th)
    return dth, dph


def synth_rings(nside: int, rings: np.ndarray, lmax: int, alm: np.ndarray, spin: int = 0,
                blm: np.ndarray | None = None, gradient: bool = False, chunk: int = 256):
    """Field on whole HEALPix rings (1-based indices).

    Returns (pixel indices, values): values real (spin 0), complex (spin 2), or
    an (n, 2) array (d_theta, d_phi) when ``gradient``.  The sum over m is an
    FFT along each ring, with m folded modulo the ring length.
    """
    rings = np.asarray(rings, dtype=np.int64)
    first, n_in, z, s, f, nq = hp.ring_info(nside, rings)
    theta = np.arctan2(s, z)
    mode = 1 if gradient else (0 if spin == 0 else 2)
    pix_all, val_all = [], []
    m = np.arange(lmax + 1)
    for a in range(0, rings.size, chunk):
        F = theta_coeffs(lmax, mode, alm, blm, theta[a:a + chunk])
        for k in range(F.shape[0]):
            r = a + k
            n = int(n_in[r])
            phi0 = f[r] * np.pi / (2.0 * nq[r])

            def ring_sum(Gpos, Gneg):
                H = np.zeros(n, dtype=np.complex128)
                np.add.at(H, m % n, Gpos * np.exp(1j * m * phi0))
                np.add.at(H, (-m[1:]) % n, Gneg[1:] * np.exp(-1j * m[1:] * phi0))
                return n * np.fft.ifft(H)

            if gradient:
                Fv, Gd = F[k, 0], F[k, 1]
                dth = np.real(ring_sum(Gd, np.conj(Gd)))
                dph = np.real(ring_sum(1j * m * Fv, np.conj(1j * m * Fv))) / s[r]
                vals = np.stack([dth, dph], axis=1)
            elif spin == 0:
                vals = np.real(ring_sum(F[k, 0], np.conj(F[k, 0])))
            else:
                vals = ring_sum(F[k, 0], F[k, 1])
            pix_all.append(first[r] + np.arange(n))
            val_all.append(vals)
    return np.concatenate(pix_all), np.concatenate(val_all)


def synth_map(nside: int, lmax: int, alm: np.ndarray, spin: int = 0, blm: np.ndarray | None = None,
              gradient: bool = False) -> np.ndarray:
    """Whole RING map: real (spin 0), complex (spin 2) or (Npix, 2) gradient."""
    pix, vals = synth_rings(nside, np.arange(1, 4 * nside), lmax, alm, spin, blm, gradient)
    out = np.empty((hp.npix(nside),) + vals.shape[1:], dtype=vals.dtype)
    out[pix] = vals
    return out
