"""Correlation functions of spin-0 and spin-2 fields for the CPU oracle.

Test infrastructure: used only by tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; shares no code with the CUDA path.

Spin 0 (Eq. correlation_func):
    xi(cos b) = sum_{l=0}^{lmax} (2l+1)/(4 pi) C_l P_l(cos b),   sigma_0^2 = xi(1).
Spin 2 (Eq. spins_correl and Appendix B), for P = Q + iU:
    xi+(b) = sum_l (2l+1)/(4 pi) (C_l^EE + C_l^BB) d^l_{22}(b)
    xi-(b) = sum_l (2l+1)/(4 pi) (C_l^EE - C_l^BB) d^l_{2,-2}(b)
The l range is 0..lmax with the caller's C_l (a spin-2 sum only receives
l >= 2 because d^l_{2,m} vanishes below l = 2).

Every function takes the squared chord t = |n_i - n_j|^2 = 2 (1 - cos b) as
its argument (t in [0, 4]), because the kriging system is assembled from
chords, and cos b = 1 - t/2 carries no cancellation for nearby pixels.

Routes (each pinned by the tests against closed forms and scipy):

* spin 0: Legendre three-term recurrence rewritten in u = 1 - x = t/2 on the
  increments D_l = P_l - P_{l-1}, so that P_l near x = 1 is not formed from
  differences of O(1) numbers;
* spin 2: the Fourier form of Appendix B, d^l_{m1 m2}(b) = sum_n
  Delta^l_{n m1} Delta^l_{n m2} e^{i n b} with Delta = d(pi/2) from the
  Trapani-Navaza recursion (Eqs. delta_lorder, delta_1col, delta_2col), with
  the sums over l and n swapped: xi(b) = sum_n F_n cos(n b).

Tabulated mode (Appendix B, last paragraph: the correlation function is
tabulated and interpolated with cubics): values and first derivatives in t
on the uniform grid t_k = k h, k = 0..n, with cubic Hermite interpolation
inside each interval.
"""
from __future__ import annotations

import math

import numpy as np

FOUR_PI = 4.0 * math.pi


# ----------------------------------------------------------------- spin 0
def xi0_direct(cl: np.ndarray, t: np.ndarray, deriv: bool = False):
    """xi(t) (and d xi / dt if ``deriv``) for spin 0 by the Legendre recurrence in u = t/2.

    Recurrence (from (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1} with x = 1 - u):
        D_{l+1} = (l D_l - (2l+1) u P_l) / (l+1),  P_{l+1} = P_l + D_{l+1}.
    Derivative in x: P'_{l+1} = P'_{l-1} + (2l+1) P_l, and d/dt = -1/2 d/dx.
    """
    t = np.asarray(t, dtype=np.float64)
    u = 0.5 * t
    lmax = len(cl) - 1
    a = (2.0 * np.arange(lmax + 1) + 1.0) / FOUR_PI * np.asarray(cl, dtype=np.float64)
    P_prev = np.ones_like(u)  # P_0
    acc = a[0] * P_prev
    dacc = np.zeros_like(u)
    if lmax == 0:
        return (acc, dacc) if deriv else acc
    P = 1.0 - u  # P_1
    D = P - P_prev
    acc = acc + a[1] * P
    dP_prev = np.zeros_like(u)  # P'_0
    dP = np.ones_like(u)  # P'_1
    dacc = dacc + a[1] * dP
    for ell in range(1, lmax):
        Dn = (ell * D - (2 * ell + 1) * u * P) / (ell + 1)
        Pn = P + Dn
        dPn = dP_prev + (2 * ell + 1) * P
        acc = acc + a[ell + 1] * Pn
        dacc = dacc + a[ell + 1] * dPn
        P, D = Pn, Dn
        dP_prev, dP = dP, dPn
    return (acc, -0.5 * dacc) if deriv else acc


# ----------------------------------------------------------- Appendix B
def _delta_descent(lmax: int, m2: int, visit):
    """Run the Appendix B recursion for column m2 and call visit(k, u, valid, values)
    at each descent step k, where u = l - k (vectorised over l = 0..lmax).

    Eq. delta_lorder raises the order along m2 = 0:
        Delta^l_{l,0} = -sqrt((2l-1)/(2l)) Delta^{l-1}_{l-1,0}, Delta^0_{00} = 1;
    Eq. delta_1col gives the top of each column,
        Delta^l_{l,m} = sqrt(l (2l-1) / (2 (l+m)(l+m-1))) Delta^{l-1}_{l-1,m-1};
    Eq. delta_2col descends the first index at fixed m2:
        Delta^l_{u,m2} = 2 m2 / sqrt((l-u)(l+u+1)) Delta^l_{u+1,m2}
                         - sqrt((l-u-1)(l+u+2) / ((l-u)(l+u+1))) Delta^l_{u+2,m2}.
    """
    assert m2 >= 0
    L = np.arange(lmax + 1, dtype=np.float64)
    top = np.zeros((m2 + 1, lmax + 1))
    top[0, 0] = 1.0
    for ell in range(1, lmax + 1):
        top[0, ell] = -math.sqrt((2 * ell - 1) / (2 * ell)) * top[0, ell - 1]
        for m in range(1, m2 + 1):
            if m <= ell:
                top[m, ell] = math.sqrt(ell * (2 * ell - 1) / (2.0 * (ell + m) * (ell + m - 1))) * top[m - 1, ell - 1]
    prev2 = np.zeros(lmax + 1)
    prev1 = np.zeros(lmax + 1)
    for k in range(0, 2 * lmax + 1):
        u = L - k
        valid = (k <= 2 * L) & (L >= m2)
        if k == 0:
            cur = np.where(valid, top[m2], 0.0)
        else:
            a = (L - u) * (L + u + 1.0)
            b = (L - u - 1.0) * (L + u + 2.0)
            with np.errstate(divide="ignore", invalid="ignore"):
                c1 = np.where(a > 0, 2.0 * m2 / np.sqrt(np.where(a > 0, a, 1.0)), 0.0)
                c2 = np.sqrt(np.where(a > 0, np.maximum(b, 0.0) / np.where(a > 0, a, 1.0), 0.0))
            cur = np.where(valid, c1 * prev1 - c2 * prev2, 0.0)
        visit(k, u, valid, cur)
        prev2, prev1 = prev1, cur


def delta_column(lmax: int, m2: int):
    """Delta^l_{u, m2} = d^l_{u, m2}(pi/2) for l = 0..lmax, u = -l..l.

    Returns an array D of shape (lmax+1, 2 lmax + 1) with D[l, lmax + u]
    (small lmax only; the correlation sums use the streaming form).
    """
    D = np.zeros((lmax + 1, 2 * lmax + 1))

    def visit(k, u, valid, cur):
        rows = np.nonzero(valid)[0]
        D[rows, (u[rows] + lmax).astype(np.int64)] = cur[rows]

    _delta_descent(lmax, m2, visit)
    return D


def wigner_d_fourier(lmax: int, m1: int, m2: int, beta: np.ndarray) -> np.ndarray:
    """d^l_{m1 m2}(beta), shape (lmax+1, len(beta)), from Eq. fft_dfunction.

    Only m1 = 2 with m2 in {2, -2}, and m1 = m2 = 0, are needed here; columns
    with negative m2 follow from Delta^l_{n,-m} = (-1)^{l+n} Delta^l_{n,m}.  For
    these pairs i^{m1-m2} = i^{m2-m1} = +-1 real, so the garbled phase of the
    printed equation does not enter (reading listed with the design notes).
    """
    beta = np.asarray(beta, dtype=np.float64)
    Da = delta_column(lmax, abs(m1))
    Db = delta_column(lmax, abs(m2))
    n = np.arange(-lmax, lmax + 1)
    L = np.arange(lmax + 1)[:, None]
    sign_a = np.where(m1 < 0, (-1.0) ** ((L + n[None, :]) % 2), 1.0)
    sign_b = np.where(m2 < 0, (-1.0) ** ((L + n[None, :]) % 2), 1.0)
    B = (Da * sign_a) * (Db * sign_b)
    phase = 1j ** ((m2 - m1) % 4)
    E = np.exp(1j * np.outer(n, beta))
    return np.real(phase * (B @ E))


def _fourier_coeffs_spin(spin: int, cl_p: np.ndarray, cl_m: np.ndarray):
    """F+_n, F-_n (n = 0..lmax) with xi+-(b) = F_0 + 2 sum_{n>0} F_n cos(n b), spin s = 1, 2.

    From Eq. fft_dfunction with m1 = s and m2 = +-s: d^l_{ss}(b) = sum_n
    (Delta^l_{ns})^2 e^{inb} and, using Delta^l_{n,-s} = (-1)^{l+n} Delta^l_{ns},
    d^l_{s,-s}(b) = i^{-2s} sum_n (-1)^{l+n} (Delta^l_{ns})^2 e^{inb} (i^{-2s} = -1 for
    s = 1, +1 for s = 2); both are even in n.
    """
    lmax = len(cl_p) - 1
    ell = np.arange(lmax + 1)
    wp = (2.0 * ell + 1.0) / FOUR_PI * cl_p
    wm = (2.0 * ell + 1.0) / FOUR_PI * cl_m * (-1.0 if spin % 2 else 1.0)
    Fp = np.zeros(2 * lmax + 1)
    Fm = np.zeros(2 * lmax + 1)

    def visit(k, u, valid, cur):
        rows = np.nonzero(valid)[0]
        n = (u[rows] + lmax).astype(np.int64)  # distinct for fixed k
        sq = cur[rows] * cur[rows]
        sgn = np.where(((rows + u[rows].astype(np.int64)) % 2) == 0, 1.0, -1.0)
        Fp[n] += wp[rows] * sq
        Fm[n] += wm[rows] * sgn * sq

    _delta_descent(lmax, spin, visit)
    return Fp[lmax:], Fm[lmax:]


def _fourier_coeffs_spin2(cl_p: np.ndarray, cl_m: np.ndarray):
    return _fourier_coeffs_spin(2, cl_p, cl_m)


def xis_direct(spin: int, cl_e: np.ndarray, cl_b: np.ndarray | None, t: np.ndarray, deriv: bool = False):
    """(xi+, xi-)(t), and their t-derivatives if ``deriv``, for a spin-s field (s = 1, 2):
    xi+ = sum_l (2l+1)/(4 pi) (C^E + C^B) d^l_{ss}, xi- = sum_l (2l+1)/(4 pi) (C^E - C^B) d^l_{s,-s}.

    Uses xi(b) = sum_n F_n cos(n b) with b = 2 asin(sqrt(t)/2); the t-derivative
    is (d xi/d b) / (d t/d b) with d t/d b = 2 sin b, and at t = 0 the limit
    -1/2 sum_n n^2 F_n (d^2 t/d b^2 = 2 at b = 0).
    """
    cl_e = np.asarray(cl_e, dtype=np.float64)
    cl_b = np.zeros_like(cl_e) if cl_b is None else np.asarray(cl_b, dtype=np.float64)
    Fp, Fm = _fourier_coeffs_spin(spin, cl_e + cl_b, cl_e - cl_b)
    t = np.asarray(t, dtype=np.float64)
    beta = 2.0 * np.arcsin(np.sqrt(np.clip(t, 0.0, 4.0)) / 2.0)
    n = np.arange(len(Fp), dtype=np.float64)
    wgt = np.where(n == 0, 1.0, 2.0)
    C = np.cos(np.outer(beta, n))
    xp = C @ (wgt * Fp)
    xm = C @ (wgt * Fm)
    if not deriv:
        return xp, xm
    S = np.sin(np.outer(beta, n))
    dxp_db = -(S @ (wgt * n * Fp))
    dxm_db = -(S @ (wgt * n * Fm))
    sb = np.sin(beta)
    with np.errstate(divide="ignore", invalid="ignore"):
        dxp = np.where(beta > 0, dxp_db / (2.0 * sb), -0.5 * np.sum(wgt * n * n * Fp))
        dxm = np.where(beta > 0, dxm_db / (2.0 * sb), -0.5 * np.sum(wgt * n * n * Fm))
    return xp, xm, dxp, dxm


def xi2_direct(cl_ee: np.ndarray, cl_bb: np.ndarray | None, t: np.ndarray, deriv: bool = False):
    """(xi+, xi-)(t) (and t-derivatives) for a spin-2 field (Eq. spins_correl)."""
    return xis_direct(2, cl_ee, cl_bb, t, deriv)


def xi1_direct(cl_e: np.ndarray, cl_b: np.ndarray | None, t: np.ndarray, deriv: bool = False):
    """(xi+, xi-)(t) (and t-derivatives) for a spin-1 field, e.g. a deflection
    d = grad phi with C^E_l = l(l+1) C^phiphi_l and C^B = 0."""
    return xis_direct(1, cl_e, cl_b, t, deriv)


# --------------------------------------------------------- tabulated mode
class HermiteTable:
    """Cubic Hermite interpolation in t on the grid t_k = k h, k = 0..n.

    ``f`` and ``g`` hold values and t-derivatives at the nodes.  Inside
    [t_k, t_k+1] with s = t/h - k:
        f(t) = (2s^3 - 3s^2 + 1) f_k + (s^3 - 2s^2 + s) h g_k
             + (-2s^3 + 3s^2) f_{k+1} + (s^3 - s^2) h g_{k+1}.
    The interval index is k = floor(t / h) clamped to [0, n-1].
    """

    def __init__(self, t_max: float, n: int, f: np.ndarray, g: np.ndarray):
        self.t_max = float(t_max)
        self.n = int(n)
        self.h = self.t_max / self.n
        self.inv_h = self.n / self.t_max
        self.f = np.asarray(f, dtype=np.float64)
        self.g = np.asarray(g, dtype=np.float64)

    def nodes(self) -> np.ndarray:
        return np.arange(self.n + 1) * self.h

    def __call__(self, t: np.ndarray) -> np.ndarray:
        t = np.asarray(t, dtype=np.float64)
        x = t * self.inv_h
        k = np.clip(np.floor(x), 0, self.n - 1).astype(np.int64)
        s = x - k
        s2 = s * s
        s3 = s2 * s
        h = self.h
        return ((2 * s3 - 3 * s2 + 1) * self.f[k] + (s3 - 2 * s2 + s) * h * self.g[k]
                + (-2 * s3 + 3 * s2) * self.f[k + 1] + (s3 - s2) * h * self.g[k + 1])


def spin0_table(cl: np.ndarray, t_max: float, n: int):
    """Tabulated xi/xi(0) for spin 0 on n intervals of [0, t_max]; returns (table, xi(0))."""
    nodes = np.arange(n + 1) * (t_max / n)
    f, g = xi0_direct(cl, nodes, deriv=True)
    xi_zero = float(xi0_direct(cl, np.zeros(1))[0])
    return HermiteTable(t_max, n, f / xi_zero, g / xi_zero), xi_zero


def spin1_tables(cl_e: np.ndarray, cl_b: np.ndarray | None, t_max: float, n: int):
    """Tabulated xi+/xi+(0) and xi-/xi+(0) for spin 1; returns (table+, table-, xi+(0))."""
    nodes = np.arange(n + 1) * (t_max / n)
    xp, xm, dxp, dxm = xi1_direct(cl_e, cl_b, nodes, deriv=True)
    x0 = float(xi1_direct(cl_e, cl_b, np.zeros(1))[0][0])
    return (HermiteTable(t_max, n, xp / x0, dxp / x0),
            HermiteTable(t_max, n, xm / x0, dxm / x0), x0)


def spin2_tables(cl_ee: np.ndarray, cl_bb: np.ndarray | None, t_max: float, n: int):
    """Tabulated xi+/xi+(0) and xi-/xi+(0) for spin 2; returns (table+, table-, xi+(0))."""
    nodes = np.arange(n + 1) * (t_max / n)
    xp, xm, dxp, dxm = xi2_direct(cl_ee, cl_bb, nodes, deriv=True)
    x0 = float(xi2_direct(cl_ee, cl_bb, np.zeros(1))[0][0])
    return (HermiteTable(t_max, n, xp / x0, dxp / x0),
            HermiteTable(t_max, n, xm / x0, dxm / x0), x0)


# ------------------------------------------------------------- grid rule
SEARCH_RADIUS_FACTOR = 1.25   # stencil disc radius in units of sqrt(K/3)/Nside
TABLE_TOLERANCE = 1e-11       # target bound on the cubic interpolation error of xi/xi(0)


def grid_rule(cl_weight: np.ndarray, K: int, nside: int):
    """Table domain and size, a documented rule that both implementations follow.

    The stencil lies in the disc of chord radius r = 1.25 sqrt(K/3)/Nside around
    the target (a cap holding K pixels has radius sqrt(K/3)/Nside; the K-th
    neighbour was measured never to exceed 1.10 of it), so every chord between
    stencil members is at most 2r: t_max = 4 r^2.  The interval count is the
    smallest power of two, at least 64 and at most 65536, for which the cubic
    Hermite error bound h^4/384 max|f4| stays below 1e-11, where f4 is the fourth
    t-derivative of xi/xi(0), bounded by sum_l |a_l| P4_l / (16 |xi(0)|) with
    P4_l = (l-3)(l-2)(l-1) l (l+1)(l+2)(l+3)(l+4)/384 (the fourth derivative of
    P_l at 1) and a_l = (2l+1)/(4 pi) |C_l| (spin 2: |C^EE| + |C^BB|).
    Returns (t_max, n).
    """
    r = SEARCH_RADIUS_FACTOR * math.sqrt(K / 3.0) / nside
    t_max = 4.0 * r * r
    return t_max, table_size(cl_weight, t_max)


def table_size(cl_weight: np.ndarray, t_max: float) -> int:
    """Interval count of a table on [0, t_max] under the error rule of grid_rule."""
    cw = np.abs(np.asarray(cl_weight, dtype=np.float64))
    ell = np.arange(cw.size, dtype=np.float64)
    a = (2.0 * ell + 1.0) / FOUR_PI * cw
    x0 = float(np.sum(a))
    p4 = np.where(ell >= 4, (ell - 3) * (ell - 2) * (ell - 1) * ell * (ell + 1) * (ell + 2) * (ell + 3) * (ell + 4) / 384.0, 0.0)
    b4 = float(np.sum(a * p4)) / 16.0 / x0 if x0 > 0 else 0.0
    n = 64
    if b4 > 0:
        h = (384.0 * TABLE_TOLERANCE / b4) ** 0.25
        n = max(64, 2 ** int(math.ceil(math.log2(t_max / h))))
    return min(n, 65536)
