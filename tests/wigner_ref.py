"""Independent reference for Wigner d^j_{m'm}(beta): the Jacobi-polynomial closed form.

d^j_{m'm}(b) = (-1)^lam sqrt(C(2j-k, k+a) / C(k+b, b)) sin(b/2)^a cos(b/2)^b P_k^{(a,b)}(cos b)
with k = min(j+m, j-m, j+m', j-m'), and (a, lam) = (m'-m, m'-m) if k is j+m or
j-m', (m-m', 0) otherwise; b = 2j - 2k - a.  P_k^{(a,b)} is scipy's
``eval_jacobi``, so this reference shares nothing with the oracle's routes.
"""
import math

import numpy as np
from scipy.special import eval_jacobi


def wigner_d(j: int, mp: int, m: int, beta) -> np.ndarray:
    beta = np.asarray(beta, dtype=np.float64)
    if abs(m) > j or abs(mp) > j:
        return np.zeros_like(beta)
    cands = [(j + m, "jm+"), (j - m, "jm-"), (j + mp, "jmp+"), (j - mp, "jmp-")]
    k, which = min(cands, key=lambda c: c[0])
    if which in ("jm+", "jmp-"):
        a = mp - m
        lam = mp - m
    else:
        a = m - mp
        lam = 0
    b = 2 * j - 2 * k - a
    pref = (-1.0) ** lam * math.sqrt(math.comb(2 * j - k, k + a) / math.comb(k + b, b))
    return pref * np.sin(beta / 2) ** a * np.cos(beta / 2) ** b * eval_jacobi(k, a, b, np.cos(beta))
