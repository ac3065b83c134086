"""Shared helpers of the GPU parity tests (inputs from ``workloads`` and the oracle)."""
import itertools

import numpy as np

import workloads as wl
from oracle import kriging as kr
from oracle import sht
from oracle import xi


def require_gpu():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_4984_gb300.build import build

    build()
    import paper_1003_4984_gb300 as fl

    fl.load_library()
    return fl


def oracle_table(cl, cl_bb, spin, K, nside):
    """The oracle's own tabulated correlation function on the documented grid."""
    weight = np.abs(cl) if (spin == 0 or cl_bb is None) else np.abs(cl) + np.abs(cl_bb)
    t_max, n = xi.grid_rule(weight, K, nside)
    if spin == 0:
        tab, x0 = xi.spin0_table(cl, t_max, n)
    elif spin == 1:
        tab, _, x0 = xi.spin1_tables(cl, cl_bb, t_max, n)
    else:
        tab, _, x0 = xi.spin2_tables(cl, cl_bb, t_max, n)
    return tab, x0, t_max, n


def parity_metric(v_gpu, v_ref, sigma):
    return float(np.max(np.abs(v_gpu - v_ref)) / sigma)


def to_host(t):
    return t.detach().cpu().numpy()


def realistic_inputs(nside, lmax, spin, cl, seed_map, seed_phi, l_damp=None):
    """Band-limited map (oracle synthesis) and a lensing deflection grad(phi)."""
    alm = wl.draw_alm(cl, seed_map)
    m = sht.synth_map(nside, lmax, alm, spin=spin)
    if spin == 2:
        m = np.stack([m.real, m.imag], axis=1)
    phi = wl.draw_alm(wl.cl_phiphi(lmax), seed_phi)
    defl = sht.synth_map(nside, lmax, phi, gradient=True)
    return alm, np.ascontiguousarray(m), np.ascontiguousarray(defl)


TIE_REL = 1e-12  # squared chords this close (relative) are an exact tie up to rounding


def unexplained_mismatches(nside, K, spin, maps, targets, v_gpu, s2_gpu, ref, f_plus, x0, sigma, tol):
    """Targets where the GPU result is farther than ``tol`` from the oracle's and no
    exact tie explains it.

    Where pixels tie for the last places of the stencil (squared chords equal to
    TIE_REL, as at the symmetric centres of a finer grid), every choice among them
    is a valid K-nearest set and rounding decides which one each side takes; the
    GPU result must then equal the oracle's estimate on one of those sets."""
    bad = np.nonzero((np.abs(v_gpu - ref.value) > tol * sigma) | (np.abs(s2_gpu - ref.variance) > tol * x0))[0]
    out = []
    if bad.size == 0:
        return out
    idx_all, key_all = kr.knn(nside, targets[bad], K + 8)
    for p, idx, key in zip(bad, idx_all, key_all):
        kK = key[K - 1]
        tied = np.abs(key - kK) <= TIE_REL * kK
        must = idx[key < kK * (1 - TIE_REL)]
        group = idx[tied]
        need = K - must.size
        ok = False
        if group.size > need and not tied[-1]:
            for comb in itertools.combinations(group, need):
                st = np.concatenate([must, np.array(comb, dtype=np.int64)])[None, :]
                v, s2, _ = kr.estimate(nside, spin, maps, targets[p:p + 1], st, f_plus, x0)
                if abs(v[0] - v_gpu[p]) <= tol * sigma and abs(s2[0] - s2_gpu[p]) <= tol * x0:
                    ok = True
                    break
        if not ok:
            out.append(int(p))
    return out
