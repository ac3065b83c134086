"""Shared helpers of the GPU parity tests (inputs from ``workloads`` and the oracle)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
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
