"""GPU harmonic synthesis (flints_synthesize) against the oracle's synthesis:
whole small skies (spin 0, the spin-1 gradient of a potential, spin 2 Q/U,
band limits above 2 Nside so that ring folding is exercised) and sampled
rings of the full-size Nside 2048 / 4096, lmax 4096 maps of the lensing
workloads.  Tolerance: max |gpu - oracle| <= 1e-10 of the map's rms for the
FP64 recurrence (both are FP64 sums of the same series, differing in rounding
order), 1e-9 for the double-float recurrence (about 2^-44 per operation over
up to 4096 recurrence steps; 1.1e-10 measured at lmax 4096)."""

TOL = {"fp64": 1e-10, "mixed": 1e-9}
import numpy as np
import pytest

import workloads as wl
from oracle import sht
from tests.gpu_common import require_gpu, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fl():
    return require_gpu()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _gpu(fl, torch, nside, lmax, spin, alm, blm=None, precision="fp64"):
    s = fl.Synth(nside, lmax, spin, precision)
    out = s.run(_dev(torch, alm), None if blm is None else _dev(torch, blm))
    torch.cuda.synchronize()
    s.close()
    v = to_host(out)
    return v if spin == 0 else v[:, 0] + 1j * v[:, 1]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.sqrt(np.mean(np.abs(b) ** 2)))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nside,lmax", [(16, 32), (8, 40), (1, 4), (32, 50)])
def test_spin0_whole_sky(fl, nside, lmax, precision):
    import torch

    alm = wl.draw_alm(wl.cl_tt(lmax, 0.7 * lmax), 11)
    ref = sht.synth_map(nside, lmax, alm)
    assert _rel(_gpu(fl, torch, nside, lmax, 0, alm, precision=precision), ref) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nside,lmax", [(16, 32), (8, 40)])
def test_spin2_whole_sky(fl, nside, lmax, precision):
    import torch

    cl = wl.cl_ee(lmax, 0.7 * lmax)
    alm, blm = wl.draw_alm(cl, 12), wl.draw_alm(0.4 * cl, 13)
    ref = sht.synth_map(nside, lmax, alm, spin=2, blm=blm)
    assert _rel(_gpu(fl, torch, nside, lmax, 2, alm, blm, precision), ref) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nside,lmax", [(16, 32), (8, 40)])
def test_spin1_gradient_whole_sky(fl, nside, lmax, precision):
    # the deflection d = grad phi as the spin-1 field with E_lm = sqrt(l(l+1)) phi_lm
    import torch

    phi = wl.draw_alm(wl.cl_phiphi(lmax), 14)
    ell = np.arange(lmax + 1)
    e = phi * np.sqrt(ell * (ell + 1.0))[:, None]
    g = sht.synth_map(nside, lmax, phi, gradient=True)
    assert _rel(_gpu(fl, torch, nside, lmax, 1, e, precision=precision), g[:, 0] + 1j * g[:, 1]) <= TOL[precision]


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("W", [wl.C2, wl.C3], ids=["c2", "c3"])
def test_fullsize_sampled_rings(fl, W, precision):
    # the Nside 2048 (spin 0) and Nside 4096 (spin 2) maps at lmax 4096, checked on
    # rings of the north cap, the cap/belt boundary, the equator and the south cap
    import torch

    cl, bb = W.cl()
    alm = wl.draw_alm(cl, W.seed_map)
    blm = None if W.spin == 0 else wl.draw_alm(bb, W.seed_map + 1) if bb is not None and np.any(bb) else None
    got = _gpu(fl, torch, W.nside, W.lmax, W.spin, alm, blm, precision)
    rings = np.array([3, W.nside // 2, W.nside, W.nside + 1, 2 * W.nside, 4 * W.nside - 7])
    pix, ref = sht.synth_rings(W.nside, rings, W.lmax, alm, spin=W.spin, blm=blm)
    assert _rel(got[pix], ref) <= TOL[precision]
