"""The oracle against numbers the paper prints (tests/golden/paper_values.txt)."""
import numpy as np
import pytest

from oracle import faces as fc
from oracle import healpix as hp
from oracle import kriging as kr
from tests import paper_values as pv


def test_every_printed_value_has_a_citation():
    vals = pv.load()
    assert vals and all(cite and np.isfinite(v) for v, cite in vals.values())


def test_nugget_is_the_printed_epsilon():
    # Sec. 2.4: 1.49e-8, the square root of the double-precision machine epsilon
    assert float(f"{np.sqrt(np.finfo(np.float64).eps):.2e}") == pv.NUGGET_EPSILON_FP64
    assert float(f"{kr.EPS_NUGGET:.2e}") == pv.NUGGET_EPSILON_FP64


@pytest.mark.parametrize("y", [1, 2])
def test_stencil_has_the_printed_pixel_count(y):
    # Sec. 2.3: 9 x 4^(y-1) pixels around a direction whose pixel has 8 neighbours.
    # Directions with |z| < 1/2 are away from the eight points at z = +-2/3 where three
    # base faces meet (the only pixels with 7 neighbours), so every stencil is full.
    N = 64
    rng = np.random.default_rng(y)
    z = rng.uniform(-0.5, 0.5, 200)
    phi = rng.uniform(0, 2 * np.pi, 200)
    s = np.sqrt(1 - z * z)
    tv = np.stack([s * np.cos(phi), s * np.sin(phi), z], 1)
    st = fc.stencil(N, tv, y)
    sizes = np.sum(st >= 0, axis=1)
    assert st.shape[1] == pv.STENCIL_PIXELS[y]
    assert np.all(sizes == pv.STENCIL_PIXELS[y])
    assert np.all([np.unique(r).size == r.size for r in st])
    assert np.all(st < hp.npix(N))
