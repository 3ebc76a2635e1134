"""GPU stability diagnostics (ebr_stats, Eq. stability_alpha_max) against the
oracle: per-geometry extrema of alpha_i = (x_s - x_1)_i / (x_2 - x_1)_i within
1e-12, the alpha histogram (bin for bin, except ghosts whose alpha lies within
1e-10 of a bin edge), the r_i and level histograms exactly; and the paper's
printed maxima for a unit-diameter cylinder at dx = 0.015 (Sec. 8.1: CGC
0.924, HGC 0.464) as a loose check (the body's offset to the grid is not
given)."""

import numpy as np
import pytest

import oracle as O
from paper_2609_10165_b300 import inputs as I
from paper_2609_10165_b300.api import Reconstructor
from tests.test_gpu_parity import _small_cases
from tests.test_oracle_stretched import CASES as STRETCHED

pytestmark = pytest.mark.gpu


def _oracle_alpha(c):
    d = c.grid.dim
    x2 = c.x2 if c.x2 is not None else c.r * c.e * np.array(c.grid.h)[None, :]
    return c.psi[:, None] * c.n / x2


@pytest.mark.parametrize("placement,layers", [("HGC", 1), ("CGC", 1), ("CGC_ES", 1), ("HGC", 2)])
def test_stats_match_the_oracle(placement, layers):
    cases = [c for c in _small_cases()] + [{"grid": g, "body": b} for g, b in STRETCHED]
    for case in cases:
        R = Reconstructor(case["grid"], case["body"], placement, layers=layers)
        R.build_levels()
        st = R.stats(n_bins=60)
        c = O.classify(case["grid"], case["body"], placement, layers=layers)
        lev = O.build_levels(c)
        al = _oracle_alpha(c)
        d = c.grid.dim
        assert np.allclose(st["alpha_max"][0], al.max(0), rtol=0, atol=1e-12)
        assert np.allclose(st["alpha_min"][0], al.min(0), rtol=0, atol=1e-12)
        edges = st["bin_edges"]
        for a in range(d):
            want = np.histogram(np.clip(al[:, a], -0.5, 1.0 - 1e-15), bins=edges)[0]
            near = np.min(np.abs(al[:, a][:, None] - edges[None, :]), axis=1) < 1e-10
            assert np.sum(np.abs(st["alpha_hist"][a] - want)) <= 2 * int(near.sum()), a
            assert np.array_equal(st["r_hist"][a][:16], np.bincount(c.r[:, a], minlength=16)[:16])
        lh = np.bincount(lev.level, minlength=st["level_hist"].size + 1)[1:st["level_hist"].size + 1]
        assert np.array_equal(st["level_hist"], lh)


def test_cylinder_alpha_near_the_printed_values():
    # unit-diameter cylinder, dx = 0.015: CGC max alpha 0.924 and HGC 0.464 in Sec. 8.1
    gd = I.grid(2, [400, 400], [-3.0, -3.0], [3.0, 3.0])
    bd = I.circle(0.0031, 0.0017, 0.5)
    out = {}
    for pl in ("HGC", "CGC", "CGC_ES"):
        R = Reconstructor(gd, bd, pl)
        R.build_levels()
        out[pl] = R.stats()["alpha_max"][0]
    assert 0.4 < out["HGC"].max() <= 0.5
    assert 0.85 < out["CGC"].max() < 1.0
    assert out["CGC_ES"].max() <= 0.5 + 1e-12
