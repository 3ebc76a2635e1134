"""Pins of the oracle's second ghost layer (Sec. 7, "Additional ghost-cell
layers": solid cells with psi <= 1.5 dn join the ghost set; Eq.
stencil_anisotropic gives every ghost its stencil multipliers).

- Closed form on a circle with unit cells: dn = 1 for every normal (Eq.
  delta_n), so the second layer is exactly the solid cells with centre
  radius >= R - 1.5 that the first layer left solid, and r_i = max(1,
  ceil(2 (R - |x|) |x_i| / |x|)).
- The candidate box (layer_reach) loses nothing: evaluating psi on every
  cell gives the same ghost set, on isotropic and anisotropic grids.
- The fill reproduces (bi/tri)linear fields exactly through both layers.
- Every ghost satisfies the normalized-distance bound of Eq.
  stencil_anisotropic: |x_1,i - x_s,i| / (r_i dx_i) <= 1/2."""

import math

import numpy as np
import pytest

import oracle as O
from paper_2609_10165_b300 import inputs as I


@pytest.mark.parametrize("n,R", [(12, 3.75), (64, 20.3), (97, 31.1)])
def test_circle_second_layer_closed_form(n, R):
    gd = I.grid(2, [n, n], [-n / 2, -n / 2], [n / 2, n / 2])       # unit cells
    bd = I.circle(0.0, 0.0, R)
    c1 = O.classify(gd, bd, "HGC")
    c2 = O.classify(gd, bd, "HGC", layers=2)
    g = c1.grid
    X = g.centre(g.unlin(np.arange(g.N)))
    rad = np.sqrt((X ** 2).sum(1))
    want = (c1.tags == 1) & (rad >= R - 1.5) & (rad <= R)
    added = np.setdiff1d(c2.idx, c1.idx)
    assert np.array_equal(added, np.nonzero(want)[0])
    assert set(c1.idx.tolist()) <= set(c2.idx.tolist())
    # r_i of every solid ghost from psi = R - |x|, n = x / |x|
    sel = c2.tags[c2.idx] == 2
    xs = X[c2.idx[sel]]
    rr = rad[c2.idx[sel]]
    r_want = np.maximum(1, np.ceil(2 * (R - rr)[:, None] * np.abs(xs) / rr[:, None]))
    assert np.array_equal(c2.r[sel], r_want.astype(np.int64))
    # the first layer keeps r = 1 (HGC: |n_i psi| / dx_i <= 1/2)
    first = np.isin(c2.idx, c1.idx)
    assert np.all(c2.r[first] == 1)


CASES = [
    (I.grid(2, [40, 36], [-1.0, -1.0], [1.0, 1.0]), I.ellipse(0.03, -0.02, 0.6, 0.35, 0.7)),
    (I.grid(2, [131, 67], [-1.0, -1.0], [3.0, 1.0]), I.airfoil(0.0, 0.0, 0.12, 1.0, 5.0)),
    (I.grid(2, [96, 96], [-1.0, -1.0], [3.0, 1.0]), I.airfoil(0.0, 0.0, 0.15, 1.0, 7.0)),   # dx = 2 dy
    (I.grid(3, [21, 18, 19], [-1.0, -1.0, -1.0], [1.0, 1.0, 1.0]), I.sphere(0.02, -0.01, 0.03, 0.6)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("placement", ["HGC", "CGC_ES"])
def test_candidate_box_is_complete(case, placement):
    gd, bd = CASES[case]
    c = O.classify(gd, bd, placement, layers=2)
    assert c.ties == []
    # brute force: psi on every cell, as candidates of both layers
    N = c.grid.N
    cb = O.classify(gd, bd, placement, cells=np.arange(N), layers=2, layer_cells=np.arange(N))
    assert np.array_equal(c.tags, cb.tags)
    assert np.array_equal(c.idx, cb.idx)
    assert np.array_equal(c.r, cb.r)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("placement", ["HGC", "CGC_ES"])
def test_two_layers_reproduce_multilinear_fields(case, placement):
    gd, bd = CASES[case]
    d = gd["dim"]
    c = O.classify(gd, bd, placement, layers=2)
    lev = O.build_levels(c)
    X = c.grid.centre(c.grid.unlin(c.idx))
    S = (X + c.psi[:, None] * c.n)[lev.order]
    nn = c.n[lev.order]
    fields = [I.Polynomial(d, 500 + case), I.Polynomial(d, 600 + case)]
    kinds = [O.DIRICHLET, O.NEUMANN]
    arrs = [f.on_grid(gd) for f in fields]
    for a in arrs:
        a[c.idx] = 1e30                       # ghost slots must be overwritten
    out = O.fill(c, lev, arrs, kinds, [I.bc_values(f, k, S, nn) for f, k in zip(fields, kinds)])
    for f, a in zip(fields, out):
        assert np.max(np.abs(a[c.idx] - f.value(X))) < 1e-11
    # the normalized distance of every ghost is at most 1/2 (Eq. stencil_anisotropic)
    h = np.array(c.grid.h)
    q = np.abs(c.psi[:, None] * c.n) / (c.r * h[None, :])
    assert q.max() <= 0.5 + 1e-12
    # the second layer deepens the chains: some ghost depends on a ghost
    assert lev.n_levels >= 2


def test_layer_reach_bound():
    # isotropic 2D / 3D: 3 cells; dx = 2 dy: 3 cells along x, 5 along y
    assert O.classify.__globals__["layer_reach"](O.Grid(2, [8, 8], [0, 0], [8, 8])) == [3, 3]
    assert O.classify.__globals__["layer_reach"](O.Grid(3, [8, 8, 8], [0] * 3, [8] * 3)) == [3, 3, 3]
    assert O.classify.__globals__["layer_reach"](O.Grid(2, [8, 8], [0, 0], [16, 8])) == [3, 5]


def test_candidate_at_a_sphere_centre():
    # a 17^3 grid whose centre cell is the sphere's centre: the candidate box
    # reaches it; at depth R > 1.5 h it stays solid (the normal is undefined
    # there, and no dn admits it)
    gd = I.grid(3, [17, 17, 17], [-1.0, -1.0, -1.0], [1.0, 1.0, 1.0])
    c = O.classify(gd, I.sphere(0.0, 0.0, 0.0, 0.55), "HGC", layers=2)
    centre = int(c.grid.lin(np.array([[8, 8, 8]]))[0])
    assert c.tags[centre] == 1
    O.build_levels(c)
    # the same body as a brute-force check of the whole layer
    cb = O.classify(gd, I.sphere(0.0, 0.0, 0.0, 0.55), "HGC", layers=2,
                    layer_cells=np.setdiff1d(np.arange(c.grid.N), [centre]))
    assert np.array_equal(c.idx, cb.idx)
