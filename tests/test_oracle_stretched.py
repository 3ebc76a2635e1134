"""Pins of the oracle on stretched grids (per-cell widths; Sec. 7: Eq.
stencil_anisotropic with the local mesh spacing dx_i, Eq. delta_n with the
ghost's own widths; the 3 % per cell stretching of the meshes of Secs. 8.1 and
8.2, applied here around the bodies so that the stencils see it).

- The closed forms with the stencil's actual x_2 - x_1 equal the Appendix A
  Vandermonde solve, and the level-by-level fill reproduces (bi/tri)linear
  fields exactly, for every placement and with the second layer.
- Faces of a uniform grid given explicitly give the uniform classification.
- Brute-force classification (psi on every cell) agrees.
- Second-order convergence of the fill and O(dx) convergence of the surface
  weights to the perimeter on stretched grids."""

import math

import numpy as np
import pytest

import oracle as O
from paper_2609_10165_b300 import inputs as I

CASES = [
    (I.stretched_grid(2, [48, 44], [-1.0, -1.0], [1.0, 1.0], ratio=(1.03, 1.03)), I.ellipse(0.03, -0.02, 0.6, 0.35, 0.7)),
    (I.stretched_grid(2, [150, 70], [-1.0, -1.0], [3.0, 1.0], ratio=(1.02, 1.03), centre_frac=(0.35, 0.5)),
     I.airfoil(0.0, 0.0, 0.12, 1.0, 5.0)),
    (I.stretched_grid(3, [22, 20, 21], [-1.0, -1.0, -1.0], [1.0, 1.0, 1.0]), I.sphere(0.02, -0.01, 0.03, 0.6)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_stretched_grids_are_stretched(case):
    gd, _ = CASES[case]
    g = O.Grid.from_dict(gd)
    for a in range(g.dim):
        ratio = g.wid[a][1:] / g.wid[a][:-1]
        assert ratio.max() > 1.01 and ratio.max() <= 1.0301
    assert g.stretched


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("placement,layers", [("HGC", 1), ("CGC", 1), ("CGC_ES", 1), ("HGC", 2), ("CGC_ES", 2)])
def test_stretched_fill_reproduces_multilinear_fields(case, placement, layers):
    gd, bd = CASES[case]
    d = gd["dim"]
    c = O.classify(gd, bd, placement, layers=layers)
    assert c.ties == [] and c.x2 is not None
    lev = O.build_levels(c)
    X = c.grid.centre(c.grid.unlin(c.idx))
    S = (X + c.psi[:, None] * c.n)[lev.order]
    nn = c.n[lev.order]
    fields = [I.Polynomial(d, 700 + case), I.Polynomial(d, 800 + case)]
    kinds = [O.DIRICHLET, O.NEUMANN]
    arrs = [f.on_grid(gd) for f in fields]
    for a in arrs:
        a[c.idx] = 1e30
    out = O.fill(c, lev, arrs, kinds, [I.bc_values(f, k, S, nn) for f, k in zip(fields, kinds)])
    for f, a in zip(fields, out):
        assert np.max(np.abs(a[c.idx] - f.value(X))) < 1e-11
        ps, gr = O.boundary_quantities(c, lev, a)
        assert np.max(np.abs(ps - f.value(S))) < 1e-10
        assert np.max(np.abs(gr - f.gradient(S))) < 1e-8
    # the stencil spacing is not r e h: the grid really is non-uniform there
    h = np.array(c.grid.h)
    assert np.max(np.abs(np.abs(c.x2) / c.r - h[None, :])) > 1e-3 * h.min()


@pytest.mark.parametrize("case", range(len(CASES)))
def test_stretched_closed_forms_equal_vandermonde(case):
    gd, bd = CASES[case]
    c = O.classify(gd, bd, "CGC_ES")
    rng = np.random.default_rng(60 + case)
    K = 3 if gd["dim"] == 2 else 7
    for g in range(0, c.n_ghosts, max(1, c.n_ghosts // 25)):
        pm = rng.normal(size=K)
        datum = rng.normal()
        for bc in (O.DIRICHLET, O.NEUMANN):
            args = (c.grid.h, c.psi[g], c.n[g], c.e[g], c.r[g], bc, pm, datum)
            a = O.ghost_value(*args, x2=c.x2[g])
            b = O.vandermonde_ghost_value(*args, x2=c.x2[g])
            assert abs(a - b) <= 1e-10 * (1 + abs(b)), (g, bc, a, b)


def test_uniform_faces_reduce_to_the_uniform_grid():
    gu = I.grid(2, [64, 60], [-1.0, -1.0], [1.0, 1.0])
    gf = dict(gu)
    gf["faces"] = [np.linspace(-1.0, 1.0, 65).tolist(), np.linspace(-1.0, 1.0, 61).tolist()]
    bd = I.ellipse(0.03, -0.02, 0.6, 0.35, 0.7)
    for pl in ("HGC", "CGC_ES"):
        cu = O.classify(gu, bd, pl)
        cf = O.classify(gf, bd, pl)
        assert np.array_equal(cu.tags, cf.tags) and np.array_equal(cu.idx, cf.idx)
        assert np.array_equal(cu.r, cf.r)
        assert np.max(np.abs(cu.psi - cf.psi)) < 1e-14
        assert np.max(np.abs(cf.x2 - cf.r * cf.e * np.array(cu.grid.h))) < 1e-14


@pytest.mark.parametrize("case", range(len(CASES)))
def test_stretched_brute_force_classification(case):
    gd, bd = CASES[case]
    for pl in ("HGC", "CGC"):
        c = O.classify(gd, bd, pl)
        cb = O.classify(gd, bd, pl, cells=np.arange(c.grid.N))
        assert np.array_equal(c.tags, cb.tags) and np.array_equal(c.idx, cb.idx)


def test_stretched_convergence_and_perimeter():
    f = I.CylinderU()
    errs, perim = [], []
    for n in (96, 192, 384):
        gd = I.stretched_grid(2, [n, n], [-2.0, -2.0], [2.0, 2.0], ratio=(1.0 + 3.0 / n, 1.0 + 3.0 / n))
        bd = I.circle(0.0031, 0.0017, 0.5)
        c = O.classify(gd, bd, "HGC")
        lev = O.build_levels(c)
        X = c.grid.centre(c.grid.unlin(c.idx))
        S = (X + c.psi[:, None] * c.n)[lev.order]
        out = O.fill(c, lev, [f.on_grid(gd)], [O.DIRICHLET], [I.bc_values(f, 0, S, c.n[lev.order])])[0]
        errs.append(np.max(np.abs(out[c.idx] - f.value(X))))
        perim.append(abs(O.face_weights(c).sum() - 2 * math.pi * 0.5))
    assert errs[0] / errs[2] > 8.0, errs
    assert perim[2] < 0.5 * perim[0] and perim[2] < 2 * max(O.Grid.from_dict(gd).hmax), perim
