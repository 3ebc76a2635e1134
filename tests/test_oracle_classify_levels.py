"""Pins of the oracle's classification (Sec. 3.1) and dependency levels
(Sec. 3.2): the paper's worked examples (Figs. 2 and 3), brute force on tiny
grids, and the stability invariants the placements guarantee (Sec. 7-8)."""

import os

import networkx as nx
import numpy as np
import pytest

import oracle as O
from oracle.classify import Classification, EBRError, stencil_members
from paper_2609_10165_b300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _fig3(placement):
    g = O.Grid(2, [12, 12], [-6, -6], [6, 6])
    b = O.Body("circle", [0, 0, 0], [3.75, 3.75, 0])
    return g, b, O.classify(g, b, placement)


@pytest.mark.parametrize("placement", ["CGC", "HGC"])
def test_fig3_ghost_sets(placement):
    g, b, c = _fig3(placement)
    want = {(float(r[1]), float(r[2])): (float(r[3]), float(r[4]))
            for r in _read("fig3_circle_ghosts.txt") if r[0] == placement}
    X = g.centre(g.unlin(c.idx))
    got = {(x[0], x[1]): k for k, x in enumerate(X) if x[0] > 0 and x[1] > 0}
    assert set(got) == set(want)
    # four symmetric quadrants
    assert c.n_ghosts == 4 * len(want)
    # drawn boundary points S = G + psi n (drawn coordinates: +-0.03)
    for key, s in want.items():
        k = got[key]
        S = X[k] + c.psi[k] * c.n[k]
        assert np.hypot(*(S - np.array(s))) < 0.03, (key, S, s)
    # HGC places ghosts on both sides: (1.5,3.5) and (3.5,1.5) are fluid-side
    if placement == "HGC":
        tags = {key: int(c.tags[c.idx[got[key]]]) for key in got}
        assert tags[(1.5, 3.5)] == -2 and tags[(3.5, 1.5)] == -2
        assert tags[(0.5, 3.5)] == 2 and tags[(2.5, 2.5)] == 2
    else:
        assert all(int(t) == 2 for t in c.tags[c.idx])


def test_fig3_cgc_face_adjacency():
    # (2.5, 0.5) touches fluid only diagonally and is drawn as a solid cell
    g, b, c = _fig3("CGC")
    ij = np.array([[int(2.5 + 6), int(0.5 + 6)]])
    assert int(c.tags[g.lin(ij)[0]]) == 1


def test_fig2_levels():
    rows = _read("fig2_levels.txt")
    g = O.Grid(2, [9, 7], [0, 0], [9, 7])
    tags = np.ones(g.N, dtype=np.int8)
    ghosts = []
    for r in rows:
        ij = np.array([[int(float(r[1])), int(float(r[2]))]])
        k = int(g.lin(ij)[0])
        if r[0] == "F":
            tags[k] = 0
        else:
            tags[k] = 2
            ghosts.append((k, int(r[3])))
    ghosts.sort()
    idx = np.array([k for k, _ in ghosts])
    ng = idx.size
    n = np.tile(np.array([-0.6, 0.8]), (ng, 1))
    e = np.tile(np.array([-1, 1]), (ng, 1))
    cls = Classification(g, None, "HGC", tags, idx, np.full(ng, 0.2), n, e, np.ones_like(e), [])
    lev = O.build_levels(cls)
    assert [int(v) for v in lev.level] == [lv for _, lv in ghosts]
    assert lev.n_levels == 3


def test_injected_cycle_detected():
    # two ghosts whose stencils point at each other
    g = O.Grid(2, [6, 6], [0, 0], [6, 6])
    tags = np.zeros(g.N, dtype=np.int8)
    a = int(g.lin(np.array([[2, 2]]))[0])
    b = int(g.lin(np.array([[3, 2]]))[0])
    tags[a] = tags[b] = 2
    idx = np.array([a, b])
    n = np.array([[0.8, 0.6], [-0.8, 0.6]])
    e = np.array([[1, 1], [-1, 1]])
    cls = Classification(g, None, "HGC", tags, idx, np.full(2, 0.2), n, e, np.ones_like(e), [])
    with pytest.raises(EBRError) as ei:
        O.build_levels(cls)
    assert ei.value.code == "ECYCLE"


def test_stencil_errors():
    g = O.Grid(2, [6, 6], [0, 0], [6, 6])
    tags = np.zeros(g.N, dtype=np.int8)
    a = int(g.lin(np.array([[0, 2]]))[0])
    tags[a] = 2
    cls = Classification(g, None, "HGC", tags, np.array([a]), np.full(1, 0.2),
                         np.array([[-0.8, 0.6]]), np.array([[-1, 1]]), np.ones((1, 2), int), [])
    with pytest.raises(EBRError) as ei:
        O.build_levels(cls)
    assert ei.value.code == "ESTENCIL_OOB"
    b = int(g.lin(np.array([[2, 2]]))[0])
    tags[:] = 0
    tags[b] = 2
    tags[int(g.lin(np.array([[3, 2]]))[0])] = 1
    cls = Classification(g, None, "HGC", tags, np.array([b]), np.full(1, 0.2),
                         np.array([[0.8, 0.6]]), np.array([[1, 1]]), np.ones((1, 2), int), [])
    with pytest.raises(EBRError) as ei:
        O.build_levels(cls)
    assert ei.value.code == "ESTENCIL_SOLID"


TINY = [
    (I.grid(2, [24, 20], [-1.0, -1.0], [1.0, 1.0]), I.ellipse(0.03, -0.02, 0.6, 0.35, 0.7)),
    (I.grid(2, [40, 20], [-1.0, -1.0], [3.0, 1.0]), I.airfoil(0.0, 0.0, 0.18, 1.0, 8.0)),
    (I.grid(2, [17, 17], [-1.0, -1.0], [1.0, 1.0]), I.circle(0.0, 0.0, 0.55)),
    (I.grid(3, [11, 12, 13], [-1.0, -1.0, -1.0], [1.0, 1.0, 1.0]), I.sphere(0.02, -0.01, 0.03, 0.6)),
]


@pytest.mark.parametrize("case", range(len(TINY)))
@pytest.mark.parametrize("placement", ["HGC", "CGC", "CGC_ES"])
def test_restricted_equals_brute_force(case, placement):
    # psi evaluated on every cell (the literal rule) gives the same tags as the
    # interface-cell restriction the oracle uses.
    gd, bd = TINY[case]
    g = O.Grid.from_dict(gd)
    b = O.Body.from_dict(bd)
    c1 = O.classify(g, b, placement)
    X = g.centre(g.unlin(np.arange(g.N)))
    # every cell except one sitting exactly at a circle's centre (normal undefined;
    # such a cell is deep inside and can never be a ghost)
    keep = np.arange(g.N)
    if b.kind in ("circle", "sphere"):
        keep = keep[np.linalg.norm(X - b.centre[: g.dim], axis=1) > 0]
    c2 = O.classify(g, b, placement, cells=keep)
    assert np.array_equal(c1.tags, c2.tags)
    assert np.array_equal(c1.idx, c2.idx)
    assert np.array_equal(c1.r, c2.r)


@pytest.mark.parametrize("case", range(len(TINY)))
@pytest.mark.parametrize("placement", ["HGC", "CGC", "CGC_ES"])
def test_levels_vs_networkx_longest_path(case, placement):
    gd, bd = TINY[case]
    c = O.classify(gd, bd, placement)
    lev = O.build_levels(c)
    G = nx.DiGraph()
    G.add_nodes_from(range(c.n_ghosts))
    for gh, deps in enumerate(lev.deps):
        for _, d in deps:
            G.add_edge(d, gh)
    assert nx.is_directed_acyclic_graph(G)
    # level = number of nodes on the longest path ending at the ghost
    want = {}
    for v in nx.topological_sort(G):
        preds = list(G.predecessors(v))
        want[v] = 1 + max((want[p] for p in preds), default=0)
    assert [int(lev.level[v]) for v in range(c.n_ghosts)] == [want[v] for v in range(c.n_ghosts)]
    # every ghost depends only on strictly lower levels
    for gh, deps in enumerate(lev.deps):
        for _, d in deps:
            assert lev.level[d] < lev.level[gh]
    # canonical order is (level, index)
    key = [(int(lev.level[g]), int(c.idx[g])) for g in lev.order]
    assert key == sorted(key)


def _alphas(c):
    d = c.grid.dim
    return np.stack([c.psi * c.n[:, a] / (c.r[:, a] * c.e[:, a] * c.grid.h[a]) for a in range(d)], axis=1)


def test_stability_invariants_cylinder_and_airfoil():
    # HGC: alpha_i <= 1/2 (from Eqs. delta_n and HGC_criterion); CGC: alpha_i < 1;
    # CGC_ES: |x1 - xs|_i / (r_i dx_i) <= 1/2 (Sec. 7); Eq. stencil_anisotropic
    # applied to HGC ghosts gives r = 1.
    for gd, bd in [(I.cylinder()["grid"], I.cylinder()["body"]),
                   (I.grid(2, [512, 256], [-1, -1], [3, 1]), I.airfoil(0, 0, 0.12, 1.0, 5.0))]:
        h = O.classify(gd, bd, "HGC")
        a = _alphas(h)
        assert a.max() <= 0.5 + 1e-12
        q = 2 * np.abs(h.psi[:, None] * h.n) / np.array(h.grid.h)[None, :]
        assert np.all(np.maximum(1, np.ceil(q)) == 1)
        cg = O.classify(gd, bd, "CGC")
        a = _alphas(cg)
        assert a.min() >= 0 and a.max() < 1
        es = O.classify(gd, bd, "CGC_ES")
        assert np.abs(_alphas(es)).max() <= 0.5 + 1e-12
        assert np.array_equal(es.idx, cg.idx)


def test_max_alpha_near_paper_cylinder_values():
    # Sec. 8.1 prints max alpha_x = 0.924 (CGC), 0.464 (HGC) for d = 1, dx = 0.015 d.
    # The body offset relative to the grid is not stated: loose check only.
    n = 400
    gd = I.grid(2, [n, n], [-3.0, -3.0], [3.0, 3.0])      # dx = 0.015
    bd = I.circle(0.0031, 0.0017, 0.5)
    ah = _alphas(O.classify(gd, bd, "HGC")).max()
    ac = _alphas(O.classify(gd, bd, "CGC")).max()
    assert 0.4 < ah <= 0.5
    assert 0.85 < ac < 1.0


def test_adjoint_cases_cover_both_stencil_reaches():
    """The GPU adjoint cases span both fluid-target paths of the library: HGC
    stencils reach one cell, the CGC_ES cases reach two (Sec. 7's r_i)."""
    import numpy as np
    from tests.test_gpu_adjoint import _case
    for kind in ("ellipse", "airfoil", "sphere"):
        w = _case(kind)
        assert int(np.max(O.classify(w["grid"], w["body"], "HGC").r)) == 1
        assert int(np.max(O.classify(w["grid"], w["body"], "CGC_ES").r)) == 2


@pytest.mark.parametrize("placement", ["HGC", "CGC", "CGC_ES"])
def test_bodies_missing_or_covering_the_grid_have_no_ghosts(placement):
    # degenerate sets of the GPU edge-case tests: no cell of another tag
    # shares a face, so no interface and no ghost; tags all 0 or all 1
    from tests.test_gpu_edge_cases import _empty_cases
    for case in _empty_cases():
        c = O.classify(case["grid"], case["body"], placement)
        lev = O.build_levels(c)
        assert c.n_ghosts == 0 and c.ties == [] and lev.order.size == 0
        assert np.unique(c.tags).size == 1 and c.tags[0] in (0, 1)
