"""Pins of the oracle's tiled fill with per-level exchange (Sec. 3.2, the
distributed-memory paragraph): a hand-derived exchange on the Fig. 2 example,
decomposition invariance of the values (the tiles fill with the closed forms
of Secs. 4-5 and must give the global fill bit for bit, for any tile shape),
completeness of the send lists against a brute-force reading of the
stencils, and the comparison with a conventional halo exchange."""

import os

import numpy as np
import pytest

import oracle as O
from oracle.classify import Classification
from oracle.tiles import halo_exchange_volume, tile_ids, tile_plan, tiled_fill
from paper_2609_10165_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _fig2():
    rows = _read("fig2_levels.txt")
    g = O.Grid(2, [9, 7], [0, 0], [9, 7])
    tags = np.ones(g.N, dtype=np.int8)
    ghosts = []
    for r in rows:
        k = int(g.lin(np.array([[int(float(r[1])), int(float(r[2]))]]))[0])
        if r[0] == "F":
            tags[k] = 0
        else:
            tags[k] = 2
            ghosts.append(k)
    idx = np.array(sorted(ghosts))
    ng = idx.size
    n = np.tile(np.array([-0.6, 0.8]), (ng, 1))
    e = np.tile(np.array([-1, 1]), (ng, 1))
    cls = Classification(g, None, "HGC", tags, idx, np.full(ng, 0.2), n, e, np.ones_like(e), [])
    return cls, O.build_levels(cls)


def test_fig2_exchange_by_hand():
    cls, lev = _fig2()
    rows = _read("fig2_tiles.txt")
    tile = [int(v) for v in rows[0][1:]]
    want = [(int(r[1]), int(float(r[2])), int(float(r[3])), int(r[4])) for r in rows if r[0] == "SEND"]
    exchanged = int([r for r in rows if r[0] == "EXCHANGED"][0][1])
    halo = int([r for r in rows if r[0] == "HALO"][0][1])
    plan = tile_plan(cls, lev, tile)
    got = []
    for lv, qs in enumerate(plan.sends, start=1):
        for q in qs:
            i, j = cls.grid.unlin([int(cls.idx[lev.order[q]])])[0]
            for t in plan.receivers[q]:
                got.append((lv, int(i), int(j), int(t)))
    assert got == want
    assert plan.values_exchanged() == exchanged
    assert halo_exchange_volume(cls, lev, tile) == halo
    # the tiled fill of arbitrary values equals the global fill
    rng = np.random.default_rng(3)
    arr = [rng.normal(size=cls.grid.N)]
    bc = [rng.normal(size=cls.n_ghosts)]
    out, _ = tiled_fill(cls, lev, arr, [O.DIRICHLET], bc, tile)
    ref = O.fill(cls, lev, arr, [O.DIRICHLET], bc)
    assert np.array_equal(out[0], ref[0])


CASES = [
    (I.grid(2, [40, 36], [-1.0, -1.0], [1.0, 1.0]), I.ellipse(0.03, -0.02, 0.6, 0.35, 0.7)),
    (I.grid(2, [131, 67], [-1.0, -1.0], [3.0, 1.0]), I.airfoil(0.0, 0.0, 0.12, 1.0, 5.0)),
    (I.grid(3, [21, 18, 19], [-1.0, -1.0, -1.0], [1.0, 1.0, 1.0]), I.sphere(0.02, -0.01, 0.03, 0.6)),
]


def _brute_force_remote(cls, lev, tile):
    """(canonical position of h, tile of g) for every stencil member h of a
    ghost g that is itself a ghost of another tile, read from the stencil
    offsets, the multipliers and the normals directly."""
    g_ = cls.grid
    d = g_.dim
    pos = lev.position()
    ghost = {int(c): i for i, c in enumerate(cls.idx)}
    tl = tile_ids(g_, cls.idx, tile)
    out = set()
    for gi in range(cls.n_ghosts):
        ijk = g_.unlin([int(cls.idx[gi])])[0]
        for off in O.stencil_offsets(d):
            if any(off[a] and cls.n[gi, a] == 0.0 for a in range(d)):
                continue                      # a zero weight: no dependency (Sec. 3.2)
            m = [int(ijk[a] + off[a] * cls.r[gi, a] * cls.e[gi, a]) for a in range(d)]
            c = int(g_.lin(np.array([m]))[0])
            if c in ghost and tl[ghost[c]] != tl[gi]:
                out.add((int(pos[ghost[c]]), int(tl[gi])))
    return out


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("placement", ["HGC", "CGC_ES"])
def test_tiled_fill_is_decomposition_invariant(case, placement):
    gd, bd = CASES[case]
    d = gd["dim"]
    c = O.classify(gd, bd, placement)
    lev = O.build_levels(c)
    rng = np.random.default_rng(40 + case)
    kinds = [O.DIRICHLET, O.NEUMANN]
    arr = [rng.normal(size=c.grid.N) for _ in kinds]
    bc = [rng.normal(size=c.n_ghosts) for _ in kinds]
    ref = O.fill(c, lev, arr, kinds, bc)
    tiles = [[2] * d, [5] * d, [8] * d, [3, 7, 4][:d], list(c.grid.n)]
    for tile in tiles:
        out, plan = tiled_fill(c, lev, arr, kinds, bc, tile)
        for f in range(len(kinds)):
            assert np.array_equal(out[f], ref[f]), (tile, f)
        # the send lists are exactly the remote dependencies
        pairs = {(q, t) for q, ts in plan.receivers.items() for t in ts}
        assert pairs == _brute_force_remote(c, lev, tile), tile
        for lv, qs in enumerate(plan.sends, start=1):
            assert all(int(lev.level[lev.order[q]]) == lv for q in qs)
        if tile == list(c.grid.n):
            assert plan.values_exchanged() == 0
        else:
            assert plan.values_exchanged() <= halo_exchange_volume(c, lev, tile), tile


def test_tiled_fill_detects_a_missing_exchange(monkeypatch):
    # a plan whose send list drops a value makes a tile read a ghost it never
    # received: the tiled fill refuses (the simulation checks every read)
    import oracle.tiles as T
    cls, lev = _fig2()
    real = T.tile_plan

    def dropped(cls_, lev_, tile_):
        p = real(cls_, lev_, tile_)
        p.sends = [[] for _ in p.sends]
        return p

    monkeypatch.setattr(T, "tile_plan", dropped)
    rng = np.random.default_rng(4)
    with pytest.raises(AssertionError):
        T.tiled_fill(cls, lev, [rng.normal(size=cls.grid.N)], [O.DIRICHLET],
                     [rng.normal(size=cls.n_ghosts)], [3, 7])
