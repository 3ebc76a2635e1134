"""Tiled (domain-decomposed) level-by-level fill with per-level exchange
(oracle; test infrastructure).

Sec. 3.2, last paragraph: when the grid is split into subdomains, a ghost's
stencil may reach ghosts of a neighbouring subdomain.  The level ordering
does not remove that communication but confines it to the level just filled:
after L_k is reconstructed, only the ghosts of L_k that appear in stencils of
other subdomains are exchanged, before L_{k+1}.

Here the subdomains are rectangular tiles of the Cartesian grid (tile sizes
per axis, in cells; tile t of cell (i, j, k) = (i // T_x) + n_tx ((j // T_y)
+ n_ty (k // T_z))).  A ghost belongs to the tile of its cell.

* ``tile_plan`` -- the tile of every ghost and, per level k, the ghosts of L_k
  that a ghost of another tile depends on (the values sent after level k),
  with the receiving tiles.
* ``tiled_fill`` -- the fill run tile by tile: each tile keeps the values it
  owns plus the values it has received, fills its ghosts of L_k from those
  only (a stencil value that is neither owned nor received is an error), then
  sends its ghosts of the send list of level k.  It must give the values of
  ``reconstruct.fill`` (same closed forms, same inputs).
* ``halo_exchange_volume`` -- the comparison the paper draws: a conventional
  iterative reconstruction exchanges the usual halo after every sweep.  Counted
  here as the ghost values within the stencil reach of a tile face (each sent
  to the tile across that face), once per sweep, with as many sweeps as
  levels (the minimum for information to cross a chain of depth n).
"""

import numpy as np

from .classify import ghost_x2
from .reconstruct import ghost_weights


def tile_ids(grid, cells, tile):
    """Tile of each linear cell index (tile sizes per axis in cells)."""
    ijk = grid.unlin(cells)
    d = grid.dim
    nt = [(grid.n[a] + tile[a] - 1) // tile[a] for a in range(d)]
    t = ijk[:, d - 1] // tile[d - 1]
    for a in range(d - 2, -1, -1):
        t = t * nt[a] + ijk[:, a] // tile[a]
    return t.astype(np.int64)


class TilePlan:
    def __init__(self, tile_of, sends, receivers):
        self.tile_of = tile_of      # int64 [N_g], canonical order
        self.sends = sends          # list per level k (1-based, index k - 1): sorted canonical positions
        self.receivers = receivers  # dict canonical position -> sorted list of receiving tiles

    def sent_per_level(self):
        return [len(s) for s in self.sends]

    def values_exchanged(self):
        """(ghost, receiving tile) pairs over all levels."""
        return sum(len(v) for v in self.receivers.values())


def tile_plan(cls, lev, tile):
    """Tile of every ghost and the per-level send lists (canonical positions)."""
    pos = lev.position()
    ng = cls.n_ghosts
    tl = tile_ids(cls.grid, cls.idx, tile)              # per ghost, index order
    tile_of = np.empty(ng, dtype=np.int64)
    tile_of[pos] = tl
    receivers = {}
    for g in range(ng):
        for _, h in lev.deps[g]:
            if tl[h] != tl[g]:
                receivers.setdefault(int(pos[h]), set()).add(int(tl[g]))
    sends = [[] for _ in range(lev.n_levels)]
    for q in sorted(receivers):
        g = int(lev.order[q])
        sends[int(lev.level[g]) - 1].append(q)
    return TilePlan(tile_of, sends, {q: sorted(v) for q, v in receivers.items()})


def tiled_fill(cls, lev, arrays, bc_kinds, bcs, tile):
    """Level-by-level fill run by tiles that exchange their sent ghosts after
    every level.  arrays: field values [F][N] (copied); bcs: boundary data
    [F][N_g] in canonical order.  Returns (filled arrays, plan)."""
    plan = tile_plan(cls, lev, tile)
    h = cls.grid.h
    pos = lev.position()
    K = lev.midx.shape[1]
    tl = tile_ids(cls.grid, cls.idx, tile)
    ghost_of_cell = {int(c): g for g, c in enumerate(cls.idx)}
    out = [np.array(a, dtype=np.float64, copy=True) for a in arrays]
    # per tile, the ghost values it holds (owned or received): (field, cell) -> value
    held = {}
    for lv in range(1, lev.n_levels + 1):
        filled = []
        for q in range(int(lev.level_ptr[lv - 1]), int(lev.level_ptr[lv])):
            g = int(lev.order[q])
            t = int(tl[g])
            mine = held.setdefault(t, {})
            for f, (arr, kind, b) in enumerate(zip(arrays, bc_kinds, bcs)):
                w, ws = ghost_weights(h, cls.psi[g], cls.n[g], cls.e[g], cls.r[g], kind, ghost_x2(cls, g))
                v = ws * float(b[q])
                for k in range(K):
                    if not lev.active[g, k]:
                        continue
                    m = int(lev.midx[g, k])
                    if m in ghost_of_cell:
                        if (f, m) not in mine:
                            raise AssertionError("tile %d reads ghost cell %d before owning or receiving it"
                                                 % (t, m))
                        v += w[k] * mine[(f, m)]
                    else:
                        v += w[k] * float(arr[m])
                mine[(f, int(cls.idx[g]))] = v
                out[f][cls.idx[g]] = v
            filled.append(q)
        # exchange: the sent ghosts of this level go to their receiving tiles
        for q in plan.sends[lv - 1]:
            g = int(lev.order[q])
            c = int(cls.idx[g])
            src = held[int(tl[g])]
            for t in plan.receivers[q]:
                dst = held.setdefault(t, {})
                for f in range(len(arrays)):
                    dst[(f, c)] = src[(f, c)]
    return out, plan


def halo_exchange_volume(cls, lev, tile, reach=None):
    """Ghost values a conventional iterative reconstruction would exchange:
    per sweep, every ghost within `reach` cells (default: the largest stencil
    multiplier) of a face of its tile, once per neighbouring tile across such a
    face; n_levels sweeps."""
    g = cls.grid
    d = g.dim
    R = int(cls.r.max()) if reach is None and cls.n_ghosts else (reach or 1)
    ijk = g.unlin(cls.idx)
    per_sweep = 0
    for a in range(d):
        lo_face = (ijk[:, a] % tile[a]) < R
        hi_face = (tile[a] - 1 - ijk[:, a] % tile[a]) < R
        has_lo = ijk[:, a] - (ijk[:, a] % tile[a]) > 0
        has_hi = ijk[:, a] - (ijk[:, a] % tile[a]) + tile[a] < g.n[a]
        per_sweep += int(np.sum(lo_face & has_lo)) + int(np.sum(hi_face & has_hi))
    return per_sweep * lev.n_levels
