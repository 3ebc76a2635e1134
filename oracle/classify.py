"""Cell classification and ghost-cell placement (oracle; test infrastructure).

Sec. 3.1.  Cells are fluid (tag 0) or solid (tag 1) by the side of their
centre (psi >= 0 is solid).  Ghost cells are tagged +2 (centre in the solid)
or -2 (centre in the fluid).

* CGC  (Sec. 3.1, Fig. 1(a)): a solid cell with at least one fluid cell among
  its face neighbours (+-x, +-y[, +-z]) is a ghost (+2).  Face adjacency, not
  diagonal: Fig. 3(b) draws (0.5,2.5) and (2.5,0.5), which touch the fluid
  only diagonally, as plain solid cells.
* HGC  (Sec. 3.1, Eqs. delta_n, HGC_criterion): a solid cell with
  psi <= dn/2 becomes +2 and a fluid cell with -psi < dn/2 becomes -2, where
  dn = [(n_x/dx)^2 + (n_y/dy)^2 + (n_z/dz)^2]^(-1/2) uses the normal at S and the
  ghost's own cell widths.  Then the excess candidates are reclassified:
    pass A: a -2 cell with no face neighbour tagged 1 becomes fluid (0);
    pass B: a +2 cell with no face neighbour tagged 0 (tags after pass A)
            becomes solid (1).
  Each pass reads the tags as they were when the pass began.  "Solid cell"
  and "fluid cell" in the reclassification are read as the tags 1 and 0; the
  candidates (+-2) are neither.  Pass A before pass B is the reading taken
  (the paper lists both without an order); it reproduces Fig. 3(c).
* CGC_ES (Sec. 7, Eq. stencil_anisotropic): the CGC ghost set with the stencil
  multipliers r_i = max(1, ceil(2 |n_i psi| / dx_i)); CGC and HGC use r_i = 1.
* Second ghost layer (Sec. 7, "Additional ghost-cell layers", layers=2): after
  the first layer is placed (and, for HGC, reclassified), every remaining
  solid cell (tag 1) with psi <= 1.5 dn joins the ghost set (+2), and every
  ghost takes the multipliers of Eq. stencil_anisotropic (which leave HGC's
  first layer at r = 1, since there |n_i psi| / dx_i <= psi / dn <= 1/2).
  Readings: the layer is added after the first layer's reclassification (the
  passes act on the first layer only), dn is that of Eq. delta_n with the
  cell's own normal and widths, and the rule is offered with HGC and CGC_ES.
  A candidate at the exact centre of a circle or sphere (depth R, normal
  undefined) stays solid when R > 1.5 max_a h_a, which no dn admits; a body
  smaller than that has no defined second layer (error EINVAL).
  Candidates are the solid cells with a fluid cell within `layer_reach` cells
  along every axis (a box); the reach bounds the index distance from a solid
  cell with psi <= 1.5 dn to a fluid cell (see layer_reach).

Only cells with a face neighbour on the other side of the boundary can end as
ghosts: a fluid cell without a solid neighbour has no neighbour tagged 1 and
is reset by pass A; a solid cell without a fluid neighbour has no neighbour
tagged 0 after pass A and is reset by pass B; CGC needs a fluid neighbour by
definition.  So psi, S and n are evaluated on those "interface" cells only.
(The brute-force test evaluates every cell and finds the same tags.)

Stencil (Secs. 4-5): e_i = sgn(n_i) with e_i = +1 where n_i = 0 (Appendix A),
and the stencil members are G + (d_x r_x e_x dx, d_y r_y e_y dy[, d_z r_z e_z dz])
for the offsets d in the paper's order P_1..P_3 (2D) or P_1..P_7 (3D).
"""

import numpy as np

from .geometry import Grid, Body, inside, closest_point

HGC, CGC, CGC_ES = "HGC", "CGC", "CGC_ES"

# error codes shared in meaning (not in code) with the library's status values
E_STENCIL_OOB = "ESTENCIL_OOB"
E_STENCIL_SOLID = "ESTENCIL_SOLID"
E_CYCLE = "ECYCLE"


class EBRError(Exception):
    def __init__(self, code, msg=""):
        super().__init__("%s: %s" % (code, msg))
        self.code = code


def stencil_offsets(dim):
    """Offsets of P_1.. in units of (r_i e_i dx_i): 2D P1=(1,0), P2=(0,1),
    P3=(1,1) (Sec. 4); 3D P1..P7 = (1,0,0),(0,1,0),(0,0,1),(1,1,0),(0,1,1),
    (1,0,1),(1,1,1) (Sec. 5)."""
    if dim == 2:
        return [(1, 0), (0, 1), (1, 1)]
    return [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1), (1, 1, 1)]


class Classification:
    """Tags for every cell and the ghost records (sorted by linear index)."""

    def __init__(self, grid, body, placement, tags, idx, psi, n, e, r, ties, x2=None, hw=None):
        self.x2 = x2                # float64 [N_g, d]: x_2 - x_1 per ghost (stretched grids), else None
        self.hw = hw                # float64 [N_g, d]: the ghost cell's widths (stretched grids), else None
        self.grid = grid
        self.body = body
        self.placement = placement
        self.tags = tags            # int8 [N]
        self.idx = idx              # int64 [N_g], ascending
        self.psi = psi              # float64 [N_g]
        self.n = n                  # float64 [N_g, d]
        self.e = e                  # int64 [N_g, d]
        self.r = r                  # int64 [N_g, d]
        self.ties = ties            # list of (cell index, reason, margin)

    @property
    def n_ghosts(self):
        return int(self.idx.size)


def _solid_all(grid, body):
    """Inside predicate for every cell centre, slab by slab to bound memory."""
    solid = np.zeros(grid.N, dtype=bool)
    nx = grid.n[0]
    plane = grid.N // grid.n[-1]
    for s in range(grid.n[-1]):
        ids = np.arange(s * plane, (s + 1) * plane, dtype=np.int64)
        X = grid.centre(grid.unlin(ids))
        solid[ids] = inside(body, X)
    del nx
    return solid


def _face_neighbour_any(grid, flag):
    """For each cell: does any in-grid face neighbour have ``flag`` set?"""
    f = flag.reshape(grid.n[::-1])          # [(nz,) ny, nx]
    out = np.zeros_like(f)
    nd = grid.dim
    for a in range(nd):
        ax = nd - 1 - a                      # numpy axis of grid axis a
        sl_lo = [slice(None)] * nd
        sl_hi = [slice(None)] * nd
        sl_lo[ax] = slice(0, -1)
        sl_hi[ax] = slice(1, None)
        out[tuple(sl_lo)] |= f[tuple(sl_hi)]     # neighbour at +1
        out[tuple(sl_hi)] |= f[tuple(sl_lo)]     # neighbour at -1
    return out.reshape(-1)


def delta_n(grid, n, widths=None):
    """Eq. delta_n: normal cell thickness for unit normals n [M, d], with the
    cells' own widths [M, d] (a uniform grid's spacing when widths is None)."""
    s = np.zeros(n.shape[0])
    for a in range(grid.dim):
        q = n[:, a] / (grid.h[a] if widths is None else widths[:, a])
        s = s + q * q
    return 1.0 / np.sqrt(s)


def ghost_x2(cls, g):
    """x_2 - x_1 of ghost g (index order) on a stretched grid, else None (the
    closed forms then take r e h)."""
    return None if cls.x2 is None else cls.x2[g]


def layer_reach(grid):
    """Box reach (cells per axis) that holds a fluid cell for every solid cell
    with psi <= 1.5 dn (widths of a stretched grid bounded by hmax, counted in
    units of the smallest width).  For such a cell G with boundary point S and unit
    normal n, the point X = G + (psi + D/2 + eps) n, D = sqrt(sum_a h_a^2),
    lies at distance D/2 + eps from the convex body (its closest point is S),
    so the cell containing X has its centre outside: a fluid cell.  Along axis
    a that centre is at most psi + D/2 + h_a/2 from G, and psi <= 1.5 dn <=
    1.5 max_a h_a, hence at most ceil((1.5 max h + D/2) / h_a + 1/2) cells."""
    h = grid.h
    if getattr(grid, "stretched", False):
        # stretched: the largest widths in the distances, the smallest width
        # of the axis as the unit (the containing cell's half width included)
        hx = grid.hmax
        D = float(np.sqrt(sum(v * v for v in hx)))
        hm = max(hx)
        return [int(np.ceil((1.5 * hm + 0.5 * D + 0.5 * hx[a]) / h[a])) for a in range(grid.dim)]
    D = float(np.sqrt(sum(v * v for v in h)))
    hm = max(h)
    return [int(np.ceil((1.5 * hm + 0.5 * D) / h[a] + 0.5)) for a in range(grid.dim)]


def _box_neighbour_any(grid, flag, reach):
    """For each cell: does any in-grid cell within `reach[a]` cells along every
    axis a (a box) have ``flag`` set?"""
    f = flag.reshape(grid.n[::-1])
    nd = grid.dim
    out = f.copy()
    for a in range(nd):
        ax = nd - 1 - a
        cur = out.copy()
        for s_ in range(1, reach[a] + 1):
            sl_lo = [slice(None)] * nd
            sl_hi = [slice(None)] * nd
            sl_lo[ax] = slice(0, -s_)
            sl_hi[ax] = slice(s_, None)
            cur[tuple(sl_lo)] |= out[tuple(sl_hi)]
            cur[tuple(sl_hi)] |= out[tuple(sl_lo)]
        out = cur
    return out.reshape(-1)


def classify(grid, body, placement=HGC, tie_rel=1e-9, cells=None, layers=1, layer_cells=None):
    """Tags and ghost records.  ``cells`` (optional, for the brute-force test)
    evaluates psi on the given cell set instead of the interface cells;
    ``layer_cells`` likewise replaces the second layer's candidates."""
    if isinstance(grid, dict):
        grid = Grid.from_dict(grid)
    if isinstance(body, dict):
        body = Body.from_dict(body)
    d = grid.dim
    solid = _solid_all(grid, body)
    tags = solid.astype(np.int8)
    iface = (solid & _face_neighbour_any(grid, ~solid)) | (~solid & _face_neighbour_any(grid, solid))
    if cells is None:
        cells = np.nonzero(iface)[0]
    cells = np.asarray(cells, dtype=np.int64)
    ijk = grid.unlin(cells)
    X = grid.centre(ijk)
    psi_c, n_c = closest_point(body, X)
    sol_c = solid[cells]
    if not np.array_equal(psi_c >= 0, sol_c):
        raise AssertionError("inside predicate and psi sign disagree")
    tol = tie_rel * min(grid.h)
    ties = []
    for k in np.nonzero(np.abs(psi_c) < tol)[0]:
        ties.append((int(cells[k]), "psi~0", float(psi_c[k])))
    for a in range(d):
        for k in np.nonzero((n_c[:, a] != 0) & (np.abs(n_c[:, a]) < 1e-12))[0]:
            ties.append((int(cells[k]), "n%d~0" % a, float(n_c[k, a])))

    if placement in (CGC, CGC_ES):
        ghost_c = sol_c & _face_neighbour_any(grid, ~solid)[cells]
        tags[cells[ghost_c]] = 2
    elif placement == HGC:
        dn = delta_n(grid, n_c, grid.widths(ijk) if grid.stretched else None)
        cand_s = sol_c & (psi_c <= dn / 2)
        cand_f = (~sol_c) & (-psi_c < dn / 2)
        for k in np.nonzero(np.abs(np.abs(psi_c) - dn / 2) < tol)[0]:
            ties.append((int(cells[k]), "psi~dn/2", float(np.abs(psi_c[k]) - dn[k] / 2)))
        tags[cells[cand_s]] = 2
        tags[cells[cand_f]] = -2
        # pass A: -2 without a face neighbour tagged 1 -> 0 (snapshot)
        has1 = _face_neighbour_any(grid, tags == 1)
        drop = (tags == -2) & ~has1
        tags[drop] = 0
        # pass B: +2 without a face neighbour tagged 0 -> 1 (snapshot after A)
        has0 = _face_neighbour_any(grid, tags == 0)
        drop = (tags == 2) & ~has0
        tags[drop] = 1
    else:
        raise ValueError("unknown placement %r" % placement)

    if layers == 2:
        if placement not in (HGC, CGC_ES):
            raise ValueError("a second ghost layer goes with HGC or CGC_ES")
        # second layer: remaining solid cells with psi <= 1.5 dn
        if layer_cells is None:
            near = _box_neighbour_any(grid, ~solid, layer_reach(grid))
            layer_cells = np.nonzero((tags == 1) & near)[0]
        layer_cells = np.setdiff1d(np.asarray(layer_cells, dtype=np.int64), cells)
        layer_cells = layer_cells[tags[layer_cells] == 1]
        if body.kind in ("circle", "sphere"):
            # a candidate at the body's centre has depth R and no normal: it
            # stays solid when R > 1.5 max_a h_a (no dn <= max_a h_a admits
            # it); otherwise the second layer is undefined there
            Xl = grid.centre(grid.unlin(layer_cells))
            at_c = np.all(Xl == body.centre[:d][None, :], axis=1)
            if np.any(at_c):
                if not body.radii[0] > 1.5 * max(grid.hmax):
                    raise EBRError("EINVAL", "second-layer candidate at the centre of a small body")
                layer_cells = layer_cells[~at_c]
        psi_l, n_l = closest_point(body, grid.centre(grid.unlin(layer_cells)))
        if not np.all(psi_l >= 0):
            raise AssertionError("second-layer candidate outside the body")
        # the first layer's interface cells left solid are candidates too
        back = (tags[cells] == 1)
        cand = np.concatenate([cells[back], layer_cells])
        psi_k = np.concatenate([psi_c[back], psi_l])
        n_k = np.concatenate([n_c[back], n_l])
        dn = delta_n(grid, n_k, grid.widths(grid.unlin(cand)) if grid.stretched else None)
        add = psi_k <= 1.5 * dn
        for k in np.nonzero(np.abs(psi_k - 1.5 * dn) < tol)[0]:
            ties.append((int(cand[k]), "psi~1.5dn", float(psi_k[k] - 1.5 * dn[k])))
        tags[cand[add]] = 2
        cells = np.concatenate([cells, layer_cells])
        psi_c = np.concatenate([psi_c, psi_l])
        n_c = np.concatenate([n_c, n_l])
    elif layers != 1:
        raise ValueError("layers must be 1 or 2")

    gmask = np.abs(tags[cells]) == 2
    g_cells = cells[gmask]
    order = np.argsort(g_cells)
    g_cells = g_cells[order]
    psi = psi_c[gmask][order]
    n = n_c[gmask][order]
    e = np.where(n >= 0, 1, -1).astype(np.int64)          # sgn(n), 0 -> +1
    r = np.ones_like(e)
    hw = grid.widths(grid.unlin(g_cells)) if grid.stretched else None
    if placement == CGC_ES or layers == 2:
        for a in range(d):
            q = 2.0 * np.abs(psi * n[:, a]) / (grid.h[a] if hw is None else hw[:, a])
            r[:, a] = np.maximum(1, np.ceil(q)).astype(np.int64)
            near = (q > 1.0 - 1e-9) & (np.abs(q - np.round(q)) < 1e-9)
            for k in np.nonzero(near)[0]:
                ties.append((int(g_cells[k]), "r%d ceil" % a, float(q[k])))
    x2 = None
    if grid.stretched:
        # x_2 - x_1: centre of the cell r_i e_i cells away minus the ghost's
        # (indices clipped into the grid; a stencil that leaves it is an error
        # raised by check_stencils)
        gijk = grid.unlin(g_cells)
        x2 = np.zeros((g_cells.size, d))
        for a in range(d):
            far = np.clip(gijk[:, a] + r[:, a] * e[:, a], 0, grid.n[a] - 1)
            x2[:, a] = grid.cen[a][far] - grid.cen[a][gijk[:, a]]
    return Classification(grid, body, placement, tags, g_cells, psi, n, e, r, ties, x2=x2, hw=hw)


def stencil_members(cls):
    """Member cells of every ghost: (ijk [N_g, K, d], in_grid [N_g, K],
    active [N_g, K]).  A member is active (structurally non-zero weight) when
    n_i != 0 on every axis along which it is offset (Sec. 3.2: n_i = 0 removes
    the dependence on neighbours in direction i)."""
    g = cls.grid
    d = g.dim
    offs = np.array(stencil_offsets(d), dtype=np.int64)          # [K, d]
    gijk = g.unlin(cls.idx)                                        # [N_g, d]
    step = cls.r * cls.e                                           # [N_g, d]
    mijk = gijk[:, None, :] + offs[None, :, :] * step[:, None, :]
    ing = np.ones(mijk.shape[:2], dtype=bool)
    for a in range(d):
        ing &= (mijk[:, :, a] >= 0) & (mijk[:, :, a] < g.n[a])
    active = np.ones(mijk.shape[:2], dtype=bool)
    for a in range(d):
        active &= ~((offs[None, :, a] == 1) & (cls.n[:, None, a] == 0.0))
    return mijk, ing, active


def check_stencils(cls):
    """Every stencil member must lie in the grid and must not be a plain solid
    cell (tag 1): its value would be undefined.  Raises EBRError."""
    mijk, ing, _ = stencil_members(cls)
    if not np.all(ing):
        g = int(np.nonzero(~ing.all(axis=1))[0][0])
        raise EBRError(E_STENCIL_OOB, "ghost %d stencil leaves the grid" % int(cls.idx[g]))
    midx = cls.grid.lin(mijk.reshape(-1, cls.grid.dim)).reshape(ing.shape)
    bad = cls.tags[midx] == 1
    if np.any(bad):
        g = int(np.nonzero(bad.any(axis=1))[0][0])
        raise EBRError(E_STENCIL_SOLID, "ghost %d stencil contains a solid cell" % int(cls.idx[g]))
    return midx
