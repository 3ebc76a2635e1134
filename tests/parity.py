"""Shared helpers of the GPU parity tests: run the CUDA path and the CPU
oracle on the same seeded inputs and compare.

Tolerances.  Every ghost value is a linear combination; expanding the level
recursion, T_G = |w_s b| + sum_k |w_k| (T_k for ghost members, |phi_k| for
fluid members) is the magnitude of all terms that make it up.  FP64 results
must agree to 1e-12 T_G (rounding and the 1e-13-level differences between two
independent closest-point evaluations both scale with the terms).  FP32 results
must agree to 1e-5 max|phi| (HGC and CGC_ES, whose weights are bounded by the
alpha <= 1/2 placement); CGC, whose weights grow like 1/(1 - alpha), may also
use the rounding bound 8 (K + 2) u32 T_G.

Independence.  Each side evaluates the boundary data at its own boundary
points: the GPU at the S and normals that ebr_ghost_info reports (as a user
of the library does), the oracle at the S and normals of its own closest-point
solution.  No input of the oracle comes from the CUDA path.  The GPU's psi, n
and S are compared with the oracle's per ghost (compare_structure):
|psi| and every component of S within GEOM_TOL of the smallest cell width,
every component of n within NORMAL_TOL.  Two independent closest-point
solutions (the GPU's float Newton + double Halley polish, the oracle's
long-double bisection / golden-section search) agree to a few 1e-13 of a
cell width, so 1e-11 leaves a margin of two orders of magnitude while a
wrong closest point (a wrong root, a dropped term) misses by many orders.
"""

import numpy as np
import torch

import oracle as O
from paper_2609_10165_b300 import inputs as I
from paper_2609_10165_b300.api import Reconstructor

U32 = 2.0 ** -24
GEOM_TOL = 1e-11      # psi and S: fraction of the smallest cell width
NORMAL_TOL = 1e-10    # unit normal, per component

# worst observed errors of the GPU path against the oracle, per quantity, as a
# fraction of its tolerance and in absolute terms (filled by the checks; read
# by tests that report them)
WORST = {}


def note_worst(key, ratio, value):
    r0, _ = WORST.get(key, (0.0, 0.0))
    if ratio >= r0:
        WORST[key] = (float(ratio), float(value))


class DeviceRun:
    def __init__(self, geoms, placement, mode="persistent", dtype=torch.float64, layers=1):
        """geoms: list of workload dicts (grid, body, fields, bc, roles, mu)."""
        self.geoms = geoms
        self.dtype = dtype
        self.layers = layers
        self.R = Reconstructor([g["grid"] for g in geoms], [g["body"] for g in geoms], placement, layers=layers)
        self.R.build_levels()
        self.R.sync_status()
        self.info = self.R.ghost_info()
        self.F = len(geoms[0]["fields"])
        self.mode = mode

    def field_arrays(self):
        """Per field: concatenated FP64 inputs of all geometries."""
        return [np.concatenate([g["fields"][f].on_grid(g["grid"]) for g in self.geoms]) for f in range(self.F)]

    def bc_arrays(self):
        """Boundary data at the GPU's own S and normals (the CUDA path's input)."""
        info = self.info
        out = []
        for f in range(self.F):
            vals = np.zeros(info["cell"].size)
            for b, g in enumerate(self.geoms):
                sel = info["geom"] == b
                d = g["grid"]["dim"]
                vals[sel] = I.bc_values(g["fields"][f], g["bc"][f], info["S"][sel, :d], info["normal"][sel, :d])
            out.append(vals)
        return out

    def fill(self, arrays, bcs):
        dev = self.R.device
        ft = [torch.tensor(a, dtype=self.dtype, device=dev) for a in arrays]
        bt = [torch.tensor(b, dtype=self.dtype, device=dev) for b in bcs]
        self.R.reconstruct(ft, self.geoms[0]["bc"], bt, mode=self.mode)
        self.R.sync_status()
        return ft, bt


def oracle_boundary(c, lev):
    """The oracle's own boundary points S = x_c + psi n and normals, canonical order."""
    X = c.grid.centre(c.grid.unlin(c.idx))
    S = X + c.psi[:, None] * c.n
    return S[lev.order], c.n[lev.order]


def oracle_bcs(g, c, lev, f32=False):
    """Boundary data of every field of workload g at the oracle's own S and
    normals, canonical order (rounded through float32 when f32)."""
    S, nn = oracle_boundary(c, lev)
    out = [I.bc_values(fld, k, S, nn) for fld, k in zip(g["fields"], g["bc"])]
    if f32:
        out = [b.astype(np.float32).astype(np.float64) for b in out]
    return out


def oracle_run(g, placement, arrays, f32=False, layers=1):
    """Oracle classification, levels and fill of one geometry, with the
    boundary data at the oracle's own S."""
    c = O.classify(g["grid"], g["body"], placement, layers=layers)
    lev = O.build_levels(c)
    bcs = oracle_bcs(g, c, lev, f32)
    out = O.fill(c, lev, arrays, g["bc"], bcs)
    return c, lev, bcs, out


def compare_geometry(psi, normal, S, c, lev, tag=""):
    """GPU psi [Ng], normal [Ng, 3], S [Ng, 3] (canonical order, one geometry)
    against the oracle's; returns the worst errors (psi/h, S/h, n)."""
    d = c.grid.dim
    h = min(c.grid.h)
    So, no = oracle_boundary(c, lev)
    po = c.psi[lev.order]
    ep = np.abs(psi - po) / h
    es = np.abs(S[:, :d] - So) / h
    en = np.abs(normal[:, :d] - no)
    worst = (float(ep.max(initial=0.0)), float(es.max(initial=0.0)), float(en.max(initial=0.0)))
    assert worst[0] <= GEOM_TOL, ("psi", tag, worst[0], int(np.argmax(ep)))
    assert worst[1] <= GEOM_TOL, ("S", tag, worst[1])
    assert worst[2] <= NORMAL_TOL, ("normal", tag, worst[2])
    if d == 2 and normal.shape[1] > 2:
        assert np.all(normal[:, 2] == 0) and np.all(S[:, 2] == 0)
    note_worst("psi/h", worst[0] / GEOM_TOL, worst[0])
    note_worst("S/h", worst[1] / GEOM_TOL, worst[1])
    note_worst("n", worst[2] / NORMAL_TOL, worst[2])
    return worst


def term_magnitude(c, lev, arrays, bcs, kinds):
    """T_G per field (canonical order)."""
    h = c.grid.h
    pos = lev.position()
    ng = c.n_ghosts
    T = []
    for fi, (arr, b) in enumerate(zip(arrays, bcs)):
        t = np.zeros(ng)
        for p in range(ng):
            g = int(lev.order[p])
            w, ws = O.ghost_weights(h, c.psi[g], c.n[g], c.e[g], c.r[g], kinds[fi], O.ghost_x2(c, g))
            acc = abs(ws * b[p])
            for k in range(w.size):
                if not lev.active[g, k]:
                    continue
                dg = [dd for kk, dd in lev.deps[g] if kk == k]
                if dg:
                    acc += abs(w[k]) * t[pos[dg[0]]]
                else:
                    acc += abs(w[k]) * abs(arr[lev.midx[g, k]])
            t[p] = acc
        T.append(t)
    return T


def compare_structure(run, geoms, placement):
    """Bit-exact tags, ghost cells, canonical order and levels, per geometry;
    psi, n and S against the oracle's own closest points."""
    tags = run.R.tags.cpu().numpy()
    info = run.info
    res = []
    for b, g in enumerate(geoms):
        c = O.classify(g["grid"], g["body"], placement, layers=getattr(run, "layers", 1))
        assert c.ties == [], c.ties[:5]
        lev = O.build_levels(c)
        o0, o1 = run.R.cell_offset[b], run.R.cell_offset[b + 1]
        assert np.array_equal(tags[o0:o1], c.tags), "tags differ in geometry %d: %d cells" % (
            b, int(np.sum(tags[o0:o1] != c.tags)))
        sel = info["geom"] == b
        assert np.array_equal(info["cell"][sel], c.idx[lev.order]), "ghost order differs in geometry %d" % b
        assert np.array_equal(info["level"][sel], lev.level[lev.order]), "levels differ in geometry %d" % b
        gt = np.where(c.tags[c.idx[lev.order]] == -2, -2, 2)
        assert np.array_equal(info["tag"][sel], gt)
        d = g["grid"]["dim"]
        assert np.array_equal(info["r"][sel][:, :d], c.r[lev.order])
        compare_geometry(info["psi"][sel], info["normal"][sel], info["S"][sel], c, lev, tag=b)
        res.append((c, lev))
    return res
