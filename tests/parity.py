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
"""

import numpy as np
import torch

import oracle as O
from paper_2609_10165_b300 import inputs as I
from paper_2609_10165_b300.api import Reconstructor

U32 = 2.0 ** -24


class DeviceRun:
    def __init__(self, geoms, placement, mode="persistent", dtype=torch.float64):
        """geoms: list of workload dicts (grid, body, fields, bc, roles, mu)."""
        self.geoms = geoms
        self.dtype = dtype
        self.R = Reconstructor([g["grid"] for g in geoms], [g["body"] for g in geoms], placement)
        self.R.build_levels()
        self.R.sync_status()
        self.info = self.R.ghost_info()
        self.F = len(geoms[0]["fields"])
        self.mode = mode

    def field_arrays(self):
        """Per field: concatenated FP64 inputs of all geometries."""
        return [np.concatenate([g["fields"][f].on_grid(g["grid"]) for g in self.geoms]) for f in range(self.F)]

    def bc_arrays(self):
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


def oracle_run(g, placement, arrays, bcs_from_oracle=True):
    """Oracle classification, levels and fill of one geometry."""
    c = O.classify(g["grid"], g["body"], placement)
    lev = O.build_levels(c)
    d = g["grid"]["dim"]
    X = c.grid.centre(c.grid.unlin(c.idx))
    S = (X + c.psi[:, None] * c.n)[lev.order]
    nn = c.n[lev.order]
    bcs = [I.bc_values(fld, k, S, nn) for fld, k in zip(g["fields"], g["bc"])]
    out = O.fill(c, lev, arrays, g["bc"], bcs)
    return c, lev, bcs, out


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
            w, ws = O.ghost_weights(h, c.psi[g], c.n[g], c.e[g], c.r[g], kinds[fi])
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
    """Bit-exact tags, ghost cells, canonical order and levels, per geometry."""
    tags = run.R.tags.cpu().numpy()
    info = run.info
    res = []
    for b, g in enumerate(geoms):
        c = O.classify(g["grid"], g["body"], placement)
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
        res.append((c, lev))
    return res
