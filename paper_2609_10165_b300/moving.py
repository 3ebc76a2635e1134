"""Moving bodies: a time-stepping consumer of the library (Sec. 7).

When a body moves it covers and exposes cells, so every step classifies the
cells anew, places the ghost cells, rebuilds the dependency levels and only
then fills the ghost values (Sec. 7 names moving boundaries among the uses of
additional ghost layers).  This module drives that loop for prescribed rigid
motions: per step it moves the bodies (``ebr_move``, which reuses the
context's device buffers once their capacity has settled), rebuilds the
levels, evaluates the boundary data at the new boundary points, restores the
field values of the cells that were ghosts at the previous step (a solver
would supply them for the freshly exposed cells), fills the ghost cells and
evaluates the forces (and, when asked, the adjoint).

Every step runs in the library's kernels; the host evaluates the prescribed
motion and the manufactured boundary data only.
"""

import math

import numpy as np
import torch

from .api import Reconstructor


def _rot2(theta):
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


class RigidMotion:
    """Translation with constant velocity and rotation at a constant rate
    about the body's reference point (its centre; the leading edge of an
    airfoil), in the x-y plane: body(t) = shift by u t, turn by omega t."""

    def __init__(self, body, velocity=(0.0, 0.0, 0.0), omega=0.0):
        self.body = dict(body)
        self.velocity = np.asarray(velocity, dtype=np.float64)
        self.omega = float(omega)

    def at(self, t):
        b = dict(self.body)
        b["centre"] = [float(c + v * t) for c, v in zip(self.body["centre"], self.velocity)]
        R0 = np.asarray(self.body["rot"], dtype=np.float64).reshape(3, 3)
        b["rot"] = [float(v) for v in (_rot2(self.omega * t) @ R0).reshape(-1)]
        return b


class MovingStepper:
    """A geometry set whose bodies move: per step, move + levels + fill +
    forces (+ adjoint).

    grids: list of grid dicts; motions: one RigidMotion per grid; fields:
    per field one manufactured field object (value, gradient, on_grid) for
    every geometry, i.e. fields[f][b]; bc_kinds, roles, mu as for the
    library's forces and adjoint."""

    def __init__(self, grids, motions, fields, bc_kinds, vel_index, p_index, mu, dirs, placement="HGC",
                 dtype=torch.float32, device=None, layers=1):
        self.motions = motions
        self.t = 0.0
        self.R = Reconstructor(grids, [m.at(0.0) for m in motions], placement, device=device, layers=layers)
        self.grids = grids
        self.fields = fields
        self.kinds = list(bc_kinds)
        self.vel, self.p, self.mu = list(vel_index), p_index, mu
        self.dirs = np.asarray(dirs, dtype=np.float64)
        self.dtype = dtype
        dev = self.R.device
        np_dt = np.float32 if dtype == torch.float32 else np.float64
        # the manufactured field values (kept unchanged) and the working copies
        self.pristine = [torch.tensor(np.concatenate([f[b].on_grid(g, np_dt) for b, g in enumerate(grids)]),
                                      device=dev) for f in fields]
        self.work = [t.clone() for t in self.pristine]
        self.prev_cells = None
        self.R.build_levels()
        self.out = torch.empty(self.R.B * (2 * self.R.dim + 2), dtype=torch.float64, device=dev)

    def _bc(self, info):
        dim = self.R.dim
        out = []
        for f, kind in zip(self.fields, self.kinds):
            v = np.zeros(info["cell"].size)
            for b in range(self.R.B):
                sel = info["geom"] == b
                if not np.any(sel):
                    continue
                S, n = info["S"][sel, :dim], info["normal"][sel, :dim]
                v[sel] = f[b].value(S) if kind == 0 else np.sum(f[b].gradient(S) * n, axis=1)
            out.append(torch.tensor(v, dtype=self.dtype, device=self.R.device))
        return out

    def advance(self, dt, adjoint=False, seed=None):
        """Move the bodies to t + dt and reconstruct there.  Returns the
        forces [B, 2 dim + 2] (and the gradients when adjoint)."""
        R = self.R
        self.t += dt
        R.move([m.at(self.t) for m in self.motions])
        R.build_levels()
        info = R.ghost_info()
        cells = torch.tensor(R.cell_offset[info["geom"]] + info["cell"], device=R.device)
        if self.prev_cells is not None:
            for w, p0 in zip(self.work, self.pristine):
                w[self.prev_cells] = p0[self.prev_cells]
        self.prev_cells = cells
        bcs = self._bc(info)
        R.reconstruct(self.work, self.kinds, bcs)
        forces = R.forces([None if i is None else self.work[i] for i in self.vel], self.work[self.p], self.mu,
                          self.dirs, out=self.out)
        if not adjoint:
            return forces, info, bcs
        gf = [torch.zeros_like(w) for w in self.work]
        gb = [torch.zeros_like(b) for b in bcs]
        if seed is None:
            seed = torch.ones(R.B, 2, dtype=torch.float64, device=R.device)
        R.adjoint(self.kinds, self.vel, self.p, self.mu, self.dirs, seed, gf, gb)
        return forces, info, bcs, gf, gb
