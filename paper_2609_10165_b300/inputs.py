"""Seeded synthetic inputs: grids, bodies and manufactured fields.

This module only synthesises inputs.  It holds none of the reconstruction
method's arithmetic and imports nothing else from this package, so both the
CUDA path and the independent CPU check can consume exactly the same arrays.

Workloads (the paper's flows past a cylinder, Sec. 8.1, and an airfoil,
Sec. 8.2, restated as manufactured-solution fields):

* ``cylinder_128``: circle r = 0.5 centred in [-2,2]^2 on 128^2 cells;
  u = sin(2 pi x) cos(2 pi y) (Dirichlet data u(S)), p = x^2 + y^2 (Neumann
  data grad p(S) . n).
* ``airfoil_2048``: symmetric 4-digit thickness-formula airfoil t = 0.12,
  chord 1, leading edge at the origin, 5 deg nose-up, in [-1,3]x[-1,1] on
  2048 x 1024 cells; u, v (Dirichlet), p (Neumann) as tensor-product Fourier
  series with 8 modes per axis.
* ``sphere_512``: sphere r = 0.5 in [-2,2]^3 on 512^3 cells; u, v, w
  (Dirichlet), p (Neumann), 6 Fourier modes per axis.
* ``batch_256``: 256 geometries, alternating ellipses (semi-axes U(0.2,0.8),
  rotation U(0,pi), centre offset U(-0.05,0.05)^2, domain [-1,1]^2) and
  airfoils (t U(0.06,0.18), angle of attack U(0,10) deg, domain [-1,3]x[-1,1]);
  N x N cells with N log-uniform in [64, 1024]; 3 fields (u, v Dirichlet,
  p Neumann), 8 Fourier modes per axis.
* ``cylinder_1024`` / ``sphere_256``: the adjoint workloads.

Fourier fields: phi = sum_{p,q(,s)=1..M} a_pq(s) prod_axis cos(pi m xi_axis + theta_axis,m),
xi = (x - lo) / (hi - lo), a ~ U(-1,1) rescaled to sum |a| = 1 (so |phi| <= 1),
theta ~ U(0, 2 pi).  Seeds: 2609 + 1000 config + 10 geometry + field.
"""

import math

import numpy as np

SEED0 = 2609


def seed_of(config_id, geometry_id=0, field_id=0):
    return SEED0 + 1000 * config_id + 10 * geometry_id + field_id


def rot2(angle):
    """Row-major 3x3 body-to-world rotation by ``angle`` about z."""
    c, s = math.cos(angle), math.sin(angle)
    return [c, -s, 0.0, s, c, 0.0, 0.0, 0.0, 1.0]


IDENT = [1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0]


def grid(dim, n, lo, hi):
    n = list(n) + [1] * (3 - len(n))
    lo = list(lo) + [0.0] * (3 - len(lo))
    hi = list(hi) + [1.0] * (3 - len(hi))
    return {"dim": dim, "n": [int(v) for v in n], "lo": [float(v) for v in lo],
            "hi": [float(v) for v in hi]}


def axis_centres(g, a):
    """Cell centres along axis a of grid dict g: face midpoints of a stretched
    grid, lo + (i + 1/2) h of a uniform one."""
    if "faces" in g:
        f = np.asarray(g["faces"][a], dtype=np.float64)
        return 0.5 * (f[:-1] + f[1:])
    n = g["n"]
    return g["lo"][a] + (np.arange(n[a], dtype=np.float64) + 0.5) * ((g["hi"][a] - g["lo"][a]) / n[a])


def stretched_axis(lo, hi, n, ratio=1.03, centre_frac=0.5):
    """n + 1 increasing faces on [lo, hi] whose widths grow geometrically by
    `ratio` per cell away from the point centre_frac of the axis (the
    stretching of the paper's meshes, here applied everywhere so that the
    ghost stencils see it)."""
    c = centre_frac * n
    w = np.array([ratio ** abs(i + 0.5 - c) for i in range(n)], dtype=np.float64)
    w *= (hi - lo) / w.sum()
    f = np.concatenate([[lo], lo + np.cumsum(w)])
    f[-1] = hi
    return f


def stretched_grid(dim, n, lo, hi, ratio=(1.03, 1.03, 1.03), centre_frac=(0.5, 0.5, 0.5)):
    """Grid dict with explicit faces per axis (stretched_axis)."""
    g = grid(dim, n, lo, hi)
    g["faces"] = [stretched_axis(lo[a], hi[a], int(n[a]), ratio[a], centre_frac[a]).tolist() for a in range(dim)]
    return g


def circle(cx, cy, r):
    return {"kind": "circle", "centre": [cx, cy, 0.0], "radii": [r, r, 0.0], "rot": IDENT,
            "thickness": 0.0, "chord": 0.0}


def sphere(cx, cy, cz, r):
    return {"kind": "sphere", "centre": [cx, cy, cz], "radii": [r, r, r], "rot": IDENT,
            "thickness": 0.0, "chord": 0.0}


def ellipse(cx, cy, a, b, angle):
    return {"kind": "ellipse", "centre": [cx, cy, 0.0], "radii": [a, b, 0.0], "rot": rot2(angle),
            "thickness": 0.0, "chord": 0.0}


def airfoil(le_x, le_y, t, chord, aoa_deg):
    """Leading edge at (le_x, le_y); positive angle of attack pitches the nose
    up against a +x stream, i.e. the body frame is rotated by -aoa."""
    return {"kind": "airfoil", "centre": [le_x, le_y, 0.0], "radii": [0.0, 0.0, 0.0],
            "rot": rot2(-math.radians(aoa_deg)), "thickness": t, "chord": chord}


# ----------------------------------------------------------------------------
# manufactured fields
# ----------------------------------------------------------------------------

class FourierField:
    """Tensor-product cosine series on the box [lo, hi]."""

    def __init__(self, dim, modes, lo, hi, seed):
        rng = np.random.default_rng(seed)
        self.dim = dim
        self.M = modes
        self.lo = np.asarray(lo[:dim], dtype=np.float64)
        self.L = np.asarray(hi[:dim], dtype=np.float64) - self.lo
        a = rng.uniform(-1.0, 1.0, size=(modes,) * dim)
        self.a = a / np.abs(a).sum()
        self.theta = rng.uniform(0.0, 2.0 * math.pi, size=(dim, modes))
        self.k = math.pi * np.arange(1, modes + 1, dtype=np.float64)

    def _basis(self, axis, x):
        xi = (np.asarray(x, dtype=np.float64) - self.lo[axis]) / self.L[axis]
        arg = xi[:, None] * self.k[None, :] + self.theta[axis][None, :]
        return np.cos(arg), -np.sin(arg) * (self.k[None, :] / self.L[axis])

    def value(self, X):
        X = np.asarray(X, dtype=np.float64).reshape(-1, self.dim)
        B = [self._basis(a, X[:, a])[0] for a in range(self.dim)]
        if self.dim == 2:
            return np.einsum("pq,ip,iq->i", self.a, B[0], B[1])
        return np.einsum("pqs,ip,iq,is->i", self.a, B[0], B[1], B[2])

    def gradient(self, X):
        X = np.asarray(X, dtype=np.float64).reshape(-1, self.dim)
        B = [self._basis(a, X[:, a]) for a in range(self.dim)]
        out = np.zeros_like(X)
        for d in range(self.dim):
            F = [B[a][1] if a == d else B[a][0] for a in range(self.dim)]
            if self.dim == 2:
                out[:, d] = np.einsum("pq,ip,iq->i", self.a, F[0], F[1])
            else:
                out[:, d] = np.einsum("pqs,ip,iq,is->i", self.a, F[0], F[1], F[2])
        return out

    def on_grid(self, g, dtype=np.float64):
        """Values at every cell centre of grid dict ``g``, flattened x-fastest."""
        n = g["n"]
        cen = [axis_centres(g, a) for a in range(self.dim)]
        B = [self._basis(a, cen[a])[0] for a in range(self.dim)]
        if self.dim == 2:
            return (B[1] @ self.a.T @ B[0].T).astype(dtype).reshape(-1)   # [ny, nx]
        out = np.empty((n[2], n[1], n[0]), dtype=dtype)
        for kz in range(n[2]):
            Bz = np.einsum("pqs,s->pq", self.a, B[2][kz])
            out[kz] = (B[1] @ Bz.T @ B[0].T).astype(dtype)
        return out.reshape(-1)


class CylinderU:
    """u = sin(2 pi x) cos(2 pi y)."""
    dim = 2

    def value(self, X):
        X = np.asarray(X, dtype=np.float64).reshape(-1, 2)
        return np.sin(2 * math.pi * X[:, 0]) * np.cos(2 * math.pi * X[:, 1])

    def gradient(self, X):
        X = np.asarray(X, dtype=np.float64).reshape(-1, 2)
        sx, cx = np.sin(2 * math.pi * X[:, 0]), np.cos(2 * math.pi * X[:, 0])
        sy, cy = np.sin(2 * math.pi * X[:, 1]), np.cos(2 * math.pi * X[:, 1])
        return np.stack([2 * math.pi * cx * cy, -2 * math.pi * sx * sy], axis=1)

    def on_grid(self, g, dtype=np.float64):
        x = axis_centres(g, 0)
        y = axis_centres(g, 1)
        return (np.cos(2 * math.pi * y)[:, None] * np.sin(2 * math.pi * x)[None, :]).astype(dtype).reshape(-1)


class Quadratic:
    """p = |x|^2 (2D or 3D)."""

    def __init__(self, dim):
        self.dim = dim

    def value(self, X):
        X = np.asarray(X, dtype=np.float64).reshape(-1, self.dim)
        return np.sum(X * X, axis=1)

    def gradient(self, X):
        return 2.0 * np.asarray(X, dtype=np.float64).reshape(-1, self.dim)

    def on_grid(self, g, dtype=np.float64):
        n = g["n"]
        cen = [axis_centres(g, a) for a in range(self.dim)]
        if self.dim == 2:
            v = cen[1][:, None] ** 2 + cen[0][None, :] ** 2
        else:
            v = cen[2][:, None, None] ** 2 + cen[1][None, :, None] ** 2 + cen[0][None, None, :] ** 2
        return v.astype(dtype).reshape(-1)


class Polynomial:
    """Random (bi/tri)linear field C0 + C1 x + ... + C7 xyz (reproduced exactly
    by the closed forms, Secs. 4-5)."""

    def __init__(self, dim, seed):
        rng = np.random.default_rng(seed)
        self.dim = dim
        self.C = rng.uniform(-1.0, 1.0, size=4 if dim == 2 else 8)

    def value(self, X):
        X = np.asarray(X, dtype=np.float64).reshape(-1, self.dim)
        C = self.C
        if self.dim == 2:
            x, y = X[:, 0], X[:, 1]
            return C[0] + C[1] * x + C[2] * y + C[3] * x * y
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        return (C[0] + C[1] * x + C[2] * y + C[3] * z + C[4] * x * y + C[5] * y * z
                + C[6] * x * z + C[7] * x * y * z)

    def gradient(self, X):
        X = np.asarray(X, dtype=np.float64).reshape(-1, self.dim)
        C = self.C
        if self.dim == 2:
            x, y = X[:, 0], X[:, 1]
            return np.stack([C[1] + C[3] * y, C[2] + C[3] * x], axis=1)
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        return np.stack([C[1] + C[4] * y + C[6] * z + C[7] * y * z,
                         C[2] + C[4] * x + C[5] * z + C[7] * x * z,
                         C[3] + C[5] * y + C[6] * x + C[7] * x * y], axis=1)

    def on_grid(self, g, dtype=np.float64):
        n = g["n"][: self.dim]
        axes = [axis_centres(g, a) for a in range(self.dim)]
        mesh = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
        X = np.stack([m.reshape(-1) for m in mesh], axis=1)
        return self.value(X).astype(dtype)


def bc_values(field, kind, S, n):
    """Boundary data at points S [M, d] with unit normals n: phi(S) for a
    Dirichlet field (kind 0), grad phi(S) . n for a Neumann field (kind 1)."""
    if kind == 0:
        return field.value(S)
    return np.sum(field.gradient(S) * np.asarray(n, dtype=np.float64), axis=1)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

DIRICHLET, NEUMANN = 0, 1


def cylinder(n=128, config_id=1):
    g = grid(2, [n, n], [-2.0, -2.0], [2.0, 2.0])
    b = circle(0.0, 0.0, 0.5)
    fields = [CylinderU(), Quadratic(2)]
    return {"grid": g, "body": b, "fields": fields, "bc": [DIRICHLET, NEUMANN],
            "roles": {"p": 1, "vel": [0, None]}, "mu": 0.01}


def airfoil_2048(nx=2048, ny=1024, config_id=2):
    g = grid(2, [nx, ny], [-1.0, -1.0], [3.0, 1.0])
    b = airfoil(0.0, 0.0, 0.12, 1.0, 5.0)
    fields = [FourierField(2, 8, g["lo"], g["hi"], seed_of(config_id, 0, f)) for f in range(3)]
    return {"grid": g, "body": b, "fields": fields, "bc": [DIRICHLET, DIRICHLET, NEUMANN],
            "roles": {"p": 2, "vel": [0, 1]}, "mu": 5e-4}


def sphere_cfg(n=512, config_id=3):
    g = grid(3, [n, n, n], [-2.0, -2.0, -2.0], [2.0, 2.0, 2.0])
    b = sphere(0.0, 0.0, 0.0, 0.5)
    fields = [FourierField(3, 6, g["lo"], g["hi"], seed_of(config_id, 0, f)) for f in range(4)]
    return {"grid": g, "body": b, "fields": fields,
            "bc": [DIRICHLET, DIRICHLET, DIRICHLET, NEUMANN],
            "roles": {"p": 3, "vel": [0, 1, 2]}, "mu": 0.01}


def batch(n_geom=256, config_id=4, nmin=64, nmax=1024, modes=8):
    """List of geometry dicts for the batched workload."""
    out = []
    for gi in range(n_geom):
        rng = np.random.default_rng(seed_of(config_id, gi, 9))
        N = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        if gi % 2 == 0:
            g = grid(2, [N, N], [-1.0, -1.0], [1.0, 1.0])
            a, b = rng.uniform(0.2, 0.8, size=2)
            ang = rng.uniform(0.0, math.pi)
            cx, cy = rng.uniform(-0.05, 0.05, size=2)
            body = ellipse(float(cx), float(cy), float(a), float(b), float(ang))
        else:
            g = grid(2, [N, N], [-1.0, -1.0], [3.0, 1.0])
            t = rng.uniform(0.06, 0.18)
            aoa = rng.uniform(0.0, 10.0)
            body = airfoil(0.0, 0.0, float(t), 1.0, float(aoa))
        fields = [FourierField(2, modes, g["lo"], g["hi"], seed_of(config_id, gi, f)) for f in range(3)]
        out.append({"grid": g, "body": body, "fields": fields, "bc": [DIRICHLET, DIRICHLET, NEUMANN],
                    "roles": {"p": 2, "vel": [0, 1]}, "mu": 1e-3})
    return out


WORKLOADS = {
    "cylinder_128": lambda: cylinder(128, 1),
    "airfoil_2048": lambda: airfoil_2048(2048, 1024, 2),
    "sphere_512": lambda: sphere_cfg(512, 3),
    "cylinder_1024": lambda: cylinder(1024, 5),
    "sphere_256": lambda: sphere_cfg(256, 5),
}

DRAG_LIFT_DIRS_2D = [[1.0, 0.0], [0.0, 1.0]]
DRAG_LIFT_DIRS_3D = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]
