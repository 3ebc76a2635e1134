"""Cartesian grid and analytic embedded-boundary bodies (oracle; test infrastructure).

Sec. 3.1: every cell is classified by the position of its centre x_c.  For a
cell centre the boundary point S (x_s) is the intersection of the embedded
boundary (EB) with the boundary normal through x_c, and the signed normal
distance is psi = +|x_c - x_s| in the solid and -|x_c - x_s| in the fluid
(Eq. signed_distance), so psi >= 0 exactly when the centre is solid.  The unit
normal n points from the EB into the fluid.  With these conventions
S = x_c + psi * n for every cell.

Bodies (all convex): circle and sphere (closed form), ellipse (closest point
by bisection on the Lagrange-multiplier equation, Eberly's robust method, in
long double), and the symmetric 4-digit thickness-formula airfoil with an open
trailing edge closed by the base segment x = c (closest point by dense sampling
of the surface parameter u = sqrt(x/c) followed by bisection on the derivative
of the squared distance, in long double).
"""

import numpy as np

LD = np.longdouble

# 4-digit thickness-formula coefficients (open trailing edge).
AIRFOIL_A = (0.2969, -0.1260, -0.3516, 0.2843, -0.1015)


class Grid:
    """Cell-centred Cartesian grid, uniform or stretched.

    Uniform: cell (i, j[, k]) has centre lo_a + (i_a + 1/2) h_a with
    h_a = (hi_a - lo_a) / n_a.  Stretched (``faces`` given: per axis the n_a + 1
    increasing face coordinates): cell i_a spans [f_a(i_a), f_a(i_a + 1)], its
    centre is the midpoint and its width the difference (Sec. 7: local mesh
    spacing dx_i).  Linear index i + n_x (j + n_y k) (x fastest).

    ``h`` holds the spacing of a uniform grid, the smallest width per axis of a
    stretched one; ``hmax`` the largest.
    """

    def __init__(self, dim, n, lo, hi, faces=None):
        self.dim = int(dim)
        self.n = tuple(int(n[a]) for a in range(self.dim))
        self.stretched = faces is not None
        if self.stretched:
            self.faces = [np.asarray(faces[a], dtype=np.float64) for a in range(self.dim)]
            for a in range(self.dim):
                if self.faces[a].size != self.n[a] + 1 or not np.all(np.diff(self.faces[a]) > 0):
                    raise ValueError("axis %d needs %d increasing faces" % (a, self.n[a] + 1))
            self.lo = tuple(float(self.faces[a][0]) for a in range(self.dim))
            self.hi = tuple(float(self.faces[a][-1]) for a in range(self.dim))
            self.cen = [0.5 * (f[:-1] + f[1:]) for f in self.faces]
            self.wid = [np.diff(f) for f in self.faces]
            self.h = tuple(float(w.min()) for w in self.wid)
            self.hmax = tuple(float(w.max()) for w in self.wid)
        else:
            self.lo = tuple(float(lo[a]) for a in range(self.dim))
            self.hi = tuple(float(hi[a]) for a in range(self.dim))
            self.h = tuple((self.hi[a] - self.lo[a]) / self.n[a] for a in range(self.dim))
            self.hmax = self.h
        self.N = int(np.prod(self.n))

    @classmethod
    def from_dict(cls, d):
        return cls(d["dim"], d["n"], d["lo"], d["hi"], d.get("faces"))

    def centre(self, ijk):
        """Cell centres for integer index arrays ijk [M, dim] -> [M, dim] float64."""
        ijk = np.asarray(ijk, dtype=np.int64).reshape(-1, self.dim)
        out = np.empty(ijk.shape, dtype=np.float64)
        for a in range(self.dim):
            if self.stretched:
                out[:, a] = self.cen[a][ijk[:, a]]
            else:
                out[:, a] = self.lo[a] + (ijk[:, a].astype(np.float64) + 0.5) * self.h[a]
        return out

    def widths(self, ijk):
        """Cell widths [M, dim] of the cells ijk [M, dim]."""
        ijk = np.asarray(ijk, dtype=np.int64).reshape(-1, self.dim)
        out = np.empty(ijk.shape, dtype=np.float64)
        for a in range(self.dim):
            out[:, a] = self.wid[a][ijk[:, a]] if self.stretched else self.h[a]
        return out

    def lin(self, ijk):
        ijk = np.asarray(ijk, dtype=np.int64).reshape(-1, self.dim)
        idx = ijk[:, self.dim - 1].copy()
        for a in range(self.dim - 2, -1, -1):
            idx = idx * self.n[a] + ijk[:, a]
        return idx

    def unlin(self, idx):
        idx = np.asarray(idx, dtype=np.int64).reshape(-1)
        out = np.empty((idx.size, self.dim), dtype=np.int64)
        rem = idx.copy()
        for a in range(self.dim):
            out[:, a] = rem % self.n[a]
            rem //= self.n[a]
        return out

    def in_grid(self, ijk):
        ijk = np.asarray(ijk).reshape(-1, self.dim)
        ok = np.ones(ijk.shape[0], dtype=bool)
        for a in range(self.dim):
            ok &= (ijk[:, a] >= 0) & (ijk[:, a] < self.n[a])
        return ok


class Body:
    """Analytic body.  ``rot`` maps body-frame vectors to world vectors
    (x_world = rot @ x_body + centre), row-major 3x3."""

    def __init__(self, kind, centre=(0.0, 0.0, 0.0), radii=(0.0, 0.0, 0.0),
                 rot=(1, 0, 0, 0, 1, 0, 0, 0, 1), thickness=0.0, chord=1.0):
        self.kind = str(kind)
        self.centre = np.array([float(v) for v in centre] + [0.0] * (3 - len(centre)))
        self.radii = np.array([float(v) for v in radii] + [0.0] * (3 - len(radii)))
        self.rot = np.array([float(v) for v in rot], dtype=np.float64).reshape(3, 3)
        self.thickness = float(thickness)
        self.chord = float(chord)

    @classmethod
    def from_dict(cls, d):
        keys = ("kind", "centre", "radii", "rot", "thickness", "chord")
        return cls(**{k: d[k] for k in keys if k in d})

    @property
    def dim(self):
        return 3 if self.kind == "sphere" else 2


# ----------------------------------------------------------------------------
# body frame helpers
# ----------------------------------------------------------------------------

def _to_body_2d(body, X):
    dx = X[:, 0] - body.centre[0]
    dy = X[:, 1] - body.centre[1]
    R = body.rot
    px = R[0, 0] * dx + R[1, 0] * dy
    py = R[0, 1] * dx + R[1, 1] * dy
    return px, py


def airfoil_half_thickness(t, c, x):
    """y_t(x) of the symmetric 4-digit thickness formula, x in [0, c]."""
    xi = x / c
    a0, a1, a2, a3, a4 = AIRFOIL_A
    return 5.0 * t * c * (a0 * np.sqrt(xi) + a1 * xi + a2 * xi * xi
                          + a3 * xi * xi * xi + a4 * xi * xi * xi * xi)


def _airfoil_poly_u(t, c, u):
    """Upper surface as a polynomial in u = sqrt(x/c): returns (x, y, dx/du, dy/du)."""
    a0, a1, a2, a3, a4 = (LD(v) for v in AIRFOIL_A)
    k = LD(5.0) * LD(t) * LD(c)
    u2 = u * u
    x = LD(c) * u2
    y = k * (a0 * u + a1 * u2 + a2 * u2 * u2 + a3 * u2 * u2 * u2 + a4 * u2 * u2 * u2 * u2)
    dx = LD(2.0) * LD(c) * u
    dy = k * (a0 + LD(2.0) * a1 * u + LD(4.0) * a2 * u2 * u + LD(6.0) * a3 * u2 * u2 * u
              + LD(8.0) * a4 * u2 * u2 * u2 * u)
    return x, y, dx, dy


# ----------------------------------------------------------------------------
# inside predicate: psi >= 0  <=>  centre in the solid (Eq. signed_distance)
# ----------------------------------------------------------------------------

def inside(body, X):
    """True where the point is in the closed solid region (psi >= 0)."""
    X = np.asarray(X, dtype=np.float64)
    k = body.kind
    if k in ("circle", "sphere"):
        d = X - body.centre[: X.shape[1]]
        rho = np.sqrt(np.sum(d * d, axis=1))
        return (body.radii[0] - rho) >= 0.0
    if k == "ellipse":
        px, py = _to_body_2d(body, X)
        qx = px / body.radii[0]
        qy = py / body.radii[1]
        return (qx * qx + qy * qy) <= 1.0
    if k == "airfoil":
        px, py = _to_body_2d(body, X)
        c = body.chord
        ok = (px >= 0.0) & (px <= c)
        yt = np.zeros_like(px)
        yt[ok] = airfoil_half_thickness(body.thickness, c, px[ok])
        return ok & (np.abs(py) <= yt)
    raise ValueError("unknown body kind %r" % k)


# ----------------------------------------------------------------------------
# closest point
# ----------------------------------------------------------------------------

def _ellipse_closest_first_quadrant(e0, e1, y0, y1):
    """Closest point on x0^2/e0^2 + x1^2/e1^2 = 1 to (y0, y1), e0 >= e1 > 0,
    y0, y1 >= 0 (arrays, long double).  Bisection on
    F(s) = (r0 z0 / (s + r0))^2 + (z1 / (s + 1))^2 - 1, whose root gives the
    Lagrange multiplier (Eberly, "Distance from a point to an ellipse, an
    ellipsoid, or a hyperellipsoid")."""
    x0 = np.empty_like(y0)
    x1 = np.empty_like(y1)
    both = (y0 > 0) & (y1 > 0)
    on_y = (y0 == 0) & (y1 > 0)
    on_x = (y1 == 0)
    # generic case
    if np.any(both):
        a0 = y0[both]
        a1 = y1[both]
        z0 = a0 / e0
        z1 = a1 / e1
        g = z0 * z0 + z1 * z1 - LD(1)
        r0 = (e0 / e1) * (e0 / e1)
        n0 = r0 * z0
        s0 = z1 - LD(1)
        s1 = np.where(g < 0, LD(0), np.sqrt(n0 * n0 + z1 * z1) - LD(1))
        for _ in range(400):
            s = (s0 + s1) / LD(2)
            r_0 = n0 / (s + r0)
            r_1 = z1 / (s + LD(1))
            f = r_0 * r_0 + r_1 * r_1 - LD(1)
            s0 = np.where(f > 0, s, s0)
            s1 = np.where(f < 0, s, s1)
            s0 = np.where(f == 0, s, s0)
            s1 = np.where(f == 0, s, s1)
        s = (s0 + s1) / LD(2)
        s = np.where(g == 0, LD(0), s)
        x0[both] = r0 * a0 / (s + r0)
        x1[both] = a1 / (s + LD(1))
    if np.any(on_y):
        x0[on_y] = LD(0)
        x1[on_y] = e1
    if np.any(on_x):
        a0 = y0[on_x]
        numer0 = e0 * a0
        denom0 = e0 * e0 - e1 * e1
        inner = numer0 < denom0
        xde0 = np.where(inner, numer0 / np.where(denom0 > 0, denom0, LD(1)), LD(1))
        xx0 = np.where(inner, e0 * xde0, e0)
        xx1 = np.where(inner, e1 * np.sqrt(np.maximum(LD(1) - xde0 * xde0, LD(0))), LD(0))
        x0[on_x] = xx0
        x1[on_x] = xx1
    return x0, x1


def _closest_ellipse(body, X):
    px, py = _to_body_2d(body, X)
    a, b = body.radii[0], body.radii[1]
    swap = a < b
    e0, e1 = (LD(b), LD(a)) if swap else (LD(a), LD(b))
    qx = np.asarray(px, dtype=LD)
    qy = np.asarray(py, dtype=LD)
    u0, u1 = (qy, qx) if swap else (qx, qy)
    s0 = np.where(u0 < 0, LD(-1), LD(1))
    s1 = np.where(u1 < 0, LD(-1), LD(1))
    c0, c1 = _ellipse_closest_first_quadrant(e0, e1, np.abs(u0), np.abs(u1))
    c0 = c0 * s0
    c1 = c1 * s1
    sx, sy = (c1, c0) if swap else (c0, c1)          # body-frame S
    # outward normal of the ellipse at S is parallel to (sx / a^2, sy / b^2)
    nx = sx / (LD(a) * LD(a))
    ny = sy / (LD(b) * LD(b))
    nn = np.sqrt(nx * nx + ny * ny)
    nx = nx / nn
    ny = ny / nn
    dist = np.sqrt((qx - sx) ** 2 + (qy - sy) ** 2)
    return sx, sy, nx, ny, dist


def _closest_airfoil_upper(t, c, qx, qy, K=4096):
    """Closest point of the upper surface (u in [0, 1]) to body-frame points
    (qx, qy >= 0), long double.  Returns (u, squared distance)."""
    M = qx.size
    u_best = np.empty(M, dtype=LD)
    chunk = max(1, 2_000_000 // (K + 1))
    us = np.linspace(0.0, 1.0, K + 1).astype(LD)
    xs, ys, _, _ = _airfoil_poly_u(t, c, us)
    for s in range(0, M, chunk):
        e = min(M, s + chunk)
        dx = xs[None, :] - qx[s:e, None]
        dy = ys[None, :] - qy[s:e, None]
        k = np.argmin(dx * dx + dy * dy, axis=1)
        u_best[s:e] = us[k]
    # refine: bisection on g(u) = (P(u) - q) . P'(u) inside [u_k - 1/K, u_k + 1/K]
    lo = np.maximum(u_best - LD(1) / K, LD(0))
    hi = np.minimum(u_best + LD(1) / K, LD(1))

    def g(u):
        x, y, dx, dy = _airfoil_poly_u(t, c, u)
        return (x - qx) * dx + (y - qy) * dy

    glo = g(lo)
    ghi = g(hi)
    # g < 0 means the distance still decreases with u.  If g(lo) >= 0 the
    # minimum sits at lo (only possible when lo == 0); if g(hi) <= 0 at hi (== 1).
    at_lo = glo >= 0
    at_hi = ghi <= 0
    a = lo.copy()
    b = hi.copy()
    for _ in range(90):
        m = (a + b) / LD(2)
        gm = g(m)
        a = np.where(gm < 0, m, a)
        b = np.where(gm >= 0, m, b)
    u = (a + b) / LD(2)
    u = np.where(at_lo, lo, u)
    u = np.where(at_hi & ~at_lo, hi, u)
    x, y, _, _ = _airfoil_poly_u(t, c, u)
    d2 = (x - qx) ** 2 + (y - qy) ** 2
    return u, d2


def _closest_airfoil(body, X):
    px, py = _to_body_2d(body, X)
    t, c = body.thickness, body.chord
    qx = np.asarray(px, dtype=LD)
    qy_signed = np.asarray(py, dtype=LD)
    qy = np.abs(qy_signed)
    ins = inside(body, X)
    u, d2u = _closest_airfoil_upper(t, c, qx, qy)
    # base segment x = c, |y| <= y_t(c)
    _, yte, _, _ = _airfoil_poly_u(t, c, np.array([LD(1)]))
    yte = yte[0]
    by = np.minimum(qy, yte)
    d2b = (qx - LD(c)) ** 2 + (qy - by) ** 2
    use_base = d2b < d2u                 # exact tie -> upper surface
    xu, yu, dxu, dyu = _airfoil_poly_u(t, c, u)
    sx = np.where(use_base, LD(c), xu)
    sy = np.where(use_base, by, yu)
    # face normals: upper surface (-dy/du, dx/du)/|.|, base (1, 0)
    fn = np.sqrt(dxu * dxu + dyu * dyu)
    nxu = -dyu / fn
    nyu = dxu / fn
    nx = np.where(use_base, LD(1), nxu)
    ny = np.where(use_base, LD(0), nyu)
    # at the trailing-edge corner the outward direction of a fluid point is G - S
    corner = (~ins) & ((use_base & (qy > yte)) | ((~use_base) & (u == LD(1))))
    if np.any(corner):
        vx = qx[corner] - LD(c)
        vy = qy[corner] - yte
        vn = np.sqrt(vx * vx + vy * vy)
        nx[corner] = vx / vn
        ny[corner] = vy / vn
        sx[corner] = LD(c)
        sy[corner] = yte
    # mirror to the lower surface for points below the chord line
    neg = qy_signed < 0
    sy = np.where(neg, -sy, sy)
    ny = np.where(neg, -ny, ny)
    dist = np.sqrt((qx - sx) ** 2 + (qy_signed - sy) ** 2)
    return sx, sy, nx, ny, dist


def closest_point(body, X):
    """For points X [M, d]: (psi [M], n [M, d]) with psi >= 0 in the solid and
    n the unit normal at S pointing into the fluid; S = X + psi * n."""
    X = np.asarray(X, dtype=np.float64)
    M, d = X.shape
    k = body.kind
    if k in ("circle", "sphere"):
        dd = X - body.centre[:d]
        rho = np.sqrt(np.sum(dd * dd, axis=1))
        if np.any(rho == 0.0):
            raise ValueError("cell centre coincides with the body centre: normal undefined")
        psi = body.radii[0] - rho
        n = dd / rho[:, None]
        return psi, n
    if k in ("ellipse", "airfoil"):
        f = _closest_ellipse if k == "ellipse" else _closest_airfoil
        sx, sy, nxb, nyb, dist = f(body, X)
        ins = inside(body, X)
        psi = np.where(ins, dist, -dist).astype(np.float64)
        R = body.rot.astype(LD)
        nxw = R[0, 0] * nxb + R[0, 1] * nyb
        nyw = R[1, 0] * nxb + R[1, 1] * nyb
        n = np.stack([nxw, nyw], axis=1).astype(np.float64)
        return psi, n
    raise ValueError("unknown body kind %r" % k)
