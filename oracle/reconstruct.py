"""Closed-form ghost-cell reconstruction (oracle; test infrastructure).

Local coordinates with the origin at the ghost centre G (Appendix A): x_1 = 0,
x_2 = r e dx (the diagonally opposite stencil point, Sec. 7) and
x_s = psi n (S = G + psi n).  In these coordinates:

2D Dirichlet (Eq. phi_G_Dir_2d):
    phi_G = w1 phi1 + w2 phi2 - w1 w2 phi3 + (1-w1)(1-w2) phi_s,
    w1 = (x1 - xs)/(x2 - xs),  w2 = (y1 - ys)/(y2 - ys).
2D Neumann (Eq. phi_G_Neu_2d), a1 = n_x(y1-ys), a2 = n_x(y2-ys),
b1 = n_y(x1-xs), b2 = n_y(x2-xs):
    phi_G = w1 phi1 + w2 phi2 + (1-w1-w2) phi3 + ws dphi/dn,
    w1 = (a2+b1)/(a2+b2), w2 = (a1+b2)/(a2+b2), ws = -(x2-x1)(y2-y1)/(a2+b2).
3D Dirichlet (Eq. phi_G_Dir_3d) and 3D Neumann (Eq. phi_G_Neu_3d) with
a_ij = n_x(y_i-ys)(z_j-zs), b_ij = n_y(x_i-xs)(z_j-zs), c_ij = n_z(x_i-xs)(y_j-ys).

``vandermonde_ghost_value`` solves the 4x4 / 8x8 system of Appendix A by
Gaussian elimination in long double and returns C_0 = phi(G); the tests use it
to pin the closed forms.  ``fill`` applies the closed forms level by level
(Sec. 3.2): each ghost once, after every ghost it depends on.
"""

import numpy as np

from .classify import ghost_x2, stencil_offsets

DIRICHLET, NEUMANN = 0, 1
LD = np.longdouble


def local_points(h, psi, n, e, r, x2=None):
    """(x2 [d], xs [d]) in local coordinates (origin at G): x_2 = r e h on a
    uniform grid; on a stretched grid the given x_2 - x_1 (the centre of the
    cell r_i e_i cells away, Sec. 7 with the local spacing)."""
    d = len(h)
    if x2 is None:
        x2 = np.array([r[a] * e[a] * h[a] for a in range(d)], dtype=np.float64)
    else:
        x2 = np.asarray(x2, dtype=np.float64)
    xs = np.array([psi * n[a] for a in range(d)], dtype=np.float64)
    return x2, xs


def ghost_weights(h, psi, n, e, r, bc, x2=None):
    """Weights (w [K] on P_1..P_K, ws on the boundary datum)."""
    d = len(h)
    x2, xs = local_points(h, psi, n, e, r, x2)
    if d == 2:
        x1 = y1 = 0.0
        X2, Y2 = x2
        Xs, Ys = xs
        if bc == DIRICHLET:
            w1 = (x1 - Xs) / (X2 - Xs)
            w2 = (y1 - Ys) / (Y2 - Ys)
            return np.array([w1, w2, -w1 * w2]), (1 - w1) * (1 - w2)
        nx, ny = n[0], n[1]
        a1 = nx * (y1 - Ys)
        a2 = nx * (Y2 - Ys)
        b1 = ny * (x1 - Xs)
        b2 = ny * (X2 - Xs)
        den = a2 + b2
        w1 = (a2 + b1) / den
        w2 = (a1 + b2) / den
        ws = -(X2 - x1) * (Y2 - y1) / den
        return np.array([w1, w2, 1 - w1 - w2]), ws
    x1 = y1 = z1 = 0.0
    X2, Y2, Z2 = x2
    Xs, Ys, Zs = xs
    if bc == DIRICHLET:
        w1 = (x1 - Xs) / (X2 - Xs)
        w2 = (y1 - Ys) / (Y2 - Ys)
        w3 = (z1 - Zs) / (Z2 - Zs)
        w = np.array([w1, w2, w3, -w1 * w2, -w2 * w3, -w1 * w3, w1 * w2 * w3])
        return w, (1 - w1) * (1 - w2) * (1 - w3)
    nx, ny, nz = n[0], n[1], n[2]
    xi = (x1, X2)
    yi = (y1, Y2)
    zi = (z1, Z2)

    def a(i, j):
        return nx * (yi[i - 1] - Ys) * (zi[j - 1] - Zs)

    def b(i, j):
        return ny * (xi[i - 1] - Xs) * (zi[j - 1] - Zs)

    def c(i, j):
        return nz * (xi[i - 1] - Xs) * (yi[j - 1] - Ys)

    den = a(2, 2) + b(2, 2) + c(2, 2)
    w = np.array([
        (a(2, 2) + b(1, 2) + c(1, 2)) / den,
        (a(1, 2) + b(2, 2) + c(2, 1)) / den,
        (a(2, 1) + b(2, 1) + c(2, 2)) / den,
        -(a(1, 2) + b(1, 2) + c(1, 1)) / den,
        -(a(1, 1) + b(2, 1) + c(2, 1)) / den,
        -(a(2, 1) + b(1, 1) + c(1, 2)) / den,
        (a(1, 1) + b(1, 1) + c(1, 1)) / den,
    ])
    ws = -(X2 - x1) * (Y2 - y1) * (Z2 - z1) / den
    return w, ws


def ghost_value(h, psi, n, e, r, bc, phi_members, datum, x2=None):
    w, ws = ghost_weights(h, psi, n, e, r, bc, x2)
    return float(np.dot(w, phi_members) + ws * datum)


def _solve_ld(A, b):
    """Gaussian elimination with partial pivoting in long double."""
    A = np.array(A, dtype=LD)
    b = np.array(b, dtype=LD)
    m = A.shape[0]
    for k in range(m):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if p != k:
            A[[k, p]] = A[[p, k]]
            b[[k, p]] = b[[p, k]]
        for i in range(k + 1, m):
            f = A[i, k] / A[k, k]
            A[i, k:] -= f * A[k, k:]
            b[i] -= f * b[k]
    x = np.zeros(m, dtype=LD)
    for i in range(m - 1, -1, -1):
        x[i] = (b[i] - np.dot(A[i, i + 1:], x[i + 1:])) / A[i, i]
    return x


def vandermonde_ghost_value(h, psi, n, e, r, bc, phi_members, datum, x2=None):
    """C_0 of the (bi/tri)linear interpolant through the stencil and the
    boundary condition: the Appendix A system, solved directly."""
    d = len(h)
    x2, xs = local_points(h, psi, n, e, r, x2)
    offs = stencil_offsets(d)
    if d == 2:
        def row(p):
            x, y = p
            return [1.0, x, y, x * y]
        rows = [row((o[0] * x2[0], o[1] * x2[1])) for o in offs]
        if bc == DIRICHLET:
            rows.append(row(xs))
        else:
            Xs, Ys = xs
            rows.append([0.0, n[0], n[1], n[0] * Ys + n[1] * Xs])
    else:
        def row(p):
            x, y, z = p
            return [1.0, x, y, z, x * y, y * z, x * z, x * y * z]
        rows = [row((o[0] * x2[0], o[1] * x2[1], o[2] * x2[2])) for o in offs]
        if bc == DIRICHLET:
            rows.append(row(xs))
        else:
            Xs, Ys, Zs = xs
            nx, ny, nz = n
            rows.append([0.0, nx, ny, nz, Xs * ny + Ys * nx, Ys * nz + Zs * ny,
                         Xs * nz + Zs * nx, Xs * Ys * nz + Ys * Zs * nx + Xs * Zs * ny])
    rhs = list(phi_members) + [datum]
    C = _solve_ld(rows, rhs)
    return float(C[0])


def fill(cls, lev, fields, bc_kinds, bc_data):
    """Level-by-level reconstruction of every ghost for every field.

    fields:   list of F arrays [N] (copied, float64)
    bc_kinds: list of F in {DIRICHLET, NEUMANN}
    bc_data:  list of F arrays [N_g] in canonical (level, index) order: phi_s
              for Dirichlet, dphi/dn at S for Neumann.
    Returns the list of filled arrays.
    """
    out = [np.array(f, dtype=np.float64, copy=True) for f in fields]
    h = cls.grid.h
    W = {}
    for p in range(cls.n_ghosts):
        g = int(lev.order[p])
        for fi, arr in enumerate(out):
            bc = bc_kinds[fi]
            if (g, bc) not in W:
                W[(g, bc)] = ghost_weights(h, cls.psi[g], cls.n[g], cls.e[g], cls.r[g], bc, ghost_x2(cls, g))
            w, ws = W[(g, bc)]
            acc = ws * float(bc_data[fi][p])
            for k in range(w.size):
                if lev.active[g, k]:
                    acc += w[k] * arr[lev.midx[g, k]]
            arr[cls.idx[g]] = acc
    return out
