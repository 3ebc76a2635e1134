"""Boundary quantities and forces (oracle; test infrastructure).

Sec. 6: the reconstruction relations, rearranged, give the solution and its
derivatives on the embedded boundary from the ghost value and its stencil.

* phi_s: the Dirichlet relation (Eq. phi_G_Dir_2d / phi_G_Dir_3d) solved for
  phi_s, i.e. phi_s = (phi_G - sum_k w_k phi_k) / ws with Dirichlet weights.
* Cartesian derivatives at S: Eq. derivative_bilinear (2D) and
  Eqs. derivative_trilinear_x / _y / _z (3D), in local coordinates (origin at
  G, so x_1 = 0, x_2 = r e dx, x_s = psi n).
* Forces.  The paper uses the surface values and gradients directly to form
  pressure forces, wall stresses, drag and lift (Sec. 6) but gives no
  quadrature.  Reading taken here: F = sum_G w_G f(S_G) with the local
  surface-element weight w_G = sum over the faces of G shared with a fluid
  cell (tag 0) of A_face |n . n_face| (A_face = dy for x-faces, dx for y-faces
  in 2D; dy dz, dx dz, dx dy in 3D), which sums to the length (area) of a
  straight wall exactly and to the perimeter (surface area) of a smooth body
  up to O(dx).  The integrand is the Newtonian traction
      f = -p_s n + mu (grad u + grad u^T)|_s n.
  This quadrature is parity unpinned against the paper (the paper does not
  state one); the tests pin its consistency (perimeter, divergence theorem).
"""

import math

import numpy as np

from .classify import ghost_x2
from .reconstruct import ghost_weights, DIRICHLET


def _members_values(lev, g, arr, K):
    return np.array([arr[lev.midx[g, k]] for k in range(K)], dtype=np.float64)


def phi_s(h, psi, n, e, r, phi_g, phi_m, x2=None):
    """Eq. phi_G_Dir_2d / _3d solved for phi_s."""
    w, ws = ghost_weights(h, psi, n, e, r, DIRICHLET, x2)
    return (phi_g - float(np.dot(w, phi_m))) / ws


def gradient_at_s(h, psi, n, e, r, phi_g, phi_m, x2=None):
    """Eq. derivative_bilinear (2D) or Eqs. derivative_trilinear_x/y/z (3D)."""
    d = len(h)
    x2 = [r[a] * e[a] * h[a] for a in range(d)] if x2 is None else [float(v) for v in x2]
    xs = [psi * n[a] for a in range(d)]
    if d == 2:
        x1 = y1 = 0.0
        X2, Y2 = x2
        Xs, Ys = xs
        p1, p2, p3 = phi_m
        pg = phi_g
        dx = ((Y2 - Ys) / (Y2 - y1)) * ((p1 - pg) / (X2 - x1)) \
            + ((Ys - y1) / (Y2 - y1)) * ((p3 - p2) / (X2 - x1))
        dy = ((X2 - Xs) / (X2 - x1)) * ((p2 - pg) / (Y2 - y1)) \
            + ((Xs - x1) / (X2 - x1)) * ((p3 - p1) / (Y2 - y1))
        return np.array([dx, dy])
    x1 = y1 = z1 = 0.0
    X2, Y2, Z2 = x2
    Xs, Ys, Zs = xs
    p1, p2, p3, p4, p5, p6, p7 = phi_m
    pg = phi_g
    fx0 = (X2 - Xs) / (X2 - x1)
    fx1 = (Xs - x1) / (X2 - x1)
    fy0 = (Y2 - Ys) / (Y2 - y1)
    fy1 = (Ys - y1) / (Y2 - y1)
    fz0 = (Z2 - Zs) / (Z2 - z1)
    fz1 = (Zs - z1) / (Z2 - z1)
    hx = X2 - x1
    hy = Y2 - y1
    hz = Z2 - z1
    dx = (fy0 * fz0 * (p1 - pg) / hx + fy1 * fz0 * (p4 - p2) / hx
          + fy0 * fz1 * (p6 - p3) / hx + fy1 * fz1 * (p7 - p5) / hx)
    dy = (fx0 * fz0 * (p2 - pg) / hy + fx1 * fz0 * (p4 - p1) / hy
          + fx0 * fz1 * (p5 - p3) / hy + fx1 * fz1 * (p7 - p6) / hy)
    dz = (fx0 * fy0 * (p3 - pg) / hz + fx1 * fy0 * (p6 - p1) / hz
          + fx0 * fy1 * (p5 - p2) / hz + fx1 * fy1 * (p7 - p4) / hz)
    return np.array([dx, dy, dz])


def boundary_quantities(cls, lev, arr):
    """(phi_s [N_g], grad [N_g, d]) for a filled field, canonical order."""
    h = cls.grid.h
    K = lev.midx.shape[1]
    ng = cls.n_ghosts
    ps = np.zeros(ng)
    gr = np.zeros((ng, cls.grid.dim))
    for p in range(ng):
        g = int(lev.order[p])
        pm = _members_values(lev, g, arr, K)
        pg = float(arr[cls.idx[g]])
        x2 = ghost_x2(cls, g)
        ps[p] = phi_s(h, cls.psi[g], cls.n[g], cls.e[g], cls.r[g], pg, pm, x2)
        gr[p] = gradient_at_s(h, cls.psi[g], cls.n[g], cls.e[g], cls.r[g], pg, pm, x2)
    return ps, gr


def face_weights(cls):
    """w_G per ghost (index order): sum over faces shared with tag-0 cells of
    A_face |n_face . n|.  (Quadrature reading; parity unpinned vs the paper.)"""
    g = cls.grid
    d = g.dim
    ijk = g.unlin(cls.idx)
    wid = g.widths(ijk)                      # the ghost cells' own widths
    w = np.zeros(cls.n_ghosts)
    for a in range(d):
        area = np.ones(cls.n_ghosts)
        for b in range(d):
            if b != a:
                area = area * wid[:, b]
        for s in (-1, 1):
            nb = ijk.copy()
            nb[:, a] += s
            ok = g.in_grid(nb)
            fl = np.zeros(cls.n_ghosts, dtype=bool)
            fl[ok] = cls.tags[g.lin(nb[ok])] == 0
            w += np.where(fl, area * np.abs(cls.n[:, a]), 0.0)
    return w


def ghost_force_term(h, psi, n, e, r, wG, mu, p_vals, vel_vals, x2=None):
    """Per-ghost traction times weight: (Fp [d], Fv [d]).

    p_vals / vel_vals[i]: (value at G, values at P_1..P_K) of the filled
    pressure / velocity component i (None: that component is identically 0).
    """
    d = len(h)
    pg, pm = p_vals
    ps = phi_s(h, psi, n, e, r, pg, pm, x2)
    G = np.zeros((d, d))                    # G[i, j] = d u_i / d x_j at S
    for i in range(d):
        if vel_vals[i] is not None:
            ug, um = vel_vals[i]
            G[i] = gradient_at_s(h, psi, n, e, r, ug, um, x2)
    fp = -ps * np.asarray(n, dtype=np.float64)
    fv = mu * ((G + G.T) @ np.asarray(n, dtype=np.float64))
    return wG * fp, wG * fv


def forces(cls, lev, p_arr, vel_arrs, mu, dirs):
    """[Fp (d), Fv (d), drag, lift] and the per-ghost terms.

    p_arr: filled pressure field; vel_arrs: list of d filled velocity fields
    (None for an identically zero component); dirs: [2][d] unit vectors along
    which drag and lift are measured.  Sums are exactly rounded (math.fsum).
    """
    d = cls.grid.dim
    h = cls.grid.h
    K = lev.midx.shape[1]
    wf = face_weights(cls)
    terms_p = []
    terms_v = []
    for p in range(cls.n_ghosts):
        g = int(lev.order[p])
        pv = (float(p_arr[cls.idx[g]]), _members_values(lev, g, p_arr, K))
        vv = [None if a is None else (float(a[cls.idx[g]]), _members_values(lev, g, a, K))
              for a in vel_arrs]
        fp, fv = ghost_force_term(h, cls.psi[g], cls.n[g], cls.e[g], cls.r[g], wf[g], mu, pv, vv,
                                  ghost_x2(cls, g))
        terms_p.append(fp)
        terms_v.append(fv)
    terms_p = np.array(terms_p).reshape(-1, d)
    terms_v = np.array(terms_v).reshape(-1, d)
    Fp = np.array([math.fsum(terms_p[:, a]) for a in range(d)])
    Fv = np.array([math.fsum(terms_v[:, a]) for a in range(d)])
    tot = terms_p + terms_v
    drag_t = tot @ np.asarray(dirs[0], dtype=np.float64)
    lift_t = tot @ np.asarray(dirs[1], dtype=np.float64)
    out = np.concatenate([Fp, Fv, [math.fsum(drag_t), math.fsum(lift_t)]])
    scale = np.concatenate([np.abs(terms_p).sum(0), np.abs(terms_v).sum(0),
                            [np.abs(drag_t).sum(), np.abs(lift_t).sum()]])
    return out, scale
