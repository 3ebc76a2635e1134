"""Gradient of J = s_d drag + s_l lift (oracle; test infrastructure).

For fixed geometry the whole path is linear: the ghost values g_f of field f
satisfy g_f = A_gg g_f + A_gx x_f + A_gb b_f (one closed-form row per ghost,
Secs. 4-5; x_f the field values, b_f the boundary data), and J is a linear
function of the filled values (Sec. 6 relations, force reading in
``surface``).  So

    J = sum_f c_g,f . g_f + c_x,f . x_f,
    dJ/dx_f = c_x,f + A_gx^T lambda_f,   dJ/db_f = A_gb^T lambda_f,
    (I - A_gg)^T lambda_f = c_g,f.

The matrices are assembled explicitly: every closed-form row from
``ghost_weights`` and every force coefficient by evaluating the per-ghost
force term on unit inputs (it is linear in the stencil values).  The
transposed system is solved with a sparse direct solver.  This is a different
algorithm from a reverse level walk.  Values at ghost slots of the input
fields are overwritten by the fill, so their gradient is zero.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .classify import ghost_x2
from .reconstruct import ghost_weights
from .surface import face_weights, ghost_force_term


def linear_map(cls, lev, bc_kinds):
    """Per field: (A_gg, A_gx, A_gb) as scipy CSR matrices in canonical order."""
    ng = cls.n_ghosts
    N = cls.grid.N
    h = cls.grid.h
    pos = lev.position()
    K = lev.midx.shape[1]
    ghost_pos = {int(c): int(pos[g]) for g, c in enumerate(cls.idx)}
    mats = []
    for bc in bc_kinds:
        rg, cg, vg = [], [], []
        rx, cx, vx = [], [], []
        wsv = np.zeros(ng)
        for g in range(ng):
            q = int(pos[g])
            w, ws = ghost_weights(h, cls.psi[g], cls.n[g], cls.e[g], cls.r[g], bc, ghost_x2(cls, g))
            wsv[q] = ws
            for k in range(K):
                if not lev.active[g, k]:
                    continue
                m = int(lev.midx[g, k])
                if m in ghost_pos:
                    rg.append(q); cg.append(ghost_pos[m]); vg.append(w[k])
                else:
                    rx.append(q); cx.append(m); vx.append(w[k])
        Agg = sp.csr_matrix((vg, (rg, cg)), shape=(ng, ng))
        Agx = sp.csr_matrix((vx, (rx, cx)), shape=(ng, N))
        Agb = sp.diags(wsv).tocsr()
        mats.append((Agg, Agx, Agb))
    return mats


def force_coefficients(cls, lev, n_fields, p_id, vel_ids, mu, dirs, seed):
    """c_g [F][N_g] (canonical order) and c_x [F][N] with
    J = sum_f c_g[f] . g_f + c_x[f] . x_f."""
    d = cls.grid.dim
    h = cls.grid.h
    K = lev.midx.shape[1]
    N = cls.grid.N
    pos = lev.position()
    ghost_pos = {int(c): int(pos[g]) for g, c in enumerate(cls.idx)}
    wf = face_weights(cls)
    cgv = np.zeros((n_fields, cls.n_ghosts))
    cxv = np.zeros((n_fields, N))
    dirs = np.asarray(dirs, dtype=np.float64)
    roles = [("p", p_id)] + [("v%d" % i, f) for i, f in enumerate(vel_ids)]
    zero = (0.0, np.zeros(K))
    for g in range(cls.n_ghosts):
        for role, f in roles:
            if f is None:
                continue
            for slot in range(K + 1):
                unit = np.zeros(K + 1)
                unit[slot] = 1.0
                uv = (unit[0], unit[1:])
                if role == "p":
                    pv = uv
                    vv = [None] * d
                else:
                    pv = zero
                    vv = [None] * d
                    vv[int(role[1:])] = uv
                fp, fv = ghost_force_term(h, cls.psi[g], cls.n[g], cls.e[g], cls.r[g],
                                          wf[g], mu, pv, vv, ghost_x2(cls, g))
                tot = fp + fv
                c = seed[0] * float(tot @ dirs[0]) + seed[1] * float(tot @ dirs[1])
                if c == 0.0:
                    continue
                cell = int(cls.idx[g]) if slot == 0 else int(lev.midx[g, slot - 1])
                if cell in ghost_pos:
                    cgv[f, ghost_pos[cell]] += c
                else:
                    cxv[f, cell] += c
    return cgv, cxv


def fill_vjp(cls, lev, bc_kinds, ybar):
    """Vector-Jacobian product of the in-place fill (Sec. 3.2 with the closed
    forms of Secs. 4-5): the fill maps (x, b) to y with y = x on non-ghost
    cells and y_g = g on ghost cells, g = (I - A_gg)^-1 (A_gx x + A_gb b).
    Given ybar [F][N] (dJ/dy) returns (xbar [F][N], bbar [F][N_g] canonical):
        (I - A_gg)^T lambda = ybar on the ghosts,
        xbar = ybar + A_gx^T lambda, with xbar = 0 on the ghost cells,
        bbar = A_gb^T lambda."""
    kinds = sorted(set(int(k) for k in bc_kinds))
    by_kind = dict(zip(kinds, linear_map(cls, lev, kinds)))
    ng = cls.n_ghosts
    pos = lev.position()
    cells = np.zeros(ng, dtype=np.int64)
    cells[pos] = cls.idx                      # ghost cell of canonical position q
    I = sp.identity(ng, format="csc")
    xbar, bbar = [], []
    for f, kind in enumerate(bc_kinds):
        Agg, Agx, Agb = by_kind[int(kind)]
        y = np.asarray(ybar[f], dtype=np.float64)
        yg = y[cells]
        if ng > 1:
            lam = np.atleast_1d(spla.spsolve((I - Agg).T.tocsc(), yg))
        elif ng == 1:
            lam = yg / (1.0 - Agg.toarray()[0, 0])
        else:
            lam = np.zeros(0)
        xb = y + Agx.T @ lam
        xb[cells] = 0.0
        xbar.append(xb)
        bbar.append(Agb.T @ lam)
    return xbar, bbar


def adjoint_gradient(cls, lev, bc_kinds, p_id, vel_ids, mu, dirs, seed):
    """(grad_fields [F][N], grad_bc [F][N_g] canonical order) of
    J = seed[0] drag + seed[1] lift."""
    F = len(bc_kinds)
    mats = linear_map(cls, lev, bc_kinds)
    cg, cx = force_coefficients(cls, lev, F, p_id, vel_ids, mu, dirs, seed)
    ng = cls.n_ghosts
    I = sp.identity(ng, format="csc")
    gx = np.zeros((F, cls.grid.N))
    gb = np.zeros((F, ng))
    for f, (Agg, Agx, Agb) in enumerate(mats):
        if ng:
            lam = spla.spsolve((I - Agg).T.tocsc(), cg[f]) if ng > 1 else cg[f] / (1.0 - Agg.toarray()[0, 0])
            lam = np.atleast_1d(lam)
        else:
            lam = np.zeros(0)
        gx[f] = cx[f] + Agx.T @ lam
        gb[f] = Agb.T @ lam
        gx[f][cls.idx] = 0.0
    return gx, gb
