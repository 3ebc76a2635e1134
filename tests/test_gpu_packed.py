"""GPU parity of the many-field, field-minor path (ebr_reconstruct_packed and
its transpose) against the oracle's level-walk fill and its vector-Jacobian
product, on seeded random fields.  FP64 within 1e-12 of the magnitude of the
terms, FP32 within 1e-5 of the largest magnitude (tests/parity.py); the
packed fill must equal the per-field-array fill bit for bit, the two packed
kernels must satisfy the adjoint identity, and the transpose must be bitwise
reproducible."""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

import oracle as O
from paper_2609_10165_b300 import inputs as I
from paper_2609_10165_b300.api import Reconstructor
from tests.parity import compare_structure

pytestmark = pytest.mark.gpu

MIXED_2D = [
    {"grid": I.grid(2, [37, 29], [-1.0, -1.0], [1.0, 1.0]), "body": I.ellipse(0.03, -0.02, 0.6, 0.35, 0.7)},
    {"grid": I.grid(2, [131, 67], [-1.0, -1.0], [3.0, 1.0]), "body": I.airfoil(0.0, 0.0, 0.12, 1.0, 5.0)},
    {"grid": I.grid(2, [33, 33], [-1.0, -1.0], [1.0, 1.0]), "body": I.circle(0.0, 0.0, 0.55)},
    {"grid": I.grid(2, [64, 45], [-1.0, -1.0], [1.0, 1.0]), "body": I.ellipse(-0.05, 0.04, 0.7, 0.25, 2.1)},
]
SPHERE_3D = [
    {"grid": I.grid(3, [21, 18, 19], [-1.0, -1.0, -1.0], [1.0, 1.0, 1.0]), "body": I.sphere(0.02, -0.01, 0.03, 0.6)},
]


def _kinds(F):
    # a Dirichlet / Neumann pattern that is not periodic in 32
    return [I.NEUMANN if (f % 3 == 2 or f % 7 == 0) else I.DIRICHLET for f in range(F)]


def _setup(cases, placement, F, dtype, seed):
    R = Reconstructor([c["grid"] for c in cases], [c["body"] for c in cases], placement)
    R.build_levels()
    R.sync_status()
    info = R.ghost_info()
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(R.n_cells, F))
    b = rng.normal(size=(info["cell"].size, F))
    if dtype == torch.float32:
        x = x.astype(np.float32).astype(np.float64)
        b = b.astype(np.float32).astype(np.float64)
    return R, info, x, b


def _maps(c, lev):
    """The oracle's linear map of the fill, per boundary-condition kind."""
    m = O.linear_map(c, lev, [O.DIRICHLET, O.NEUMANN])
    return {O.DIRICHLET: m[0], O.NEUMANN: m[1]}


def _abs_vjp(c, lev, kinds, ybar_abs, maps):
    """Magnitude of the terms of the transpose: the same solve with |weights|."""
    ng = c.n_ghosts
    pos = lev.position()
    cells = np.zeros(ng, dtype=np.int64)
    cells[pos] = c.idx
    Id = sp.identity(ng, format="csc")
    out = []
    for f, kind in enumerate(kinds):
        Agg, Agx, Agb = maps[kind]
        yg = ybar_abs[f][cells]
        A = abs(Agg)
        lam = np.atleast_1d(spla.spsolve((Id - A).T.tocsc(), yg)) if ng > 1 else yg / (1.0 - A.toarray()[0, 0])
        out.append((ybar_abs[f] + abs(Agx).T @ lam, abs(Agb).T @ lam))
    return out


def _check_fill(R, info, cases, placement, kinds, x, b, got, dtype):
    F = len(kinds)
    for gi, case in enumerate(cases):
        o0, o1 = R.cell_offset[gi], R.cell_offset[gi + 1]
        sel = info["geom"] == gi
        c = O.classify(case["grid"], case["body"], placement)
        lev = O.build_levels(c)
        loc = [x[o0:o1, f].copy() for f in range(F)]
        bl = [b[sel, f] for f in range(F)]
        out = O.fill(c, lev, loc, kinds, bl)
        maps = _maps(c, lev) if dtype == torch.float64 else None
        cells = c.idx[lev.order]
        mask = np.ones(o1 - o0, bool)
        mask[cells] = False
        for f in range(F):
            ref = out[f][cells]
            diff = np.abs(got[o0:o1, f][cells] - ref)
            if dtype == torch.float64:
                # magnitude of the terms: the fill of |x|, |b| with |weights|
                tol = 1e-12 * (np.abs(ref) + _term_bound(c, maps[kinds[f]], loc[f], bl[f]))
            else:
                tol = 1e-5 * max(np.abs(loc[f]).max(), np.abs(bl[f]).max(), np.abs(ref).max())
            assert np.all(diff <= tol), (gi, f, float(diff.max()))
            assert np.array_equal(got[o0:o1, f][mask], x[o0:o1, f][mask])


def _term_bound(c, mats, xa, ba):
    Agg, Agx, Agb = mats
    ng = c.n_ghosts
    Id = sp.identity(ng, format="csc")
    rhs = abs(Agx) @ np.abs(xa) + abs(Agb) @ np.abs(ba)
    return np.atleast_1d(spla.spsolve((Id - abs(Agg)).tocsc(), rhs)) if ng > 1 else rhs


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("F", [1, 5, 40, 130, 1024])   # 1024: the ABI maximum
def test_packed_fill_matches_oracle(dtype, F):
    R, info, x, b = _setup(MIXED_2D, "HGC", F, dtype, 7 + F)
    compare_structure(R_run(R, info), MIXED_2D, "HGC")
    kinds = _kinds(F)
    ft = torch.tensor(x, dtype=dtype, device=R.device)
    bt = torch.tensor(b, dtype=dtype, device=R.device)
    R.reconstruct_packed(ft, kinds, bt)
    R.sync_status()
    _check_fill(R, info, MIXED_2D, "HGC", kinds, x, b, ft.double().cpu().numpy(), dtype)


class R_run:
    """Adapter for compare_structure (expects .R and .info)."""

    def __init__(self, R, info):
        self.R, self.info = R, info


@pytest.mark.parametrize("placement", ["CGC", "CGC_ES"])
def test_packed_fill_other_placements_and_3d(placement):
    for cases in (MIXED_2D, SPHERE_3D):
        R, info, x, b = _setup(cases, placement, 33, torch.float64, 11)
        kinds = _kinds(33)
        ft = torch.tensor(x, dtype=torch.float64, device=R.device)
        bt = torch.tensor(b, dtype=torch.float64, device=R.device)
        R.reconstruct_packed(ft, kinds, bt)
        R.sync_status()
        _check_fill(R, info, cases, placement, kinds, x, b, ft.cpu().numpy(), torch.float64)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_packed_fill_equals_field_arrays_bitwise(dtype):
    R, info, x, b = _setup(MIXED_2D + [], "HGC", 3, dtype, 5)
    kinds = [I.DIRICHLET, I.DIRICHLET, I.NEUMANN]
    ft = torch.tensor(x, dtype=dtype, device=R.device)
    bt = torch.tensor(b, dtype=dtype, device=R.device)
    fa = [ft[:, f].contiguous() for f in range(3)]
    ba = [bt[:, f].contiguous() for f in range(3)]
    R.reconstruct(fa, kinds, ba, mode="persistent")
    R.reconstruct_packed(ft, kinds, bt)
    R.sync_status()
    for f in range(3):
        assert torch.equal(ft[:, f], fa[f])


def test_packed_adjoint_identity_fp64():
    """<ybar, fill(x, b)> = <xbar, x> + <bbar, b> for the GPU fill and the GPU
    transpose: the two kernels are transposes of one linear map (the ghost
    entries of the filled field depend only on fluid entries and boundary
    data, every other entry passes through)."""
    for cases, F in ((MIXED_2D, 7), (SPHERE_3D, 5)):
        R, info, x, b = _setup(cases, "HGC", F, torch.float64, 17)
        kinds = _kinds(F)
        rng = np.random.default_rng(18)
        ybar = rng.normal(size=(R.n_cells, F))
        y = torch.tensor(x, device=R.device)
        R.reconstruct_packed(y, kinds, torch.tensor(b, device=R.device))
        cot = torch.tensor(ybar, device=R.device)
        gb = torch.empty((info["cell"].size, F), dtype=torch.float64, device=R.device)
        R.reconstruct_packed_adjoint(kinds, cot, gb)
        R.sync_status()
        yb = torch.tensor(ybar, device=R.device)
        xt, bt = torch.tensor(x, device=R.device), torch.tensor(b, device=R.device)
        lhs = float((yb * y).sum())
        rhs = float((cot * xt).sum() + (gb * bt).sum())
        scale = float((yb.abs() * y.abs()).sum())
        assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("placement,F", [("HGC", 5), ("HGC", 40), ("CGC_ES", 3), ("HGC", 130)])
def test_packed_adjoint_matches_oracle_vjp(dtype, placement, F):
    cases = MIXED_2D
    R, info, x, b = _setup(cases, placement, F, dtype, 21 + F)
    kinds = _kinds(F)
    rng = np.random.default_rng(99 + F)
    ybar = rng.normal(size=(R.n_cells, F))
    if dtype == torch.float32:
        ybar = ybar.astype(np.float32).astype(np.float64)
    cot = torch.tensor(ybar, dtype=dtype, device=R.device)
    gb = torch.full((info["cell"].size, F), float("nan"), dtype=dtype, device=R.device)
    R.reconstruct_packed_adjoint(kinds, cot, gb)
    R.sync_status()
    got = cot.double().cpu().numpy()
    gbn = gb.double().cpu().numpy()
    assert np.all(np.isfinite(gbn))
    for gi, case in enumerate(cases):
        o0, o1 = R.cell_offset[gi], R.cell_offset[gi + 1]
        sel = info["geom"] == gi
        c = O.classify(case["grid"], case["body"], placement)
        lev = O.build_levels(c)
        yl = [ybar[o0:o1, f] for f in range(F)]
        xbar, bbar = O.fill_vjp(c, lev, kinds, yl)
        mag = _abs_vjp(c, lev, kinds, [np.abs(v) for v in yl], _maps(c, lev))
        for f in range(F):
            if dtype == torch.float64:
                tx, tb = 1e-12 * mag[f][0], 1e-12 * mag[f][1]
            else:
                m = max(mag[f][0].max(), mag[f][1].max() if mag[f][1].size else 0.0)
                tx = tb = 1e-5 * m
            dx = np.abs(got[o0:o1, f] - xbar[f])
            db = np.abs(gbn[sel, f] - bbar[f])
            assert np.all(dx <= tx), (gi, f, float(dx.max()))
            assert np.all(db <= tb), (gi, f, float(db.max()))
            assert np.all(got[o0:o1, f][c.idx] == 0.0)


def test_packed_adjoint_bitwise_reproducible_and_3d():
    for cases in (MIXED_2D, SPHERE_3D):
        R, info, x, b = _setup(cases, "HGC", 36, torch.float32, 3)
        kinds = _kinds(36)
        rng = np.random.default_rng(4)
        ybar = torch.tensor(rng.normal(size=(R.n_cells, 36)), dtype=torch.float32, device=R.device)
        outs = []
        for _ in range(2):
            cot = ybar.clone()
            gb = torch.empty((info["cell"].size, 36), dtype=torch.float32, device=R.device)
            R.reconstruct_packed_adjoint(kinds, cot, gb)
            R.sync_status()
            outs.append((cot, gb))
        assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
        if cases is SPHERE_3D:
            c = O.classify(cases[0]["grid"], cases[0]["body"], "HGC")
            lev = O.build_levels(c)
            yl = [ybar[:, f].double().cpu().numpy() for f in range(36)]
            xbar, bbar = O.fill_vjp(c, lev, kinds, yl)
            mag = _abs_vjp(c, lev, kinds, [np.abs(v) for v in yl], _maps(c, lev))
            got = outs[0][0].double().cpu().numpy()
            for f in range(36):
                assert np.all(np.abs(got[:, f] - xbar[f]) <= 1e-5 * mag[f][0].max())


def test_packed_argument_errors():
    R, info, x, b = _setup(MIXED_2D[:1], "HGC", 4, torch.float32, 1)
    ft = torch.zeros((R.n_cells, 4), dtype=torch.float32, device=R.device)
    bt = torch.zeros((info["cell"].size, 4), dtype=torch.float32, device=R.device)
    with pytest.raises(ValueError):
        R.reconstruct_packed(ft[:-1], _kinds(4), bt)
    with pytest.raises(Exception):
        R.reconstruct_packed(ft, [5, 0, 0, 0], bt)
    big = torch.zeros((R.n_cells, 1025), dtype=torch.float32, device=R.device)
    with pytest.raises(Exception):
        R.reconstruct_packed(big, [0] * 1025, torch.zeros((info["cell"].size, 1025), device=R.device))
