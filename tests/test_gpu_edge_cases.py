"""Degenerate geometry sets on the GPU.  A body that misses the grid, or
covers all of it, leaves no interface and no ghost cell (the oracle agrees).
In a batch such geometries sit before, between and after ordinary ones,
whose tags, levels, ghost values, forces and gradients must be unchanged;
their own forces are exactly zero and their gradients untouched.  Alone
they make an empty ghost set, on which every call is a no-op."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2609_10165_b300 import inputs as I
from paper_2609_10165_b300.api import Reconstructor
from tests.parity import DeviceRun, compare_structure, oracle_bcs
from tests.test_gpu_parity import _check_values, _small_cases, _with_fields

pytestmark = pytest.mark.gpu


def _empty_cases():
    return [
        {"grid": I.grid(2, [29, 23], [-1.0, -1.0], [1.0, 1.0]), "body": I.ellipse(3.0, 2.5, 0.4, 0.3, 0.4)},
        {"grid": I.grid(2, [19, 27], [-1.0, -1.0], [1.0, 1.0]), "body": I.circle(0.0, 0.0, 5.0)},
        {"grid": I.grid(2, [40, 20], [-1.0, -1.0], [3.0, 1.0]), "body": I.airfoil(10.0, 0.0, 0.12, 1.0, 5.0)},
    ]


def _mixed_batch():
    e = [_with_fields(c, 400 + 10 * k) for k, c in enumerate(_empty_cases())]
    s = [_with_fields(c, 450 + 10 * k) for k, c in enumerate(_small_cases()[:2])]   # ellipse, airfoil
    return [e[0], s[0], e[1], s[1], e[2]]


@pytest.mark.parametrize("placement", ["HGC", "CGC", "CGC_ES"])
@pytest.mark.parametrize("mode", ["level", "persistent"])
def test_empty_geometries_inside_a_batch(placement, mode):
    geoms = _mixed_batch()
    for dtype in (torch.float64, torch.float32):
        run = DeviceRun(geoms, placement, mode=mode, dtype=dtype)
        compare_structure(run, geoms, placement)
        _check_values(run, geoms, placement, dtype)
        counts = run.R.counts()
        for b in (0, 2, 4):
            assert counts[b]["n_ghosts"] == 0 and counts[b]["n_interface"] == 0, (b, counts[b])
            assert counts[b]["n_levels"] == 0


def test_empty_geometries_forces_and_adjoint():
    geoms = _mixed_batch()
    run = DeviceRun(geoms, "HGC", mode="persistent", dtype=torch.float64)
    dev = run.R.device
    arrays = run.field_arrays()
    bcs = run.bc_arrays()
    ft, _ = run.fill(arrays, bcs)
    dirs = I.DRAG_LIFT_DIRS_2D
    vel, p, mu = geoms[0]["roles"]["vel"], geoms[0]["roles"]["p"], geoms[0]["mu"]
    out = run.R.forces([ft[i] for i in vel], ft[p], mu, dirs).cpu().numpy()
    seed = torch.tensor([[0.7, -1.3]] * len(geoms), dtype=torch.float64, device=dev)
    gf = [torch.zeros(run.R.n_cells, dtype=torch.float64, device=dev) for _ in range(3)]
    gb = [torch.zeros(run.info["cell"].size, dtype=torch.float64, device=dev) for _ in range(3)]
    run.R.adjoint(geoms[0]["bc"], vel, p, mu, dirs, seed, gf, gb)
    run.R.sync_status()
    gf = [t.cpu().numpy() for t in gf]
    gb = [t.cpu().numpy() for t in gb]
    info = run.info
    for b, g in enumerate(geoms):
        o0, o1 = run.R.cell_offset[b], run.R.cell_offset[b + 1]
        sel = info["geom"] == b
        c = O.classify(g["grid"], g["body"], "HGC")
        lev = O.build_levels(c)
        filled = O.fill(c, lev, [a[o0:o1] for a in arrays], g["bc"], oracle_bcs(g, c, lev))
        ref, scale = O.forces(c, lev, filled[p], [filled[i] for i in vel], mu, dirs)
        assert np.all(np.abs(out[b] - ref) <= 1e-12 * scale + 1e-300), (b, out[b], ref)
        gx, gbo = O.adjoint_gradient(c, lev, g["bc"], p, vel, mu, dirs, (0.7, -1.3))
        if c.n_ghosts == 0:
            assert np.all(out[b] == 0.0)
            for f in range(3):
                assert np.all(gf[f][o0:o1] == 0.0) and not np.any(sel)
            continue
        for f in range(3):
            sc = max(np.abs(gx[f]).max(), np.abs(gbo[f]).max(), 1e-300)
            assert np.max(np.abs(gf[f][o0:o1] - gx[f])) <= 1e-11 * sc, (b, f)
            assert np.max(np.abs(gb[f][sel] - gbo[f])) <= 1e-11 * sc, (b, f)


@pytest.mark.parametrize("which", [[0], [1], [2], [0, 1, 2]])
def test_empty_ghost_set(which):
    cases = [_with_fields(_empty_cases()[k], 500 + k) for k in which]
    R = Reconstructor([c["grid"] for c in cases], [c["body"] for c in cases], "HGC")
    R.build_levels()
    R.sync_status()
    assert R.n_ghosts == 0
    assert all(c["n_levels"] == 0 and c["n_interface"] == 0 for c in R.counts())
    info = R.ghost_info()
    assert all(v.shape[0] == 0 for v in info.values())
    tags = R.tags.cpu().numpy()
    for b, case in enumerate(cases):
        c = O.classify(case["grid"], case["body"], "HGC")
        assert np.array_equal(tags[R.cell_offset[b]:R.cell_offset[b + 1]], c.tags)
    dev = R.device
    # zero ghosts: the boundary data and its gradient are empty tensors (null
    # pointers, which the ABI accepts for an empty ghost set)
    fields = [torch.randn(R.n_cells, dtype=torch.float64, device=dev) for _ in range(3)]
    before = [f.clone() for f in fields]
    bc = [torch.zeros(0, dtype=torch.float64, device=dev) for _ in range(3)]
    kinds = cases[0]["bc"]
    for mode in ("level", "persistent"):
        R.reconstruct(fields, kinds, bc, mode=mode)
    out = R.forces([fields[0], fields[1]], fields[2], 0.01, I.DRAG_LIFT_DIRS_2D)
    gf = [torch.zeros(R.n_cells, dtype=torch.float64, device=dev) for _ in range(3)]
    gb = [torch.zeros(0, dtype=torch.float64, device=dev) for _ in range(3)]
    seed = torch.ones(R.B, 2, dtype=torch.float64, device=dev)
    R.adjoint(kinds, [0, 1], 2, 0.01, I.DRAG_LIFT_DIRS_2D, seed, gf, gb)
    R.sync_status()
    for f in range(3):
        assert torch.equal(fields[f], before[f])
        assert not torch.any(gf[f] != 0)
    assert not torch.any(out != 0)
