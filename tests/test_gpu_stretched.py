"""GPU parity on stretched grids (per-cell widths, ebr_plan_faces): tags,
ghost lists, levels and r_i bit-exact, psi / n / S against the oracle's
closest points, ghost values (FP64 within 1e-12 of their terms, FP32 within
1e-5 of the field maximum) for every placement and with the second layer,
forces and the adjoint gradient; a batch that mixes stretched and uniform
grids; a stretched 1024x512 airfoil."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2609_10165_b300 import inputs as I
from tests.parity import DeviceRun, compare_structure, oracle_bcs
from tests.test_gpu_parity import _check_values
from tests.test_oracle_stretched import CASES

pytestmark = pytest.mark.gpu


def _with_fields(gd, bd, seed):
    d = gd["dim"]
    return {"grid": gd, "body": bd,
            "fields": [I.FourierField(d, 4, gd["lo"], gd["hi"], seed + f) for f in range(d + 1)],
            "bc": [I.DIRICHLET] * d + [I.NEUMANN], "roles": {"p": d, "vel": list(range(d))}, "mu": 0.01}


@pytest.mark.parametrize("placement,layers", [("HGC", 1), ("CGC", 1), ("CGC_ES", 1), ("HGC", 2)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_stretched_small_cases(placement, layers, dtype):
    for k, (gd, bd) in enumerate(CASES):
        g = _with_fields(gd, bd, 1700 + 10 * k)
        for mode in ("level", "persistent"):
            run = DeviceRun([g], placement, mode=mode, dtype=dtype, layers=layers)
            compare_structure(run, [g], placement)
            if layers == 1:
                _check_values(run, [g], placement, dtype)
            else:
                from tests.test_gpu_second_layer import _values
                _values(run, [g], placement, dtype, mode)


def test_stretched_forces_and_adjoint():
    geoms = [_with_fields(gd, bd, 1800 + 10 * k) for k, (gd, bd) in enumerate(CASES[:2])]
    # a uniform geometry in the same set
    geoms.append(_with_fields(I.grid(2, [40, 36], [-1.0, -1.0], [1.0, 1.0]), I.ellipse(0.0, 0.02, 0.55, 0.3, 1.1), 1890))
    run = DeviceRun(geoms, "HGC", dtype=torch.float64)
    compare_structure(run, geoms, "HGC")
    arrays = run.field_arrays()
    ft, _ = run.fill(arrays, run.bc_arrays())
    dirs = I.DRAG_LIFT_DIRS_2D
    vel, p, mu = [0, 1], 2, 0.01
    out = run.R.forces([ft[i] for i in vel], ft[p], mu, dirs).cpu().numpy()
    dev = run.R.device
    seed = torch.tensor([[0.7, -1.3]] * len(geoms), dtype=torch.float64, device=dev)
    gf = [torch.zeros(run.R.n_cells, dtype=torch.float64, device=dev) for _ in range(3)]
    gb = [torch.zeros(run.info["cell"].size, dtype=torch.float64, device=dev) for _ in range(3)]
    run.R.adjoint(geoms[0]["bc"], vel, p, mu, dirs, seed, gf, gb)
    run.R.sync_status()
    gf = [t.cpu().numpy() for t in gf]
    gb = [t.cpu().numpy() for t in gb]
    for b, g in enumerate(geoms):
        o0, o1 = run.R.cell_offset[b], run.R.cell_offset[b + 1]
        sel = run.info["geom"] == b
        c = O.classify(g["grid"], g["body"], "HGC")
        lev = O.build_levels(c)
        filled = O.fill(c, lev, [a[o0:o1] for a in arrays], g["bc"], oracle_bcs(g, c, lev))
        ref, scale = O.forces(c, lev, filled[p], [filled[i] for i in vel], mu, dirs)
        assert np.all(np.abs(out[b] - ref) <= 1e-12 * scale + 1e-300), (b, out[b], ref)
        gx, gbo = O.adjoint_gradient(c, lev, g["bc"], p, vel, mu, dirs, (0.7, -1.3))
        for f in range(3):
            sc = max(np.abs(gx[f]).max(), np.abs(gbo[f]).max(), 1e-300)
            assert np.max(np.abs(gf[f][o0:o1] - gx[f])) <= 1e-11 * sc, (b, f)
            assert np.max(np.abs(gb[f][sel] - gbo[f])) <= 1e-11 * sc, (b, f)


def test_stretched_airfoil_1024():
    gd = I.stretched_grid(2, [1024, 512], [-1.0, -1.0], [3.0, 1.0], ratio=(1.003, 1.006), centre_frac=(0.3, 0.5))
    g = _with_fields(gd, I.airfoil(0.0, 0.0, 0.12, 1.0, 5.0), 1900)
    run = DeviceRun([g], "HGC", dtype=torch.float32)
    compare_structure(run, [g], "HGC")
    _check_values(run, [g], "HGC", torch.float32)
