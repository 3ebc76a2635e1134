"""GPU parity of the second ghost layer (Sec. 7, psi <= 1.5 dn, multipliers
of Eq. stencil_anisotropic) against the oracle: tags, ghost lists, levels and
r_i bit-exact, psi / n / S against the oracle's closest points, ghost values
(FP64 within 1e-12 of their terms, FP32 within 1e-5 of the field maximum)
through both layers, forces and the adjoint gradient; on small ragged cases
of every body kind, a batch, the 2048x1024 airfoil and the 256^3 sphere."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2609_10165_b300 import inputs as I
from tests.parity import DeviceRun, compare_structure, oracle_bcs, term_magnitude, note_worst
from tests.test_gpu_parity import _small_cases, _with_fields

pytestmark = pytest.mark.gpu


def _values(run, geoms, placement, dtype, mode):
    f32 = dtype == torch.float32
    run.dtype, run.mode = dtype, mode
    arrays = run.field_arrays()
    bcs = run.bc_arrays()
    if f32:
        arrays = [a.astype(np.float32).astype(np.float64) for a in arrays]
        bcs = [b.astype(np.float32).astype(np.float64) for b in bcs]
    ft, _ = run.fill(arrays, bcs)
    got = [t.double().cpu().numpy() for t in ft]
    for b, g in enumerate(geoms):
        o0, o1 = run.R.cell_offset[b], run.R.cell_offset[b + 1]
        c = O.classify(g["grid"], g["body"], placement, layers=2)
        lev = O.build_levels(c)
        loc = [a[o0:o1] for a in arrays]
        bl = oracle_bcs(g, c, lev, f32)
        out = O.fill(c, lev, loc, g["bc"], bl)
        cells = c.idx[lev.order]
        T = term_magnitude(c, lev, loc, bl, g["bc"]) if not f32 else None
        for f in range(len(g["fields"])):
            diff = np.abs(got[f][o0:o1][cells] - out[f][cells])
            tol = 1e-5 * np.abs(loc[f]).max() if f32 else 1e-12 * T[f]
            assert np.all(diff <= tol), (b, f, float(diff.max()))
            note_worst("values %s two layers" % ("FP32" if f32 else "FP64"),
                       float(np.max(diff / np.maximum(tol, 1e-300))), float(diff.max()))
            mask = np.ones(o1 - o0, bool)
            mask[cells] = False
            assert np.array_equal(got[f][o0:o1][mask], loc[f][mask])
    return ft, arrays


@pytest.mark.parametrize("placement", ["HGC", "CGC_ES"])
def test_second_layer_small_cases(placement):
    for k, case in enumerate(_small_cases()):
        g = _with_fields(case, 1500 + 10 * k)
        run = DeviceRun([g], placement, layers=2)
        res = compare_structure(run, [g], placement)
        c, lev = res[0]
        c1 = O.classify(g["grid"], g["body"], placement)
        assert c.n_ghosts > c1.n_ghosts            # the second layer is present
        for dtype in (torch.float64, torch.float32):
            for mode in ("level", "persistent"):
                _values(run, [g], placement, dtype, mode)


def test_second_layer_batch_forces_and_adjoint():
    geoms = I.batch()[:8]
    run = DeviceRun(geoms, "HGC", layers=2)
    compare_structure(run, geoms, "HGC")
    ft, arrays = _values(run, geoms, "HGC", torch.float64, "persistent")
    dirs = I.DRAG_LIFT_DIRS_2D
    vel, p, mu = geoms[0]["roles"]["vel"], geoms[0]["roles"]["p"], geoms[0]["mu"]
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
        c = O.classify(g["grid"], g["body"], "HGC", layers=2)
        lev = O.build_levels(c)
        filled = O.fill(c, lev, [a[o0:o1] for a in arrays], g["bc"], oracle_bcs(g, c, lev))
        ref, scale = O.forces(c, lev, filled[p], [filled[i] for i in vel], mu, dirs)
        assert np.all(np.abs(out[b] - ref) <= 1e-12 * scale + 1e-300), (b, out[b], ref)
        gx, gbo = O.adjoint_gradient(c, lev, g["bc"], p, vel, mu, dirs, (0.7, -1.3))
        for f in range(3):
            sc = max(np.abs(gx[f]).max(), np.abs(gbo[f]).max(), 1e-300)
            assert np.max(np.abs(gf[f][o0:o1] - gx[f])) <= 1e-11 * sc, (b, f)
            assert np.max(np.abs(gb[f][sel] - gbo[f])) <= 1e-11 * sc, (b, f)


@pytest.mark.parametrize("name", ["airfoil_2048", "sphere_256"])
def test_second_layer_full_size(name):
    w = I.WORKLOADS[name]()
    run = DeviceRun([w], "HGC", layers=2, dtype=torch.float32)
    compare_structure(run, [w], "HGC")
    _values(run, [w], "HGC", torch.float32, "persistent")
