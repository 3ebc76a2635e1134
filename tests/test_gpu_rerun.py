"""A re-run of the classification and the levels on a planned, levelled
context (ebr_classify + ebr_build_levels, and the fused ebr_classify_levels:
the single-pass compactions of the interface cells, the ghosts and the ghost
targets' sources; the closest points beside the levels) gives exactly
what the plan gave: tags, ghost records and levels bitwise, the same source
count, and the adjoint (which walks the source lists in their order) bitwise;
and the re-run's structure matches the oracle.  Every placement, both layer
counts, a batch of uneven 2D grids, a 3D sphere, bodies centred on odd grids
(normal components exactly zero) and stretched grids."""

import numpy as np
import pytest
import torch

from paper_2609_10165_b300 import inputs as I
from tests.parity import DeviceRun, compare_structure

pytestmark = pytest.mark.gpu


def _sphere():
    g = {"grid": I.grid(3, [41, 37, 39], [-1.0, -1.0, -1.0], [1.0, 1.0, 1.0]),
         "body": I.sphere(0.02, -0.01, 0.03, 0.55)}
    g.update({"fields": [I.FourierField(3, 4, g["grid"]["lo"], g["grid"]["hi"], 900 + f) for f in range(4)],
              "bc": [I.DIRICHLET] * 3 + [I.NEUMANN], "roles": {"p": 3, "vel": [0, 1, 2]}, "mu": 0.02})
    return g


def _adjoint(run, geoms):
    d = geoms[0]["grid"]["dim"]
    dirs = I.DRAG_LIFT_DIRS_2D if d == 2 else I.DRAG_LIFT_DIRS_3D
    F = len(geoms[0]["fields"])
    dev = run.R.device
    gf = [torch.zeros(run.R.n_cells, dtype=torch.float32, device=dev) for _ in range(F)]
    gb = [torch.zeros(run.info["cell"].size, dtype=torch.float32, device=dev) for _ in range(F)]
    seed = torch.tensor([[1.0 + 0.1 * b, -0.5 + 0.05 * b] for b in range(len(geoms))], dtype=torch.float64,
                        device=dev)
    w = geoms[0]
    run.R.adjoint(w["bc"], w["roles"]["vel"], w["roles"]["p"], w["mu"], dirs, seed, gf, gb, mode="persistent")
    run.R.sync_status()
    return [t.cpu().numpy() for t in gf + gb]


def _fields(g, seed):
    d = g["grid"]["dim"]
    g.update({"fields": [I.FourierField(d, 4, g["grid"]["lo"], g["grid"]["hi"], seed + f) for f in range(d + 1)],
              "bc": [I.DIRICHLET] * d + [I.NEUMANN], "roles": {"p": d, "vel": list(range(d))}, "mu": 0.01})
    return g


def _axis_aligned():
    # odd grids centred on the bodies: cell centres on the bodies' axes, where
    # normal components are exactly zero (structurally inactive members)
    return [_fields({"grid": I.grid(2, [41, 41], [-1.0, -1.0], [1.0, 1.0]), "body": I.circle(0.0, 0.0, 0.5)}, 960),
            _fields({"grid": I.grid(2, [45, 31], [-1.5, -1.0], [1.5, 1.0]),
                     "body": I.ellipse(0.0, 0.0, 0.83, 0.47, 0.0)}, 970)]


def _stretched():
    from tests.test_oracle_stretched import CASES as SC
    return [_fields({"grid": gd, "body": bd}, 980 + 10 * k) for k, (gd, bd) in enumerate(SC[:2])]


CASES = [("batch", "HGC", 1), ("batch", "CGC", 1), ("batch", "CGC_ES", 1), ("batch", "HGC", 2),
         ("sphere", "HGC", 1), ("sphere", "CGC_ES", 1), ("sphere", "HGC", 2),
         ("axis_aligned", "HGC", 1), ("stretched", "HGC", 1), ("stretched", "CGC_ES", 1)]


@pytest.mark.parametrize("which,placement,layers", CASES)
def test_rerun_equals_plan(which, placement, layers):
    if which == "batch":
        # the smaller grids of the batch (ellipses and airfoils), so that the
        # oracle's structure finishes in seconds
        geoms = [g for g in I.batch(64) if int(np.prod(g["grid"]["n"])) <= 160_000][:12]
    elif which == "axis_aligned":
        geoms = _axis_aligned()
    elif which == "stretched":
        geoms = _stretched()
    else:
        geoms = [_sphere()]
    run = DeviceRun(geoms, placement, dtype=torch.float32, layers=layers)
    tags0 = run.R.tags.clone()
    info0 = run.R.ghost_info()
    n_gsrc0 = run.R.diagnostics()["n_gsrc"]
    adj0 = _adjoint(run, geoms)
    # the two calls, then the fused call (for one-layer HGC the closest
    # points overlap the levels there)
    run.R.classify()
    run.R.build_levels()
    for _ in range(2):
        run.R.classify_levels()
    run.R.sync_status()
    assert torch.equal(run.R.tags, tags0)
    info1 = run.R.ghost_info()
    for k in info0:
        assert np.array_equal(info0[k], info1[k]), k
    assert run.R.diagnostics()["n_gsrc"] == n_gsrc0
    adj1 = _adjoint(run, geoms)
    for a, b in zip(adj0, adj1):
        assert np.array_equal(a, b)
    run.info = info1
    compare_structure(run, geoms, placement)
