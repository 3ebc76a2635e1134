"""Adjoint on the GPU: against the oracle's explicit-matrix gradient, against
central finite differences of the GPU forward path (h = 1e-6 in FP64; the map
is linear, so FD is exact up to rounding), through torch.autograd, and for
bitwise reproducibility."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2609_10165_b300 import inputs as I
from tests.parity import DeviceRun, compare_structure, note_worst

pytestmark = pytest.mark.gpu


def _case(kind):
    if kind == "ellipse":
        g = {"grid": I.grid(2, [45, 39], [-1.0, -1.0], [1.0, 1.0]), "body": I.ellipse(0.03, -0.02, 0.6, 0.35, 0.7)}
    elif kind == "airfoil":
        # 151 columns: with 150 a cell centre would sit exactly on the leading edge (a tie)
        g = {"grid": I.grid(2, [151, 71], [-1.0, -1.0], [3.0, 1.0]), "body": I.airfoil(0.0, 0.0, 0.14, 1.0, 6.0)}
    elif kind == "sphere":
        g = {"grid": I.grid(3, [23, 21, 22], [-1.0, -1.0, -1.0], [1.0, 1.0, 1.0]), "body": I.sphere(0.02, -0.01, 0.03, 0.6)}
    d = g["grid"]["dim"]
    g.update({"fields": [I.FourierField(d, 4, g["grid"]["lo"], g["grid"]["hi"], 700 + f) for f in range(d + 1)],
              "bc": [I.DIRICHLET] * d + [I.NEUMANN], "roles": {"p": d, "vel": list(range(d))}, "mu": 0.02})
    return g


def _gpu_grad(run, w, seed, dtype, mode):
    d = w["grid"]["dim"]
    dirs = I.DRAG_LIFT_DIRS_2D if d == 2 else I.DRAG_LIFT_DIRS_3D
    F = len(w["fields"])
    dev = run.R.device
    gf = [torch.zeros(run.R.n_cells, dtype=dtype, device=dev) for _ in range(F)]
    gb = [torch.zeros(run.info["cell"].size, dtype=dtype, device=dev) for _ in range(F)]
    s = torch.tensor([seed], dtype=torch.float64, device=dev)
    run.R.adjoint(w["bc"], w["roles"]["vel"], w["roles"]["p"], w["mu"], dirs, s, gf, gb, mode=mode)
    run.R.sync_status()
    return [t.double().cpu().numpy() for t in gf], [t.double().cpu().numpy() for t in gb]


@pytest.mark.parametrize("kind", ["ellipse", "airfoil", "sphere"])
@pytest.mark.parametrize("placement", ["HGC", "CGC", "CGC_ES"])
@pytest.mark.parametrize("mode", ["level", "persistent"])
def test_adjoint_matches_oracle(kind, placement, mode):
    # HGC and CGC stencils reach 1 cell (the fluid targets' two-pass probe +
    # pull); the CGC_ES cases here reach r = 2 (the one-pass kernel): both
    # paths of the fluid-target gradient are compared with the oracle
    w = _case(kind)
    run = DeviceRun([w], placement)
    seed = (0.7, -1.3)
    d = w["grid"]["dim"]
    dirs = I.DRAG_LIFT_DIRS_2D if d == 2 else I.DRAG_LIFT_DIRS_3D
    c = O.classify(w["grid"], w["body"], placement)
    assert c.ties == []
    lev = O.build_levels(c)
    gx, gbo = O.adjoint_gradient(c, lev, w["bc"], w["roles"]["p"], w["roles"]["vel"], w["mu"], dirs, seed)
    for dtype, rtol in ((torch.float64, 1e-11), (torch.float32, 2e-5)):
        gf, gb = _gpu_grad(run, w, seed, dtype, mode)
        for f in range(len(w["fields"])):
            sc = max(np.abs(gx[f]).max(), np.abs(gbo[f]).max(), 1e-300)
            assert np.max(np.abs(gf[f] - gx[f])) <= rtol * sc, (dtype, f, np.max(np.abs(gf[f] - gx[f])) / sc)
            assert np.max(np.abs(gb[f] - gbo[f])) <= rtol * sc, (dtype, f)


@pytest.mark.parametrize("name", ["cylinder_1024", "sphere_256"])
def test_adjoint_full_size_matches_oracle(name):
    # the adjoint configurations at their full sizes (1024^2 cylinder, 256^3
    # sphere), FP64 and FP32 fields with FP64 coefficients, against the
    # oracle's explicit-matrix gradient
    w = I.WORKLOADS[name]()
    run = DeviceRun([w], "HGC")
    res = compare_structure(run, [w], "HGC")
    c, lev = res[0]
    d = w["grid"]["dim"]
    dirs = I.DRAG_LIFT_DIRS_2D if d == 2 else I.DRAG_LIFT_DIRS_3D
    seed = (1.0, 0.5)
    gx, gbo = O.adjoint_gradient(c, lev, w["bc"], w["roles"]["p"], w["roles"]["vel"], w["mu"], dirs, seed)
    for dtype, rtol in ((torch.float64, 1e-11), (torch.float32, 2e-5)):
        gf, gb = _gpu_grad(run, w, seed, dtype, "persistent")
        for f in range(len(w["fields"])):
            sc = max(np.abs(gx[f]).max(), np.abs(gbo[f]).max(), 1e-300)
            e = max(np.max(np.abs(gf[f] - gx[f])), np.max(np.abs(gb[f] - gbo[f]))) / sc
            assert e <= rtol, (name, dtype, f, e)
            note_worst("adjoint %s %s" % ("FP64" if dtype == torch.float64 else "FP32", name), e / rtol, e)


def _J_gpu(run, w, arrays, bcs, seed):
    ft, _ = run.fill(arrays, bcs)
    d = w["grid"]["dim"]
    dirs = I.DRAG_LIFT_DIRS_2D if d == 2 else I.DRAG_LIFT_DIRS_3D
    vel = [None if i is None else ft[i] for i in w["roles"]["vel"]]
    out = run.R.forces(vel, ft[w["roles"]["p"]], w["mu"], dirs).cpu().numpy()[0]
    return seed[0] * out[2 * d] + seed[1] * out[2 * d + 1]


@pytest.mark.parametrize("name", ["cylinder_1024", "sphere_256", "airfoil"])
def test_adjoint_finite_differences(name):
    if name == "airfoil":
        w = _case("airfoil")
    else:
        w = I.WORKLOADS[name]()
    run = DeviceRun([w], "HGC", dtype=torch.float64)
    seed = (1.0, 0.5)
    rng = np.random.default_rng(5)
    arrays = run.field_arrays()
    bcs = run.bc_arrays()
    g64, gb64 = _gpu_grad(run, w, seed, torch.float64, "persistent")
    g32, gb32 = _gpu_grad(run, w, seed, torch.float32, "persistent")
    for _ in range(2):
        vx = [rng.normal(size=a.size) for a in arrays]
        vb = [rng.normal(size=b.size) for b in bcs]
        h = 1e-6
        jp = _J_gpu(run, w, [a + h * v for a, v in zip(arrays, vx)], [b + h * v for b, v in zip(bcs, vb)], seed)
        jm = _J_gpu(run, w, [a - h * v for a, v in zip(arrays, vx)], [b - h * v for b, v in zip(bcs, vb)], seed)
        fd = (jp - jm) / (2 * h)
        for gx, gb, tol in ((g64, gb64, 1e-7), (g32, gb32, 1e-4)):
            an = sum(float(g @ v) for g, v in zip(gx, vx)) + sum(float(g @ v) for g, v in zip(gb, vb))
            scale = sum(float(np.abs(g) @ np.abs(v)) for g, v in zip(gx, vx)) + \
                sum(float(np.abs(g) @ np.abs(v)) for g, v in zip(gb, vb))
            assert abs(fd - an) <= tol * scale, (name, fd, an, scale)


def test_autograd_function():
    w = _case("ellipse")
    run = DeviceRun([w], "HGC", dtype=torch.float64)
    dev = run.R.device
    arrays = run.field_arrays()
    bcs = run.bc_arrays()
    ft = [torch.tensor(a, device=dev, requires_grad=True) for a in arrays]
    bt = [torch.tensor(b, device=dev, requires_grad=True) for b in bcs]
    dl = run.R.drag_lift(ft, bt, w["bc"], w["roles"]["vel"], w["roles"]["p"], w["mu"], I.DRAG_LIFT_DIRS_2D)
    J = 0.3 * dl[0, 0] - 0.9 * dl[0, 1]
    J.backward()
    gf, gb = _gpu_grad(run, w, (0.3, -0.9), torch.float64, "persistent")
    for f in range(len(ft)):
        assert np.allclose(ft[f].grad.cpu().numpy(), gf[f], rtol=0, atol=1e-14 * max(1, np.abs(gf[f]).max()))
        assert np.allclose(bt[f].grad.cpu().numpy(), gb[f], rtol=0, atol=1e-14 * max(1, np.abs(gb[f]).max()))
    # the inputs were not modified (out-of-place forward)
    assert np.array_equal(ft[0].detach().cpu().numpy(), arrays[0])


def test_adjoint_bitwise_reproducible():
    w = _case("airfoil")
    run = DeviceRun([w], "HGC")
    for dtype in (torch.float32, torch.float64):
        a = _gpu_grad(run, w, (1.0, 1.0), dtype, "persistent")
        b = _gpu_grad(run, w, (1.0, 1.0), dtype, "persistent")
        for x, y in zip(a[0] + a[1], b[0] + b[1]):
            assert np.array_equal(x, y)
