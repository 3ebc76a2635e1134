"""The full 256-geometry batch (48M cells) in the launch configuration the
benchmark times: FP32 fields, the persistent fill, the adjoint overlapped on
a second stream, launch shapes chosen by the autotuner, the whole step
captured in a CUDA graph and replayed.

- Structure, every geometry, bit-exact: tags, canonical ghost cells, levels
  and r_i against the oracle (which classifies all 256 geometries in a spawn
  process pool while the GPU works).
- Values, a seeded sample of geometries plus the smallest and the largest:
  filled ghost values, forces and the adjoint gradient against the oracle,
  with the FP32 tolerances of the smaller parity tests.
- Properties, every geometry: finite outputs, non-ghost cells untouched,
  zero gradient at ghost cells, and the graph replay equal bit for bit to a
  serial (non-overlapped) eager step."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2609_10165_b300 import inputs as I
from tests.oracle_pool import batch_structure, start_pool
from tests.parity import GEOM_TOL, NORMAL_TOL, oracle_bcs

pytestmark = pytest.mark.gpu

N_GEOMS = 256
N_SAMPLE = 12
SEED = (1.0, 1.0)          # the benchmark's seed: d(drag + lift)


def _sample(geoms):
    rng = np.random.default_rng(2609)
    sizes = [g["grid"]["n"][0] for g in geoms]
    pick = {int(i) for i in rng.choice(len(geoms), N_SAMPLE, replace=False)}
    pick |= {int(np.argmax(sizes)), int(np.argmin(sizes))}
    return sorted(pick)


def _bench_step_outputs(geoms, dev):
    """Run the benchmark's step as the benchmark runs it; return the device
    results as host arrays and the bitwise-comparable serial results."""
    import bench
    from paper_2609_10165_b300.autotune import autotune

    R, _, host_fields, host_bcs, fields, bcs = bench.setup(geoms, dev, torch.float32)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    step = bench.Step(R, fields, bcs, geoms, "persistent", adjoint=True, overlap=True)
    for _ in range(3):
        step()
    R.sync_status()
    autotune(R, bench.Step(R, fields, bcs, geoms, "persistent", adjoint=True, overlap=False),
             reps=2, flush=flush.zero_)
    R.sync_status()
    del flush
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
            step()
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    R.sync_status()
    out = {
        "tags": R.tags.cpu().numpy(),
        "info": R.ghost_info(),
        "fields": [f.cpu().numpy() for f in fields],
        "forces": step.out.view(R.B, 6).cpu().numpy(),
        "gf": [t.cpu().numpy() for t in step.gf],
        "gb": [t.cpu().numpy() for t in step.gb],
        "offset": R.cell_offset.copy(),
    }
    # one serial eager step (no second stream, no graph) on fresh outputs
    serial = bench.Step(R, fields, bcs, geoms, "persistent", adjoint=True, overlap=False)
    serial()
    torch.cuda.synchronize()
    R.sync_status()
    out["serial"] = {
        "fields": [f.cpu().numpy() for f in fields],
        "forces": serial.out.view(R.B, 6).cpu().numpy(),
        "gf": [t.cpu().numpy() for t in serial.gf],
        "gb": [t.cpu().numpy() for t in serial.gb],
    }
    return out, host_fields, host_bcs


def _check_structure(dev_out, structure):
    tags, info, off = dev_out["tags"], dev_out["info"], dev_out["offset"]
    for gi, tie_free, c_tags, cells, levels, r, psi, nrm, S, h in structure:
        assert tie_free, gi
        o0, o1 = off[gi], off[gi + 1]
        assert np.array_equal(tags[o0:o1], c_tags), (gi, int(np.sum(tags[o0:o1] != c_tags)))
        sel = info["geom"] == gi
        assert np.array_equal(info["cell"][sel], cells), gi
        assert np.array_equal(info["level"][sel], levels), gi
        assert np.array_equal(info["r"][sel][:, :2], r), gi
        # the GPU's closest points against the oracle's own
        assert np.max(np.abs(info["psi"][sel] - psi), initial=0.0) <= GEOM_TOL * h, gi
        assert np.max(np.abs(info["S"][sel][:, :2] - S), initial=0.0) <= GEOM_TOL * h, gi
        assert np.max(np.abs(info["normal"][sel][:, :2] - nrm), initial=0.0) <= NORMAL_TOL, gi


def _check_properties(dev_out, host_fields, n_geoms):
    info, off = dev_out["info"], dev_out["offset"]
    ghost = np.zeros(int(off[-1]), bool)
    ghost[off[info["geom"]] + info["cell"]] = True
    assert int(ghost.sum()) == info["cell"].size         # one ghost per cell at most
    assert np.array_equal(np.unique(info["geom"]), np.arange(n_geoms))
    for f, a in enumerate(dev_out["fields"]):
        assert np.all(np.isfinite(a[ghost])), f
        assert np.array_equal(a[~ghost], host_fields[f][~ghost]), f
    for f in range(len(dev_out["gf"])):
        assert np.all(np.isfinite(dev_out["gf"][f])) and np.all(np.isfinite(dev_out["gb"][f])), f
        assert np.all(dev_out["gf"][f][ghost] == 0), f
    assert np.all(np.isfinite(dev_out["forces"]))
    s = dev_out["serial"]
    for key in ("fields", "gf", "gb"):
        for f, (x, y) in enumerate(zip(dev_out[key], s[key])):
            assert np.array_equal(x, y), (key, f)
    assert np.array_equal(dev_out["forces"], s["forces"])


def _check_sample(dev_out, geoms, host_fields, host_bcs, sample):
    info, off = dev_out["info"], dev_out["offset"]
    dirs = I.DRAG_LIFT_DIRS_2D
    for gi in sample:
        g = geoms[gi]
        o0, o1 = off[gi], off[gi + 1]
        sel = info["geom"] == gi
        # the oracle on the uploaded FP32 field values, with FP32-rounded
        # boundary data evaluated at its own S
        arrays = [np.asarray(a[o0:o1], dtype=np.float64) for a in host_fields]
        c = O.classify(g["grid"], g["body"], "HGC")
        lev = O.build_levels(c)
        filled = O.fill(c, lev, arrays, g["bc"], oracle_bcs(g, c, lev, f32=True))
        cells = c.idx[lev.order]
        for f in range(3):
            got = dev_out["fields"][f][o0:o1][cells]
            tol = 1e-5 * np.abs(arrays[f]).max()
            assert np.max(np.abs(got - filled[f][cells])) <= tol, (gi, f)
        vel = [filled[i] for i in g["roles"]["vel"]]
        ref, scale = O.forces(c, lev, filled[g["roles"]["p"]], vel, g["mu"], dirs)
        got = dev_out["forces"][gi]
        assert np.all(np.abs(got - ref) <= 1e-4 * scale), (gi, got, ref, scale)
        gx, gbo = O.adjoint_gradient(c, lev, g["bc"], g["roles"]["p"], g["roles"]["vel"], g["mu"], dirs, SEED)
        for f in range(3):
            sc = max(np.abs(gx[f]).max(), np.abs(gbo[f]).max(), 1e-300)
            assert np.max(np.abs(dev_out["gf"][f][o0:o1] - gx[f])) <= 2e-5 * sc, (gi, f)
            assert np.max(np.abs(dev_out["gb"][f][sel] - gbo[f])) <= 2e-5 * sc, (gi, f)


def test_full_batch_in_the_benchmark_configuration():
    geoms = I.batch(N_GEOMS)
    dev = torch.device("cuda", torch.cuda.current_device())
    with start_pool(N_GEOMS) as pool:
        pending = pool.map_async(batch_structure, [(N_GEOMS, gi, "HGC") for gi in range(N_GEOMS)])
        dev_out, host_fields, host_bcs = _bench_step_outputs(geoms, dev)
        _check_properties(dev_out, host_fields, N_GEOMS)
        _check_sample(dev_out, geoms, host_fields, host_bcs, _sample(geoms))
        structure = pending.get(timeout=1800)
    _check_structure(dev_out, structure)
