"""Launch shapes on the GPU: every tunable kernel must give bitwise the same
tags, ghost records, levels, filled fields, forces and adjoint gradients at
every allowed block size (the block size changes scheduling only); bad
names and sizes are rejected; the autotuner leaves every kernel at one of
its candidates and the results unchanged."""

import numpy as np
import pytest
import torch

from paper_2609_10165_b300 import inputs as I
from paper_2609_10165_b300.api import Reconstructor
from paper_2609_10165_b300.autotune import autotune

pytestmark = pytest.mark.gpu

N_GEOMS = 6


def _setup():
    geoms = I.batch(N_GEOMS, nmax=320)
    R = Reconstructor([g["grid"] for g in geoms], [g["body"] for g in geoms], "HGC")
    R.build_levels()
    R.sync_status()
    info = R.ghost_info()
    fields = [torch.tensor(np.concatenate([g["fields"][f].on_grid(g["grid"], np.float32) for g in geoms]),
                           device=R.device) for f in range(3)]
    bcs = []
    for f in range(3):
        v = np.zeros(info["cell"].size)
        for b, g in enumerate(geoms):
            sel = info["geom"] == b
            v[sel] = I.bc_values(g["fields"][f], g["bc"][f], info["S"][sel, :2], info["normal"][sel, :2])
        bcs.append(torch.tensor(v, dtype=torch.float32, device=R.device))
    return R, geoms, fields, bcs


def _step(R, geoms, fields0, bcs):
    """classify + levels + fill + forces + adjoint; every result as host arrays."""
    g0 = geoms[0]
    fields = [f.clone() for f in fields0]
    R.classify()
    R.build_levels()
    R.reconstruct(fields, g0["bc"], bcs)
    out = torch.empty(R.B * 6, dtype=torch.float64, device=R.device)
    R.forces([fields[i] for i in g0["roles"]["vel"]], fields[g0["roles"]["p"]], g0["mu"], I.DRAG_LIFT_DIRS_2D,
             out=out)
    seed = torch.ones(R.B, 2, dtype=torch.float64, device=R.device)
    gf = [torch.zeros_like(f) for f in fields]
    gb = [torch.zeros_like(b) for b in bcs]
    R.adjoint(g0["bc"], g0["roles"]["vel"], g0["roles"]["p"], g0["mu"], I.DRAG_LIFT_DIRS_2D, seed, gf, gb)
    R.sync_status()
    info = R.ghost_info()
    res = [R.tags.cpu().numpy(), out.cpu().numpy()]
    res += [info[k] for k in ("geom", "cell", "level", "psi", "normal", "r")]
    res += [t.cpu().numpy() for t in fields + gf + gb]
    return res


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and x.shape == y.shape
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))


def test_results_bitwise_equal_at_every_block_size():
    R, geoms, fields, bcs = _setup()
    ref = _step(R, geoms, fields, bcs)
    names = R.tunable_kernels()
    assert len(names) == 12 and all(R.block_size(n) == 128 for n in names)
    for T in (32, 64, 96, 256):
        for n in names:
            R.set_block_size(n, T)
        _same(_step(R, geoms, fields, bcs), ref)


def test_bad_names_and_sizes_are_rejected():
    R, geoms, fields, bcs = _setup()
    with pytest.raises(Exception):
        R.set_block_size("no_such_kernel", 128)
    for bad in (0, 16, 48, 288, 512, 1024):
        with pytest.raises(Exception):
            R.set_block_size("tables", bad)
        assert R.block_size("tables") == 128
    with pytest.raises(ValueError):
        R.block_size("no_such_kernel")


def test_autotune_picks_candidates_and_keeps_results(tmp_path):
    R, geoms, fields, bcs = _setup()
    ref = _step(R, geoms, fields, bcs)
    cands = (64, 128, 256)
    shapes, rep = autotune(R, lambda: _step(R, geoms, fields, bcs), candidates=cands, reps=2,
                           cache_path=str(tmp_path / "shapes.json"), key="test")
    assert rep["source"] == "search"
    assert set(shapes) == set(R.tunable_kernels())
    for n, t in shapes.items():
        assert t in cands and R.block_size(n) == t
    _same(_step(R, geoms, fields, bcs), ref)
    R2, _, _, _ = _setup()
    shapes2, rep2 = autotune(R2, lambda: None, cache_path=str(tmp_path / "shapes.json"), key="test")
    assert rep2["source"] == "cache" and shapes2 == shapes
