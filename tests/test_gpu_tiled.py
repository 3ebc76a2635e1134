"""GPU parity of the tiled fill with a per-level exchange (Sec. 3.2,
distributed memory) against the oracle's tiled schedule and fill.

- Schedule, bit-exact: the tile of every ghost, the ghosts sent after each
  level (those another tile's stencil reads), the number of (ghost,
  receiving tile) pairs and the conventional halo volume.
- Values: the tiled launch gives the same bits as the level-launch fill (same
  closed forms and summation order) and matches the oracle's tiled fill at
  the parity tolerances, on small ragged cases, a batch, the 2048x1024
  airfoil and the 512^3 sphere.
- The bounded barrier: a launch told to wait for an arrival that never comes
  reports EBR_ETIMEOUT and leaves the context usable."""

import numpy as np
import pytest
import torch

import oracle as O
from oracle.tiles import halo_exchange_volume, tile_ids, tile_plan
from paper_2609_10165_b300 import inputs as I
from tests.parity import DeviceRun, compare_structure, oracle_bcs, U32
from tests.test_gpu_parity import _small_cases, _with_fields

pytestmark = pytest.mark.gpu


def _check_schedule(run, geoms, placement, tile):
    R = run.R
    R.tiled_plan(tile)
    tl, slot = R.tiled_lists()
    info = R.tiled_info()
    pairs = halo = 0
    toff = 0
    for b, g in enumerate(geoms):
        c = O.classify(g["grid"], g["body"], placement)
        lev = O.build_levels(c)
        plan = tile_plan(c, lev, tile)
        sel = run.info["geom"] == b
        assert np.array_equal(tl[sel], toff + plan.tile_of), (b, tile)
        sent = np.zeros(c.n_ghosts, bool)
        for qs in plan.sends:
            sent[qs] = True
        assert np.array_equal(slot[sel] >= 0, sent), (b, tile)
        pairs += plan.values_exchanged()
        halo += halo_exchange_volume(c, lev, tile)
        d = g["grid"]["dim"]
        toff += int(np.prod([(g["grid"]["n"][a] + tile[a] - 1) // tile[a] for a in range(d)]))
    assert info["values_exchanged"] == pairs and info["halo_values"] == halo, (info, pairs, halo)
    assert info["tiles"] == toff
    assert sum(info["sent_per_level"]) == info["sent_ghosts"] == int(np.sum(slot >= 0))
    return info


def _tiled_vs_level(run, arrays, bcs, kinds, dtype):
    dev = run.R.device
    ft = [torch.tensor(a, dtype=dtype, device=dev) for a in arrays]
    fl = [t.clone() for t in ft]
    bt = [torch.tensor(b, dtype=dtype, device=dev) for b in bcs]
    run.R.reconstruct_tiled(ft, kinds, bt)
    run.R.reconstruct(fl, kinds, bt, mode="level")
    run.R.sync_status()
    for a, b in zip(ft, fl):
        assert torch.equal(a, b)
    return [t.double().cpu().numpy() for t in ft]


def _check_against_oracle(run, geoms, placement, got, arrays, dtype):
    f32 = dtype == torch.float32
    for b, g in enumerate(geoms):
        o0, o1 = run.R.cell_offset[b], run.R.cell_offset[b + 1]
        c = O.classify(g["grid"], g["body"], placement)
        lev = O.build_levels(c)
        loc = [a[o0:o1] for a in arrays]
        out, _ = O.tiles.tiled_fill(c, lev, loc, g["bc"], oracle_bcs(g, c, lev, f32), run.tile)
        cells = c.idx[lev.order]
        for f in range(len(g["fields"])):
            diff = np.abs(got[f][o0:o1][cells] - out[f][cells])
            scale = np.abs(loc[f]).max()
            tol = 1e-5 * scale if f32 else 1e-11 * max(scale, 1.0)
            assert diff.max(initial=0.0) <= tol, (b, f, float(diff.max()))


@pytest.mark.parametrize("placement", ["HGC", "CGC_ES"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_tiled_small_cases(placement, dtype):
    for k, case in enumerate(_small_cases()):
        g = _with_fields(case, 1200 + 10 * k)
        d = g["grid"]["dim"]
        run = DeviceRun([g], placement, dtype=dtype)
        compare_structure(run, [g], placement)
        arrays = run.field_arrays()
        if dtype == torch.float32:
            arrays = [a.astype(np.float32).astype(np.float64) for a in arrays]
        bcs = run.bc_arrays()
        if dtype == torch.float32:
            bcs = [b.astype(np.float32).astype(np.float64) for b in bcs]
        for tile in ([4] * d, [7, 5, 6][:d], [3] * d):
            _check_schedule(run, [g], placement, tile)
            run.tile = tile
            got = _tiled_vs_level(run, arrays, bcs, g["bc"], dtype)
            _check_against_oracle(run, [g], placement, got, arrays, dtype)


def test_tiled_batch_of_geometries():
    geoms = [_with_fields(c, 1300 + 10 * k) for k, c in enumerate(_small_cases()) if c["grid"]["dim"] == 2]
    geoms += I.batch()[:6]
    for g in geoms[3:]:
        g["fields"] = g["fields"][:3]
    run = DeviceRun(geoms, "HGC", dtype=torch.float64)
    tile = [16, 16]
    _check_schedule(run, geoms, "HGC", tile)
    run.tile = tile
    arrays = run.field_arrays()
    got = _tiled_vs_level(run, arrays, run.bc_arrays(), geoms[0]["bc"], torch.float64)
    _check_against_oracle(run, geoms, "HGC", got, arrays, torch.float64)


@pytest.mark.parametrize("name,tile", [("airfoil_2048", [64, 64]), ("sphere_512", [32, 32, 32])])
def test_tiled_full_size(name, tile):
    w = I.WORKLOADS[name]()
    run = DeviceRun([w], "HGC", dtype=torch.float32)
    info = _check_schedule(run, [w], "HGC", tile)
    run.tile = tile
    arrays = [a.astype(np.float32).astype(np.float64) for a in run.field_arrays()]
    bcs = [b.astype(np.float32).astype(np.float64) for b in run.bc_arrays()]
    got = _tiled_vs_level(run, arrays, bcs, w["bc"], torch.float32)
    # the oracle's global fill (the tiled one equals it bit for bit, pinned on
    # the CPU) at the FP32 tolerance
    c = O.classify(w["grid"], w["body"], "HGC")
    lev = O.build_levels(c)
    ref = O.fill(c, lev, arrays, w["bc"], oracle_bcs(w, c, lev, True))
    cells = c.idx[lev.order]
    for f in range(len(arrays)):
        assert np.max(np.abs(got[f][cells] - ref[f][cells])) <= 1e-5 * np.abs(arrays[f]).max(), f
    assert info["values_exchanged"] < info["halo_values"]


def test_tiled_barrier_timeout_is_reported():
    from paper_2609_10165_b300._lib import EBRError
    g = _with_fields(_small_cases()[1], 1400)          # the airfoil: several levels
    run = DeviceRun([g], "HGC", dtype=torch.float64)
    run.R.tiled_plan([8, 8])
    arrays = run.field_arrays()
    bcs = run.bc_arrays()
    dev = run.R.device
    ft = [torch.tensor(a, device=dev) for a in arrays]
    bt = [torch.tensor(b, device=dev) for b in bcs]
    run.R.tiled_wait_test(2000)
    with pytest.raises(EBRError) as ei:
        run.R.reconstruct_tiled(ft, g["bc"], bt)
        run.R.sync_status()
    assert ei.value.name == "EBR_ETIMEOUT"
    # the context is usable: the next launch completes and is right
    ft = [torch.tensor(a, device=dev) for a in arrays]
    fl = [t.clone() for t in ft]
    run.R.reconstruct_tiled(ft, g["bc"], bt)
    run.R.reconstruct(fl, g["bc"], bt, mode="level")
    run.R.sync_status()
    for a, b in zip(ft, fl):
        assert torch.equal(a, b)
