"""Benchmark: ghost-cell updates/s of the batched FP32 (FP64-coefficient)
direct reconstruction, forward + adjoint, on the 256-geometry batch.

One step = the whole hot path over the batch: classify + place ghosts,
dependency levels, level-by-level fill of 3 fields, boundary forces
(drag / lift), and the adjoint of fill + forces.  One update = one
(ghost, field) value (forward value plus its adjoint contribution).

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl mine|reference]

Prints one JSON line (rank 0).  Inputs are synthetic (seeded ellipses and
4-digit airfoils, manufactured Fourier fields); the L2 cache is flushed
between timed steps.  Under torchrun every rank runs its own batch (weak
scaling: the geometries of a 256 x N batch are partitioned over the
ranks by estimated work, no collective on the data path).
"""

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "batch_256"
METRIC = "ghost-cell updates/s (fwd+adjoint), batched FP32 with FP64 coefficients"
UNIT = "updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--geoms", type=int, default=256)
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--sets", type=int, default=64,
                    help="field sets of the throughput mode (0: skip); 64 sets move about 6x L2 per step")
    ap.add_argument("--no-single-grid", dest="single_grid", action="store_false",
                    help="skip the 512^3 single-grid tiled fill")
    ap.add_argument("--lite", action="store_true",
                    help="headline step only (no plain FP64 path, no e2e, no CPU baseline), for profilers")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def measured_sm_mhz():
    """Maximum SM clock recorded beside the measured peaks (2032 MHz on B300
    when the file is absent)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if d.get("sm_max_mhz"):
            return float(d["sm_max_mhz"])
    return 2032.0


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------

def make_batch(n_geoms):
    from paper_2609_10165_b300 import inputs as I
    return I.batch(n_geoms)


def rank_batch(n_geoms, rank, world):
    """This rank's geometries: the seeded batch of n_geoms x world geometries
    partitioned over the ranks by estimated work (ghosts x fields), so that
    every rank holds n_geoms distinct geometries (weak scaling); one rank
    gets the whole n_geoms batch.  Returns (geometries, shard summary)."""
    from paper_2609_10165_b300 import shard
    geoms_all = make_batch(n_geoms * world)
    if world == 1:
        return geoms_all, None
    shards, load = shard.partition(geoms_all, world)
    mine = shards[rank]
    return [geoms_all[i] for i in mine], {
        "geometries_all_ranks": len(geoms_all), "geometries_this_rank": len(mine),
        "estimated_work_per_rank": [round(v) for v in load],
        "imbalance": max(load) / (sum(load) / len(load)) - 1.0}


def setup(geoms, device, dtype):
    import torch
    from paper_2609_10165_b300 import inputs as I
    from paper_2609_10165_b300.api import Reconstructor

    R = Reconstructor([g["grid"] for g in geoms], [g["body"] for g in geoms], "HGC", device=device)
    R.build_levels()
    R.sync_status()
    info = R.ghost_info()
    F = 3
    host_fields = []
    for f in range(F):
        host_fields.append(np.concatenate([g["fields"][f].on_grid(g["grid"], np.float32 if dtype == torch.float32 else np.float64)
                                           for g in geoms]))
    bcs = []
    for f in range(F):
        v = np.zeros(info["cell"].size)
        for b, g in enumerate(geoms):
            sel = info["geom"] == b
            v[sel] = I.bc_values(g["fields"][f], g["bc"][f], info["S"][sel, :2], info["normal"][sel, :2])
        bcs.append(v)
    fields = [torch.tensor(a, dtype=dtype, device=device) for a in host_fields]
    bct = [torch.tensor(b, dtype=dtype, device=device) for b in bcs]
    return R, info, host_fields, bcs, fields, bct


class Step:
    """The timed hot path on resident device buffers.

    With `overlap`, the adjoint (which needs the coefficients but not the
    filled values: the path is linear) runs on a second stream beside the
    fill and the forces, joined at the end of the step."""

    def __init__(self, R, fields, bcs, geoms, mode, adjoint=True, overlap=False, geometry=True):
        import torch
        self.R, self.fields, self.bcs, self.mode, self.adjoint = R, fields, bcs, mode, adjoint
        self.geometry = geometry     # False: a stationary body, classified and levelled once
        self.kinds = geoms[0]["bc"]
        self.vel = geoms[0]["roles"]["vel"]
        self.p = geoms[0]["roles"]["p"]
        self.mu = geoms[0]["mu"]
        from paper_2609_10165_b300 import inputs as I
        self.dirs = I.DRAG_LIFT_DIRS_2D
        dev = R.device
        self.out = torch.empty(R.B * 6, dtype=torch.float64, device=dev)
        self.seed = torch.ones(R.B, 2, dtype=torch.float64, device=dev)
        self.gf = [torch.zeros_like(f) for f in fields]
        self.gb = [torch.zeros_like(b) for b in bcs]
        self.side = torch.cuda.Stream(dev) if (overlap and adjoint) else None

    def _adjoint(self):
        self.R.adjoint(self.kinds, self.vel, self.p, self.mu, self.dirs, self.seed, self.gf, self.gb,
                       mode=self.mode)

    def __call__(self):
        import torch
        R = self.R
        if self.geometry:
            R.classify_levels()
        if self.side is not None:
            main = torch.cuda.current_stream()
            self.side.wait_stream(main)
            with torch.cuda.stream(self.side):
                self._adjoint()
        R.reconstruct(self.fields, self.kinds, self.bcs, mode=self.mode)
        R.forces([None if i is None else self.fields[i] for i in self.vel], self.fields[self.p], self.mu,
                 self.dirs, out=self.out)
        if self.side is not None:
            torch.cuda.current_stream().wait_stream(self.side)
        elif self.adjoint:
            self._adjoint()


def reduce_over_ranks(ms, updates, device):
    """Whole-job numbers under torchrun: the slowest rank's step time and the
    updates of all ranks (every rank runs its own batch; this is the only
    cross-rank communication).  A single process returns its own numbers."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, updates
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([updates], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def count_graph_kernels(g):
    """Kernel nodes of a captured CUDA graph (all of them are this library's:
    the step issues no other kernels).  None if the runtime bindings are missing."""
    try:
        from cuda.bindings import runtime as cr
        h = cr.cudaGraph_t(init_value=g.raw_cuda_graph())
        err, _, n = cr.cudaGraphGetNodes(h, 0)
        err, nodes, n = cr.cudaGraphGetNodes(h, n)
        kinds = [cr.cudaGraphNodeGetType(x)[1] for x in nodes[:n]]
        return sum(1 for k in kinds if k == cr.cudaGraphNodeType.cudaGraphNodeTypeKernel)
    except Exception as e:  # reported in the JSON line, not hidden
        return "unavailable: %s" % (str(e)[:80],)


def time_steps(fn, steps, stream, flush):
    """Per-step device time with CUDA events on the launching stream, the L2
    cache flushed (untimed) before every step.  Returns list of ms."""
    import torch
    ts = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ts.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ts]


def _oracle_geometry(g, keep=False):
    """The oracle's whole path on one geometry; seconds per phase and the
    updates (ghosts x 3 fields) it produced (and, with keep, its results:
    canonical ghost cells, ghost values, forces with their term magnitudes,
    gradients)."""
    import oracle as O
    from paper_2609_10165_b300 import inputs as I

    t = [time.perf_counter()]
    c = O.classify(g["grid"], g["body"], "HGC")
    lev = O.build_levels(c)
    t.append(time.perf_counter())
    X = c.grid.centre(c.grid.unlin(c.idx))
    S = (X + c.psi[:, None] * c.n)[lev.order]
    nn = c.n[lev.order]
    arrays = [f.on_grid(g["grid"], np.float32).astype(np.float64) for f in g["fields"]]
    bcs = [I.bc_values(f, k, S, nn) for f, k in zip(g["fields"], g["bc"])]
    t.append(time.perf_counter())
    out = O.fill(c, lev, arrays, g["bc"], bcs)
    t.append(time.perf_counter())
    fo, fscale = O.forces(c, lev, out[2], [out[0], out[1]], g["mu"], I.DRAG_LIFT_DIRS_2D)
    t.append(time.perf_counter())
    gx, gb = O.adjoint_gradient(c, lev, g["bc"], 2, [0, 1], g["mu"], I.DRAG_LIFT_DIRS_2D, (1.0, 1.0))
    t.append(time.perf_counter())
    phases = {"classify_levels": t[1] - t[0], "inputs": t[2] - t[1], "fill": t[3] - t[2],
              "forces": t[4] - t[3], "adjoint": t[5] - t[4]}
    if not keep:
        return c.n_ghosts * 3, phases
    cells = c.idx[lev.order]
    res = {"cells": cells, "values": [o[cells] for o in out], "fmax": [float(np.abs(a).max()) for a in arrays],
           "forces": fo, "fscale": fscale, "gx": gx, "gb": gb}
    return c.n_ghosts * 3, phases, res


def _oracle_geometry_index(args):
    """Pool worker: rebuild the seeded batch (parameters only) and run one
    geometry."""
    n_geoms, gi = args
    from paper_2609_10165_b300 import inputs as I
    return _oracle_geometry(I.batch(n_geoms)[gi])


# the step's kernels by phase of the method (the serial per-kernel profile;
# a re-run has no separate scans: "iface", "ghost_compact" and "gsrc" scan in
# the same launch; "scan", "ghost_flags" and "ghost_write" are the planning
# path's kernels)
PHASES = {
    "classify": ("rows", "iface", "scan", "place", "reclassify", "ghost_flags", "ghost_write", "ghost_compact",
                 "ghost_geom"),
    "levels": ("poscell", "deps", "levels", "reorder", "tables", "gsrc"),
    "fill": ("fill_part", "fill_chain"),
    "forces": ("forces",),
    "adjoint": ("adj_seed", "adj_part", "adj_chain", "adj_probe", "adj_fluid", "adj_bc"),
}


def phase_sums(prof_ms):
    out = {ph: round(sum(prof_ms.get(k, 0.0) for k in ks), 5) for ph, ks in PHASES.items()}
    named = {k for ks in PHASES.values() for k in ks}
    rest = sum(v for k, v in prof_ms.items() if k not in named)
    if rest:
        out["other"] = round(rest, 5)
    return out


def sample_order(n, seed=2609):
    """A seeded permutation of the geometry indices: the CPU samples draw
    from the whole batch, not from its first geometries."""
    return [int(i) for i in np.random.default_rng(seed).permutation(n)]


def accuracy(gpu, res_by_geom, offsets, info):
    """Worst error of the FP32 GPU path against the FP64 oracle (which ran on
    the same FP32 field values, with FP64 boundary data at its own boundary
    points) over the sampled geometries: ghost values relative to the field's
    maximum, forces relative to the magnitude of their terms, gradients
    relative to their maximum."""
    ev = ef = eg = 0.0
    for b, r in res_by_geom.items():
        o0 = int(offsets[b])
        sel = info["geom"] == b
        cells = r["cells"]
        for f in range(3):
            if cells.size:
                d = np.abs(gpu["fields"][f][o0 + cells].astype(np.float64) - r["values"][f])
                ev = max(ev, float(d.max()) / max(r["fmax"][f], 1e-300))
        d = np.abs(gpu["forces"][b] - r["forces"]) / np.maximum(r["fscale"], 1e-300)
        ef = max(ef, float(d.max()))
        o1 = o0 + r["gx"].shape[1]
        for f in range(3):
            sc = max(np.abs(r["gx"][f]).max(), np.abs(r["gb"][f]).max(), 1e-300)
            d1 = np.abs(gpu["gf"][f][o0:o1].astype(np.float64) - r["gx"][f]).max()
            d2 = np.abs(gpu["gb"][f][sel].astype(np.float64) - r["gb"][f]).max() if sel.any() else 0.0
            eg = max(eg, float(max(d1, d2)) / sc)
    return {"against": "FP64 oracle on the same FP32 field values, boundary data at its own S (FP64)",
            "geometries": len(res_by_geom),
            "ghost_values_rel_field_max": ev, "forces_rel_terms": ef, "gradients_rel_max": eg,
            "test_tolerances": {"ghost_values_rel_field_max": 1e-5, "forces_rel_terms": 1e-4,
                                "gradients_rel_max": 2e-5}}


def cpu_baseline(geoms_all, budget_s=15.0, gpu=None, offsets=None, info=None):
    """The oracle as it stands on a bounded sample of the batch, one thread:
    classify, levels, fill of 3 fields, forces and the explicit-matrix
    adjoint, with the seconds of each phase.  Geometries are taken in a
    seeded random order over the whole batch until the budget is spent.
    With the GPU results of the step (gpu), the oracle's results on the same
    sample also give the `accuracy` of the FP32 path (compared after the
    timing)."""
    t0 = time.perf_counter()
    updates = 0
    done = []
    phases = {}
    kept = {}
    for b in sample_order(len(geoms_all)):
        r = _oracle_geometry(geoms_all[b], keep=gpu is not None)
        updates += r[0]
        done.append(b)
        for k, v in r[1].items():
            phases[k] = phases.get(k, 0.0) + v
        if gpu is not None:
            kept[b] = r[2]
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    out = {"value": updates / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%d of %d geometries of %s in a seeded random order (classify, levels, fill of 3 "
                     "fields, forces, explicit-matrix adjoint), %.1f s" % (len(done), len(geoms_all), WORKLOAD, dt),
           "sample_geometries": sorted(done),
           "phases_s": {k: round(v, 3) for k, v in phases.items()}}
    if gpu is not None:
        out["accuracy"] = accuracy(gpu, kept, offsets, info)
    return out


def cpu_baseline_all_cores(n_geoms, budget_s=15.0):
    """The same oracle path over all host cores: a process pool (spawn, so
    that no worker inherits a CUDA context) runs geometries in parallel,
    largest first, until the budget is spent; the sample is the geometries
    finished by then."""
    import multiprocessing as mp
    from paper_2609_10165_b300 import inputs as I

    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    geoms = I.batch(n_geoms)
    order = sorted(range(n_geoms), key=lambda i: -geoms[i]["grid"]["n"][0])
    ctx = mp.get_context("spawn")
    updates = done = 0
    with ctx.Pool(cores) as pool:
        t0 = time.perf_counter()
        for u, _ in pool.imap_unordered(_oracle_geometry_index, [(n_geoms, i) for i in order]):
            updates += u
            done += 1
            if time.perf_counter() - t0 > budget_s:
                break
        dt = time.perf_counter() - t0
        pool.terminate()
    return {"value": updates / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of %d geometries of %s, largest first, on a %d-process pool, %.1f s "
                      "(worker start-up included)" % (done, n_geoms, WORKLOAD, cores, dt)}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    geoms = make_batch(args.geoms)
    ts = []
    covered = set()
    for s in range(args.warmup + args.steps):
        # each step a bounded sample: 2 geometries drawn (seeded, without
        # replacement) from the whole batch
        pick = [int(i) for i in np.random.default_rng(2609 + s).choice(len(geoms), 2, replace=False)]
        t0 = time.perf_counter()
        u = sum(_oracle_geometry(geoms[i])[0] for i in pick)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            ts.append(u / dt)
            covered.update(pick)
    val = float(np.mean(ts))
    sample = ("per step 2 geometries of %s drawn at random (seeded) from all %d; the timed steps covered "
              "%d distinct geometries" % (WORKLOAD, len(geoms), len(covered)))
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "impl": "reference",
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "2 geometries per step"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": val, "sample": sample,
                             "sample_geometries": sorted(covered)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# Algorithmic bytes per step of every kernel (2D: K = 3 stencil members, FP32
# fields, s = 4 B; FP64 coefficients).  A kernel's minimum HBM traffic: the
# records it must read once and the outputs it must write once.
def algorithmic_bytes(n_cells, rows, ni, ng, n_gsrc, F, dim=2):
    K = 3 if dim == 2 else 7
    s = 4
    return {
        "rows": n_cells * 1 + rows * 8,                          # tags + row runs
        "iface": rows * (8 + 4) + ni * 9,                        # runs, offsets; cell, geo, side
        "place": ni * 10,                                        # interface record + tag
        "reclassify": ni * 9,                                    # pass A over the interface
        # passes A and B (a step's fused re-run), flags, offsets and ghost
        # records: interface record, tag, normal byte, final tag, offset; per
        # ghost cell, geometry, meta
        "ghost_compact": ni * 15 + ng * 12,
        "ghost_geom": ng * (12 + 8 + 8 * dim + 4),               # record in; psi, n, meta out
        # the planning path's separate kernels (counts, scans, compaction)
        "scan": 8 * (rows + ni + ng),
        "ghost_flags": ni * 13,
        "ghost_write": ni * 13 + ng * (12 + 12 + 8 + 8 * dim + 4),
        # positions and preset counts; a step's fused re-run also writes the
        # final tags of the interface cells (record, final tag in, tag out)
        "poscell": 2 * ng * 12 + ni * 10,
        "deps": ng * (12 + 8 * dim + K + 4 * K + 4 * K + 4),
        "levels": ng * (4 * K + 12),
        "reorder": ng * 2 * (4 + 4 + 8 + 8 * dim + 4 + 4 * K + 4),
        "tables": ng * (4 + 4 + 8 + 8 * dim + 4 + 2 * dim + 16 * 8 + (1 + (1 + K) + dim * (K + 1)) * 8),
        "gsrc": ng * 32 + n_gsrc * 4,                            # probes, offsets, sources
        # partial sums: per update the boundary datum and the fluid members
        # read, the sum written; per ghost geometry, cell, meta and weights
        "fill_part": ng * F * (K * s + s + s) + ng * (4 + 4 + 4 + (K + 1) * 8),
        # chain: per update the partial read and the ghost written; per ghost
        # cell, meta, dependency positions and weights of both kinds
        "fill_chain": ng * F * (s + s) + ng * (4 + 4 + 4 * K + 2 * K * 8),
        "fill_level": ng * F * (K * s + s + s) + ng * (4 + 4 + 2 * (K + 1) * 8),
        "forces": ng * (4 + 4 + 8 * dim + 4 + (2 + K + dim * (K + 1)) * 8 + s * (dim + 1) * (K + 1)),
        "adj_seed": ng * (4 + 8 * dim + (2 + K + dim * (K + 1)) * 8 + F * (K + 1) * 8),
        # start values and incidence records: per source entry its word,
        # F force coefficients, the consumer's meta and two weights read, a
        # record (consumer, two weights) written; per update lambda0 written
        "adj_part": ng * (4 + s * F) + n_gsrc * (4 + F * 8 + 4 + 16 + 4 + 2 * s),
        # chain: per update lambda0 read and lambda written; per source entry
        # its record read
        "adj_chain": ng * (4 + 2 * s * F) + n_gsrc * (4 + 2 * s),
        "adj_level": ng * (4 + s * F) + n_gsrc * (4 + 4 + F * 8 + 16),
        # fluid targets' sources: per ghost its record, per incidence the
        # member's tag, the neighbours' tags, its count and cell written, about
        # two source words
        "adj_probe": ng * 12 + ng * K * (1 + 8 + 8 + 2 * 4),
        "adj_fluid": ng * 12 + ng * K * (F * 8 + 8 + F * s) + ng * K * F * s,
        "adj_bc": ng * (4 + 4 + 16 + 3 * F * s),
    }


# Source file of each kernel group's device code; with the shared headers it
# keys the counters below to the code they were measured on.
CSRC = os.path.join(ROOT, "paper_2609_10165_b300", "csrc")
KERNEL_SOURCE = {
    "rows": "classify.cu", "iface": "classify.cu", "place": "classify.cu", "reclassify": "classify.cu",
    "ghost_compact": "classify.cu", "ghost_geom": "classify.cu", "ghost_flags": "classify.cu",
    "ghost_write": "classify.cu", "scan": "scan.cu",
    "poscell": "levels.cu", "deps": "levels.cu", "levels": "levels.cu", "reorder": "levels.cu",
    "tables": "levels.cu", "gsrc": "levels.cu", "fill_part": "fill.cu", "fill_chain": "fill.cu",
    "fill_level": "fill.cu", "forces": "forces.cu", "adj_seed": "adjoint.cu", "adj_part": "adjoint.cu",
    "adj_chain": "adjoint.cu", "adj_level": "adjoint.cu", "adj_probe": "adjoint.cu",
    "adj_fluid": "adjoint.cu", "adj_bc": "adjoint.cu", "pfill": "packed.cu", "padj": "packed.cu",
    "tiled_fill": "tiled.cu",
}
SHARED_HEADERS = ("ebr_device.cuh", "ebr_probe.cuh", "ebr_kernels.cuh", "lookback.cuh", "traction.cuh")


def kernel_source_hash(kernel):
    """First 16 hex digits of the SHA-256 of the kernel's source file and the
    shared device headers (None for an unknown kernel)."""
    f = KERNEL_SOURCE.get(kernel)
    if f is None:
        return None
    h = hashlib.sha256()
    for name in (f,) + SHARED_HEADERS:
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture
# on this workload, with the source hash of the kernel version captured (L2
# write-back hides most writes of a short kernel).  A figure whose hash no
# longer matches the source is reported as null, with the reason.
TRAFFIC_PER_LAUNCH = {
    "rows": (0.82e6, "fd3f4e6fc115cb04"),
    "iface": (1.62e6, "fd3f4e6fc115cb04"),
    "place": (2.92e6, "fd3f4e6fc115cb04"),
    "reclassify": (7.38e6, "fd3f4e6fc115cb04"),
    "ghost_compact": (7.65e6, "fd3f4e6fc115cb04"),
    "ghost_geom": (1.28e6, "fd3f4e6fc115cb04"),
    "poscell": (2.87e6, "123c8594a95264bf"),
    "deps": (11.11e6, "123c8594a95264bf"),
    "levels": (1.13e6, "123c8594a95264bf"),
    "reorder": (7.45e6, "123c8594a95264bf"),
    "tables": (9.88e6, "123c8594a95264bf"),
    "gsrc": (3.43e6, "123c8594a95264bf"),
    "fill_part": (25.41e6, "c73c35a163a29288"),
    "fill_chain": (5.66e6, "c73c35a163a29288"),
    "forces": (28.10e6, "983ee207011997bd"),
    "adj_seed": (6.17e6, "e86c2f12d673d229"),
    "adj_part": (4.00e6, "e86c2f12d673d229"),
    "adj_chain": (3.13e6, "e86c2f12d673d229"),
    "adj_probe": (13.96e6, "e86c2f12d673d229"),
    "adj_fluid": (19.21e6, "e86c2f12d673d229"),
    "adj_bc": (5.44e6, "e86c2f12d673d229"),
    # many-field mode (192 FP32 fields): all launches of one call, summed
    "pfill": (279.88e6, "8058ec0ee428c269"),
    "padj": (359.71e6, "8058ec0ee428c269"),
}

# FP64 flops per launch (DADD + DMUL + 2 x DFMA thread instructions from one
# ncu capture on this workload) of the kernels bound by the FP64 pipe, with
# the source hash of the captured version.
FP64_FLOPS_PER_LAUNCH = {
    "ghost_geom": (11_920_293, "fd3f4e6fc115cb04"), "tables": (10_419_154, "123c8594a95264bf"),
}


def counter(table, kernel):
    """(value, None) when the table holds a figure measured on the current
    source of the kernel, else (None, reason)."""
    if kernel not in table:
        return None, "no ncu capture of this kernel on this workload"
    value, h = table[kernel]
    cur = kernel_source_hash(kernel)
    if cur != h:
        return None, "kernel source changed since the capture (captured %s, now %s)" % (h, cur)
    return value, None
# the FP64 pipe of one SM issues two double FMAs per clock (the counter's
# sustained peak), i.e. 4 flops per SM per clock
FP64_FLOPS_PER_SM_CLK = 4


def fp64_peak_tflops(n_sm, sm_mhz):
    return n_sm * FP64_FLOPS_PER_SM_CLK * sm_mhz * 1e6 / 1e12


def roofline_object(prof_ms, prof_n, algo, hbm_peak, hbm_peak_kind, n_sm, sm_mhz):
    """The dominant kernel of the serial per-kernel profile against its bound:
    the FP64 pipe (flops per launch / event-timed duration vs. the peak from
    the SM count and clock) for the kernels in FP64_FLOPS_PER_LAUNCH, HBM
    (algorithmic bytes per launch / duration vs. the measured copy bandwidth)
    otherwise.  The HBM figures are kept for every kernel."""
    top = max(prof_ms, key=prof_ms.get)
    per_kernel = {}
    for k, v in sorted(prof_ms.items(), key=lambda kv: -kv[1]):
        gbs = algo[k] / (v * 1e-3) / 1e9 if k in algo else None
        per_kernel[k] = {"ms": round(v, 5), "launches": prof_n[k],
                         "algo_bytes": algo.get(k), "gbs": round(gbs, 1) if gbs else None}
        fl, _ = counter(FP64_FLOPS_PER_LAUNCH, k)
        if fl is not None:
            per_kernel[k]["fp64_tflops"] = round(fl / (v / prof_n[k] * 1e-3) / 1e12, 4)
    t_launch = prof_ms[top] / prof_n[top] * 1e-3      # seconds per launch
    tb = algo[top] / prof_n[top]                      # bytes per launch
    gbs = tb / t_launch / 1e9
    hbm = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
           "peak_source": hbm_peak_kind, "algo_bytes_per_launch": tb}
    fp64_peak = fp64_peak_tflops(n_sm, sm_mhz)
    traffic, why = counter(TRAFFIC_PER_LAUNCH, top)
    roof = {"kernel": top, "traffic": traffic, "source_hash": kernel_source_hash(top)}
    if why:
        roof["traffic_null_because"] = why
    flops, why_f = counter(FP64_FLOPS_PER_LAUNCH, top)
    if flops is not None:
        ach = flops / t_launch / 1e12
        roof.update({"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": ach / fp64_peak, "flops_per_launch": flops,
                     "peak_source": "derived: %d SMs x %d FP64 flops per SM per clock x %.0f MHz"
                                    % (n_sm, FP64_FLOPS_PER_SM_CLK, sm_mhz),
                     "hbm": hbm})
    else:
        roof.update({"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": gbs / hbm_peak, "peak_source": hbm_peak_kind, "algo_bytes_per_launch": tb})
        if top in ("ghost_geom", "tables"):
            roof["fp64_flops_null_because"] = why_f
    roof["fp64_peak_tflops"] = fp64_peak
    roof["per_kernel"] = per_kernel
    roof["phases_ms"] = phase_sums(prof_ms)
    return roof

def unique_fluid_targets(R, info, dim=2):
    """Active (ghost, member) incidences whose member is a fluid cell, and the
    number of distinct such cells (host count from the ghost records: member
    k is active when n_a != 0 on every axis it is offset along)."""
    tags = R.tags.cpu().numpy()
    off = np.asarray(R.cell_offset)
    geom, cell, r, nrm = info["geom"], info["cell"], info["r"], info["normal"]
    nx = np.array([R._grids[b].n[0] for b in range(R.B)], dtype=np.int64)[geom]
    e = np.where(nrm[:, :dim] < 0.0, -1, 1)
    offs = [(1, 0), (0, 1), (1, 1)]
    targets, n_inc = [], 0
    for ox, oy in offs:
        act = np.ones(cell.size, bool)
        if ox:
            act &= nrm[:, 0] != 0.0
        if oy:
            act &= nrm[:, 1] != 0.0
        t = off[geom] + cell + ox * r[:, 0] * e[:, 0] + nx * (oy * r[:, 1] * e[:, 1])
        fl = act & (tags[np.clip(t, 0, tags.size - 1)] == 0)
        n_inc += int(fl.sum())
        targets.append(t[fl])
    return n_inc, int(np.unique(np.concatenate(targets)).size)


def throughput_mode(R, info, fields, bcs, kinds3, flush, stream, steps, warmup, peak, n_sets=32):
    """Many fields per cell in the field-minor layout: n_sets copies of the
    (u, v, p) set (scaled), 3 n_sets FP32 fields, fill + transpose of the fill
    per step on the classified batch (the geometry part is not repeated)."""
    import torch
    dev = R.device
    F = 3 * n_sets
    kinds = list(kinds3) * n_sets
    scale = torch.tensor([1.0 + 0.01 * k for k in range(n_sets) for _ in range(3)], device=dev)
    P = torch.stack([fields[f % 3] for f in range(F)], dim=1).mul_(scale)
    Pbc = torch.stack([bcs[f % 3] for f in range(F)], dim=1).mul_(scale)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2609)
    C = torch.randn((R.n_cells, F), generator=gen, device=dev, dtype=torch.float32)
    Gbc = torch.empty((Pbc.shape[0], F), device=dev, dtype=torch.float32)
    side = torch.cuda.Stream(dev)

    def step(adjoint=True):
        if adjoint:
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                R.reconstruct_packed_adjoint(kinds, C, Gbc)
        R.reconstruct_packed(P, kinds, Pbc)
        if adjoint:
            torch.cuda.current_stream().wait_stream(side)

    graphs = {}
    cap = torch.cuda.Stream(dev)
    for adj in (True, False):
        step(adj)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(cap):
            with torch.cuda.graph(g, stream=cap, capture_error_mode="relaxed"):
                step(adj)
        torch.cuda.synchronize()
        graphs[adj] = g
    for _ in range(warmup):
        graphs[True].replay()
    torch.cuda.synchronize()
    R.sync_status()
    ms = time_steps(graphs[True].replay, steps, stream, flush)
    ms_f = time_steps(graphs[False].replay, max(5, steps // 2), stream, flush)
    R.sync_status()
    # per-kernel device times inside a captured step
    R.profile(True)
    gp = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap):
        with torch.cuda.graph(gp, stream=cap, capture_error_mode="relaxed"):
            step(True)
    torch.cuda.synchronize()
    R.profile(False)
    prof = {}
    for _ in range(5):
        flush.zero_()
        gp.replay()
        torch.cuda.synchronize()
        for k, (v, n) in R.profile_read(keep=True).items():
            prof[k] = (prof.get(k, (0.0, n))[0] + v / 5, n)
    R.profile_read(keep=False)
    del gp, graphs
    ng = int(Pbc.shape[0])
    n_inc, n_tgt = unique_fluid_targets(R, info)
    diag = R.diagnostics()
    s = 4
    K = 3
    # algorithmic bytes per call (2D, FP32): forward per update K stencil
    # reads + boundary datum + ghost write, per ghost its record (cell, meta)
    # and the weights of both kinds; adjoint per update the ghost cotangent
    # read and cleared and dJ/db written, every fluid target read and written
    # once per field, per ghost the record and the weights
    algo = {
        "pfill": ng * F * (K * s + s + s) + ng * (8 + 2 * (K + 1) * 8),
        "padj": ng * F * 3 * s + n_tgt * F * 2 * s + ng * (8 + 2 * (K + 1) * 8) + diag["n_gsrc"] * 4,
    }
    groups = {"pfill": ("pfill_part", "pfill_lvl", "pfill_tail"),
              "padj": ("padj_tail", "padj_lvl", "padj_fluid")}
    med = float(np.median(ms))
    med_f = float(np.median(ms_f))
    per = {k: {"ms": round(v, 5), "launches": n} for k, (v, n) in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    call_ms = {gname: sum(prof[k][0] for k in ks if k in prof) for gname, ks in groups.items()}
    for gname in algo:
        per[gname] = {"ms": round(call_ms[gname], 5), "algo_bytes": algo[gname],
                      "gbs": round(algo[gname] / (call_ms[gname] * 1e-3) / 1e9, 1) if call_ms[gname] else None}
    top = max(algo, key=lambda k: call_ms[k])
    ach = algo[top] / (call_ms[top] * 1e-3) / 1e9
    step_bytes = sum(algo.values())
    out = {
        "fields": F, "field_sets": n_sets, "layout": "field-minor [cells][fields], FP32",
        "updates_per_step": ng * F, "value": ng * F / (med * 1e-3), "unit": "updates/s",
        "ms_per_step": med, "p10_ms": float(np.percentile(ms, 10)), "p90_ms": float(np.percentile(ms, 90)),
        "fwd_value": ng * F / (med_f * 1e-3), "fwd_ms_per_step": med_f,
        "step_algo_bytes": step_bytes, "step_gbs": step_bytes / (med * 1e-3) / 1e9,
        "step_frac": step_bytes / (med * 1e-3) / 1e9 / peak,
        "fluid_incidences": n_inc, "unique_fluid_targets": n_tgt, "schedule": diag["packed"],
        "roofline": {"kernel": top, "launches": "all launches of the call", "bound": "hbm",
                     "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "traffic": counter(TRAFFIC_PER_LAUNCH, top)[0],
                     "source_hash": kernel_source_hash(top), "algo_bytes_per_call": algo[top]},
        "per_kernel": per,
        "l2": "flushed before every timed step (512 MB write)",
    }
    del P, Pbc, C, Gbc
    torch.cuda.empty_cache()
    return out


def single_grid_mode(dev, stream, flush, steps, warmup, peak, tiles=((16, 16, 16), (32, 32, 32), (64, 64, 64))):
    """One large grid: the 512^3 sphere, 4 FP32 fields (u, v, w Dirichlet, p
    Neumann), planned and levelled once.  Times the tiled fill (persistent
    cooperative launch, per-level exchange between tiles, Sec. 3.2) for a few
    tile sizes against the level-launch fill (one launch per level), each
    captured in a CUDA graph, the L2 flushed before every step."""
    import torch
    from paper_2609_10165_b300 import inputs as I
    from paper_2609_10165_b300.api import Reconstructor

    w = I.sphere_cfg(512, 3)
    R = Reconstructor(w["grid"], w["body"], "HGC", device=dev)
    R.build_levels()
    R.sync_status()
    info = R.ghost_info()
    F = len(w["fields"])
    fields = [torch.tensor(f.on_grid(w["grid"], np.float32), device=dev) for f in w["fields"]]
    bcs = [torch.tensor(I.bc_values(f, k, info["S"], info["normal"]), dtype=torch.float32, device=dev)
           for f, k in zip(w["fields"], w["bc"])]
    ng = int(info["cell"].size)
    K, sz = 7, 4
    algo = ng * F * (K * sz + 2 * sz) + ng * (4 + 4 + 2 * (K + 1) * 8)
    cap = torch.cuda.Stream(dev)

    how = {}

    def timed(fn, key):
        fn()
        torch.cuda.synchronize()
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(cap):
                with torch.cuda.graph(g, stream=cap, capture_error_mode="relaxed"):
                    fn()
            torch.cuda.synchronize()
            run, how[key] = g.replay, "graph"
        except Exception as e:  # reported: timed eagerly instead
            torch.cuda.synchronize()
            run, how[key] = fn, "eager (capture failed: %s)" % str(e)[:80]
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        ms = float(np.median(time_steps(run, steps, stream, flush)))
        R.sync_status()
        return ms

    out = {"workload": "sphere_512 (512^3 cells, r = 0.5 in [-2, 2]^3, HGC), 4 FP32 fields, FP64 coefficients",
           "ghosts": ng, "levels": int(info["level"].max()), "updates_per_step": ng * F,
           "algo_bytes": algo, "l2": "flushed before every timed step (512 MB write)"}
    ms_lv = timed(lambda: R.reconstruct(fields, w["bc"], bcs, mode="level"), "level_launch")
    out["level_launch"] = {"ms": ms_lv, "value": ng * F / (ms_lv * 1e-3), "launches": int(info["level"].max())}
    best = None
    out["tiled"] = {}
    for tile in tiles:
        R.tiled_plan(list(tile))
        ti = R.tiled_info()
        key = "x".join(str(t) for t in tile)
        ms = timed(lambda: R.reconstruct_tiled(fields, w["bc"], bcs), key)
        out["tiled"][key] = {"ms": ms, "value": ng * F / (ms * 1e-3), "active_tiles": ti["active_tiles"],
                             "ctas": ti["grid_f32"], "sent_ghosts": ti["sent_ghosts"],
                             "values_exchanged": ti["values_exchanged"], "halo_values": ti["halo_values"],
                             "sent_per_level": ti["sent_per_level"]}
        if best is None or ms < out["tiled"][best]["ms"]:
            best = key
    b = out["tiled"][best]
    out["timing"] = how
    out["best_tile"] = best
    out["value"] = b["value"]
    out["unit"] = UNIT
    out["roofline"] = {"kernel": "tiled_fill", "bound": "hbm", "achieved": algo / (b["ms"] * 1e-3) / 1e9,
                       "peak": peak, "unit": "GB/s", "frac": algo / (b["ms"] * 1e-3) / 1e9 / peak,
                       "algo_bytes_per_launch": algo,
                       "traffic": counter(TRAFFIC_PER_LAUNCH, "tiled_fill")[0],
                       "source_hash": kernel_source_hash("tiled_fill")}
    del fields, bcs, R
    torch.cuda.empty_cache()
    return out


def moving_mode(dev, n_geoms=32, steps=20, warmup=3, dt=0.02):
    """Moving bodies (Sec. 7): the first n_geoms geometries of the batch, each
    body translating and turning at a seeded rate, advanced step by step:
    move (re-plan, reusing the device buffers), levels, boundary data at the
    new boundary points, fill of 3 FP32 fields, forces and adjoint.  Every
    step synchronises with the host (the counts change), so the step time is
    taken on the host clock around a synchronised step."""
    import torch
    from paper_2609_10165_b300 import inputs as I
    from paper_2609_10165_b300.moving import MovingStepper, RigidMotion

    geoms = I.batch()[:n_geoms]
    rng = np.random.default_rng(2609)
    motions = [RigidMotion(g["body"], velocity=tuple(rng.uniform(-0.05, 0.05, 2)) + (0.0,),
                           omega=float(rng.uniform(-0.5, 0.5)) if g["body"]["kind"] == "ellipse"
                           else float(rng.uniform(-0.05, 0.05))) for g in geoms]
    fields = [[g["fields"][f] for g in geoms] for f in range(3)]
    st = MovingStepper([g["grid"] for g in geoms], motions, fields, geoms[0]["bc"], geoms[0]["roles"]["vel"],
                       geoms[0]["roles"]["p"], geoms[0]["mu"], I.DRAG_LIFT_DIRS_2D, device=dev)
    for _ in range(warmup):
        st.advance(dt, adjoint=True)
    torch.cuda.synchronize()
    a0 = st.R.diagnostics()["allocations"]
    ts, ups = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        out = st.advance(dt, adjoint=True)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
        ups.append(int(out[1]["cell"].size) * 3)
    st.R.sync_status()
    a1 = st.R.diagnostics()["allocations"]
    ms = float(np.median(ts)) * 1e3
    return {"what": "%d geometries of batch_256 moving (translation + rotation), per step: move + levels + "
                    "boundary data + fill (3 FP32 fields) + forces + adjoint; host clock around a synchronised "
                    "step" % n_geoms,
            "ms_per_step": ms, "value": float(np.median(ups)) / (ms * 1e-3), "unit": UNIT,
            "ghosts_min_max": [min(ups) // 3, max(ups) // 3], "allocations_in_timed_steps": a1 - a0,
            "steps": steps}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    geoms, shard_info = rank_batch(args.geoms, rank, world)
    R, info, host_fields, host_bcs, fields, bcs = setup(geoms, dev, torch.float32)
    ng = int(info["cell"].size)
    F = 3
    updates = ng * F
    counts = R.counts()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2

    step = Step(R, fields, bcs, geoms, "persistent", adjoint=True, overlap=True)
    for _ in range(max(args.warmup, 3)):
        step()
    R.sync_status()
    # launch shapes of the one-thread-per-item kernels, tuned on this workload
    # (eager serial steps, per-launch events, L2 flushed) before any capture
    tuned, tune_rep = None, None
    if not args.no_autotune:
        from paper_2609_10165_b300.autotune import autotune
        tuned, tune_rep = autotune(R, Step(R, fields, bcs, geoms, "persistent", adjoint=True, overlap=False),
                                   reps=5, flush=flush.zero_)
        R.sync_status()
    l0 = R.launches
    step()
    torch.cuda.synchronize()
    launches_per_step = R.launches - l0

    # CUDA graph of the whole step
    g = torch.cuda.CUDAGraph(keep_graph=True)
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
            step()
    torch.cuda.synchronize()
    graph_kernels = count_graph_kernels(g)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    R.sync_status()

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    ms = time_steps(g.replay, args.steps, stream, flush)
    t_wall = time.perf_counter() - t_wall0
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    R.sync_status()
    ms_med = float(np.median(ms))
    ms_stats = {"mean": float(np.mean(ms)), "median": ms_med, "p10": float(np.percentile(ms, 10)),
                "p90": float(np.percentile(ms, 90))}
    ms_step, total_updates = reduce_over_ranks(ms_med, updates, dev)
    value = total_updates / (ms_step * 1e-3)

    # the same step with plain launches (programmatic dependent launch off)
    from paper_2609_10165_b300.api import set_pdl
    set_pdl(False)
    try:
        g0 = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            step()
            torch.cuda.synchronize()
            with torch.cuda.graph(g0, stream=side, capture_error_mode="relaxed"):
                step()
        torch.cuda.synchronize()
        ms_plain = float(np.median(time_steps(g0.replay, max(5, args.steps // 2), stream, flush)))
        del g0
    finally:
        set_pdl(True)
    R.sync_status()

    # forward only (same graph construction)
    step_f = Step(R, fields, bcs, geoms, "persistent", adjoint=False)
    gf = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        step_f()
        torch.cuda.synchronize()
        with torch.cuda.graph(gf, stream=side, capture_error_mode="relaxed"):
            step_f()
    torch.cuda.synchronize()
    ms_f = float(np.median(time_steps(gf.replay, max(5, args.steps // 2), stream, flush)))

    # reconstruction only: a stationary body (Sec. 7: the classification is
    # redone only when the body moves), planned and levelled once; per step
    # the fill, the forces and the adjoint (same graph construction)
    step_r = Step(R, fields, bcs, geoms, "persistent", adjoint=True, overlap=True, geometry=False)
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        step_r()
        torch.cuda.synchronize()
        with torch.cuda.graph(gr, stream=side, capture_error_mode="relaxed"):
            step_r()
    torch.cuda.synchronize()
    ms_r_all = time_steps(gr.replay, max(5, args.steps // 2), stream, flush)
    ms_r = float(np.median(ms_r_all))
    del gr

    diag = R.diagnostics()

    # per-kernel device times: the step captured once more, without the
    # two-stream overlap (so that no kernel's span includes another's), with
    # the library's timing events recorded as graph nodes, replayed with the
    # L2 flushed
    step_serial = Step(R, fields, bcs, geoms, "persistent", adjoint=True, overlap=False)
    step_serial()
    torch.cuda.synchronize()
    R.profile(True)
    gp = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(gp, stream=side, capture_error_mode="relaxed"):
            step_serial()
    torch.cuda.synchronize()
    R.profile(False)
    n_prof = 5
    prof_ms, prof_n = {}, {}
    for _ in range(n_prof):
        flush.zero_()
        gp.replay()
        torch.cuda.synchronize()
        for k, (ms_k, cnt) in R.profile_read(keep=True).items():
            prof_ms[k] = prof_ms.get(k, 0.0) + ms_k / n_prof
            prof_n[k] = cnt
    R.profile_read(keep=False)
    del gp
    top = max(prof_ms, key=prof_ms.get)

    # throughput mode: many fields per cell, field-minor layout
    tput = None
    if args.sets > 0:
        tput = throughput_mode(R, info, fields, bcs, geoms[0]["bc"], flush, stream, args.steps,
                               max(args.warmup, 3), measured_peaks()[0], n_sets=args.sets)

    # one large grid: the tiled fill with its per-level exchange
    single = None
    if args.single_grid and rank == 0 and not args.lite:
        single = single_grid_mode(dev, stream, flush, max(5, args.steps // 4), max(args.warmup, 3),
                                  measured_peaks()[0])

    moving = None
    if rank == 0 and not args.lite:
        moving = moving_mode(dev)

    # plain FP64 path: one launch per level per geometry, FP64 fields, no graph
    ms64 = float("nan")
    try:
        if args.lite:
            raise StopIteration
        fields64 = [torch.tensor(a.astype(np.float64), device=dev) for a in host_fields]
        bcs64 = [torch.tensor(b, dtype=torch.float64, device=dev) for b in host_bcs]
        step64 = Step(R, fields64, bcs64, geoms, "level", adjoint=True)
        step64()
        torch.cuda.synchronize()
        ms64 = float(np.median(time_steps(step64, max(3, args.steps // 5), stream, flush)))
        del fields64, bcs64, step64
    except StopIteration:
        pass
    except Exception as e:  # reported, not hidden
        print("plain FP64 path failed: %s" % e, file=sys.stderr)

    # end to end through host buffers: H2D of the fields and boundary data
    # from pinned memory, the step, D2H of the forces
    pin_f = [torch.from_numpy(a).pin_memory() for a in host_fields]
    pin_b = [torch.from_numpy(b.astype(np.float32)).pin_memory() for b in host_bcs]
    host_out = torch.empty(R.B * 6, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in pin_f + pin_b)
    d2h = host_out.numel() * 8

    def e2e_step():
        for t, h in zip(fields, pin_f):
            t.copy_(h, non_blocking=True)
        for t, h in zip(bcs, pin_b):
            t.copy_(h, non_blocking=True)
        g.replay()
        host_out.copy_(step.out, non_blocking=True)

    e2e_ms = [float("nan")]
    e2e_val = None
    if not args.lite:
        e2e_step()
        torch.cuda.synchronize()
        e2e_ms = time_steps(e2e_step, max(5, args.steps // 3), stream, flush)
        e2e_val = total_updates / (np.median(e2e_ms) * 1e-3)

    # roofline of the dominant kernel: algorithmic bytes per launch / duration
    peak, peak_kind = measured_peaks()
    n_cells = R.n_cells
    rows = sum(c2["n_cells"] // geoms[b]["grid"]["n"][0] for b, c2 in enumerate(counts))
    ni = sum(c2["n_interface"] for c2 in counts)
    algo = algorithmic_bytes(n_cells, rows, ni, ng, diag["n_gsrc"], F, dim=2)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = roofline_object(prof_ms, prof_n, algo, peak, peak_kind, n_sm, measured_sm_mhz())
    roof.update({
        "timing": "CUDA events recorded as nodes of a captured graph of the step without the two-stream overlap, mean of 5 replays, L2 flushed",
        "step_algo_bytes": sum(algo.values()),
        "step_frac": sum(algo.values()) / (ms_step * 1e-3) / 1e9 / peak})

    recon_keys = [k for k in PHASES["fill"] + PHASES["forces"] + PHASES["adjoint"] if k in algo]
    recon_bytes = sum(algo[k] for k in recon_keys)
    reconstruction = {
        "what": "fill (3 FP32 fields) + forces + adjoint per step on a geometry planned and levelled "
                "once (stationary body); CUDA graph, adjoint on a second stream, L2 flushed",
        "value": total_updates / (ms_r * 1e-3), "unit": UNIT, "ms_per_step": ms_r,
        "p10_ms": float(np.percentile(ms_r_all, 10)), "p90_ms": float(np.percentile(ms_r_all, 90)),
        "step_algo_bytes": recon_bytes,
        "step_frac": recon_bytes / (ms_r * 1e-3) / 1e9 / peak,
        "phases_ms_serial": {ph: phase_sums(prof_ms)[ph] for ph in ("fill", "forces", "adjoint")},
    }

    baseline = None
    if rank == 0 and not args.no_baseline and not args.lite:
        gpu_out = {"fields": [f.cpu().numpy() for f in fields], "forces": step.out.view(R.B, 6).cpu().numpy(),
                   "gf": [t.cpu().numpy() for t in step.gf], "gb": [t.cpu().numpy() for t in step.gb]}
        baseline = cpu_baseline(geoms, budget_s=15.0, gpu=gpu_out, offsets=R.cell_offset, info=info)
        del gpu_out
        baseline["all_cores"] = cpu_baseline_all_cores(args.geoms, budget_s=15.0)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "ms_stats_rank0": ms_stats, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 fields, f64 coefficients", "data": "synthetic",
        "config": {"workload": WORKLOAD, "geometries": args.geoms, "cells": n_cells, "ghosts": ng,
                   "fields": F, "placement": "HGC", "max_levels": max(c2["n_levels"] for c2 in counts),
                   "l2": "flushed before every timed step (512 MB write)", "graph": True,
                   "parallelism": "geometry shards, no exchange on the data path" if world > 1 else "single",
                   "shards": shard_info,
                   "row_fallbacks_since_plan": diag["row_fallbacks"],
                   "block_sizes": tuned if tuned is not None else "defaults (128)"},
        "autotune": tune_rep,
        "fwd_updates_per_s": total_updates / (ms_f * 1e-3), "fwd_ms_per_step": ms_f,
        "plain_launch": {"what": "the headline step captured with programmatic dependent launch off",
                         "ms_per_step": ms_plain},
        "reconstruction_only": reconstruction,
        "accuracy": baseline.get("accuracy") if baseline else None,
        "plain_fp64_updates_per_s": total_updates / (ms64 * 1e-3) if ms64 == ms64 else None,
        "plain_fp64_ms_per_step": ms64,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": float(np.median(e2e_ms))},
        "gpu_launches": int(launches_per_step * args.steps),
        "graph_kernel_nodes_per_step": graph_kernels,
        "roofline": roof,
        "throughput_mode": tput,
        "single_grid": single,
        "moving_bodies": moving,
        "clocks": clk,
        "cpu_baseline": baseline,
        "wall_s_timed": t_wall,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
