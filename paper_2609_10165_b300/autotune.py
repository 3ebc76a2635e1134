"""Launch-shape autotuner.

For each tunable kernel of a Reconstructor (the kernels that run one thread
per interface cell, ghost or fluid target; see ``ebr_set_block_size`` in the
C header) it picks the threads per block that make the kernel fastest on this
GPU for this geometry set and field count.  Timing uses the library's own
per-launch CUDA events (``ebr_profile``): every candidate runs the caller's
step ``reps`` times and keeps the median of that kernel's time per step.  The
search is coordinate-wise: one kernel at a time, the others at their current
shapes.  The block size changes scheduling only, never a result, so the
search is free to try any allowed value.

Results can be cached in a JSON file keyed by the GPU name, the dimension,
the field type, the field count and a signature of the geometry set, so that
a repeated run of the same workload skips the search.
"""

import hashlib
import json
import os
import tempfile
import time

import numpy as np

DEFAULT_CANDIDATES = (32, 64, 96, 128, 192, 256)


def choose(times):
    """The candidate with the least time; ties go to the smaller block."""
    if not times:
        raise ValueError("no timings")
    return min(sorted(times), key=lambda t: times[t])


def workload_key(R, dtype, n_fields, device_name):
    """Cache key: GPU, dimension, field type and count, and a hash of the
    geometry set's cell offsets and ghost count (its shape)."""
    h = hashlib.sha1()
    h.update(np.asarray(R.cell_offset, dtype=np.int64).tobytes())
    h.update(np.int64(R.n_ghosts).tobytes())
    return "%s|d%d|%s|F%d|B%d|%s" % (device_name, R.dim, dtype, int(n_fields), len(R.cell_offset) - 1,
                                     h.hexdigest()[:16])


def _load_cache(path):
    if not path or not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def _store_cache(path, cache):
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_candidate(R, name, step, reps, flush):
    """Median over `reps` steps of the time `name` took in one step (ms);
    None when the step does not launch it."""
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush()
        R.profile(True)
        step()
        prof = R.profile_read(keep=False)
        R.profile(False)
        if name not in prof:
            return None
        ts.append(prof[name][0])
    return float(np.median(ts))


def autotune(R, step, candidates=DEFAULT_CANDIDATES, reps=5, kernels=None, flush=None,
             cache_path=None, key=None):
    """Tune the block sizes of R's kernels for the work `step` issues (a
    callable making the library calls to tune, e.g. classify + levels + fill
    + forces + adjoint).  Returns (shapes, report): shapes {kernel: threads}
    now set on R; report {"source": "cache" | "search", "seconds": ...,
    "times_ms": {kernel: {threads: ms}}}."""
    t0 = time.perf_counter()
    names = list(kernels) if kernels is not None else R.tunable_kernels()
    cache = _load_cache(cache_path) if key is not None else {}
    if key is not None and key in cache and all(n in cache[key] for n in names):
        shapes = {n: int(cache[key][n]) for n in names}
        for n, t in shapes.items():
            R.set_block_size(n, t)
        return shapes, {"source": "cache", "seconds": time.perf_counter() - t0, "times_ms": {}}
    step()                                   # first call plans / warms up
    R.profile_read(keep=False)
    shapes, times_ms = {}, {}
    for name in names:
        orig = R.block_size(name)
        times = {}
        for T in candidates:
            R.set_block_size(name, T)
            t = _time_candidate(R, name, step, reps, flush)
            if t is None:
                break
            times[T] = t
        if not times:                        # not launched by this step: leave as is
            R.set_block_size(name, orig)
            shapes[name] = orig
            continue
        best = choose(times)
        R.set_block_size(name, best)
        shapes[name] = best
        times_ms[name] = {int(k): round(v, 5) for k, v in times.items()}
    if key is not None and cache_path:
        cache = _load_cache(cache_path)
        cache[key] = shapes
        _store_cache(cache_path, cache)
    return shapes, {"source": "search", "seconds": time.perf_counter() - t0, "times_ms": times_ms}
