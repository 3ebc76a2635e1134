"""Host-side logic of the benchmark, without a GPU: the reference arm's JSON
line (the oracle timed on a bounded sample), the per-phase sums of the
per-kernel profile, and the algorithmic-byte formulas' basic properties."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_phase_sums_cover_every_profiled_kernel():
    prof = {"rows": 0.04, "iface": 0.03, "scan": 0.03, "levels": 0.02, "fill_part": 0.01,
            "fill_chain": 0.04, "forces": 0.035, "adj_probe": 0.03, "adj_fluid": 0.02, "other_kernel": 0.005}
    ph = bench.phase_sums(prof)
    assert ph["classify"] == pytest.approx(0.10)
    assert ph["levels"] == pytest.approx(0.02)
    assert ph["fill"] == pytest.approx(0.05)
    assert ph["adjoint"] == pytest.approx(0.05)
    assert ph["other"] == pytest.approx(0.005)
    assert sum(ph.values()) == pytest.approx(sum(prof.values()))
    # every kernel name the library profiles belongs to a phase
    named = {k for ks in bench.PHASES.values() for k in ks}
    for k in ("rows", "iface", "scan", "place", "reclassify", "ghost_flags", "ghost_write", "poscell",
              "deps", "levels", "reorder", "tables", "gsrc", "fill_part", "fill_chain", "forces",
              "adj_seed", "adj_part", "adj_chain", "adj_probe", "adj_fluid", "adj_bc"):
        assert k in named, k


def test_algorithmic_bytes_grow_with_the_workload():
    a = bench.algorithmic_bytes(1_000_000, 2000, 10_000, 5000, 12_000, 3)
    b = bench.algorithmic_bytes(2_000_000, 4000, 20_000, 10_000, 24_000, 3)
    assert set(a) == set(b)
    for k in a:
        assert a[k] > 0
        assert b[k] == pytest.approx(2 * a[k]), k
    # the tag stream is one byte per cell plus the row runs
    assert a["rows"] == 1_000_000 + 8 * 2000
