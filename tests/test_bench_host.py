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
    for k in ("rows", "iface", "scan", "place", "reclassify", "ghost_flags", "ghost_write", "ghost_compact",
              "ghost_geom", "poscell",
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


def _profile(top_ms):
    prof_ms = {"ghost_geom": 0.0438, "fill_chain": 0.0418, "rows": 0.0400, "tables": 0.0235, "forces": 0.0377,
               "gsrc": 0.0270}
    prof_ms.update(top_ms)
    prof_n = {k: (2 if k == "gsrc" else 1) for k in prof_ms}
    algo = bench.algorithmic_bytes(48_250_166, 126_000, 171_700, 85_556, 160_000, 3)
    return prof_ms, prof_n, algo


def test_fp64_peak_from_unit_counts_and_clock():
    # 148 SMs x 2 double FMAs (4 flops) per SM per clock x 2032 MHz
    assert bench.fp64_peak_tflops(148, 2032.0) == pytest.approx(1.202944)


def test_roofline_of_an_fp64_bound_dominant_kernel(monkeypatch):
    h = bench.kernel_source_hash
    monkeypatch.setattr(bench, "FP64_FLOPS_PER_LAUNCH", {"ghost_geom": (11_876_551, h("ghost_geom")),
                                                         "tables": (10_419_154, h("tables"))})
    monkeypatch.setattr(bench, "TRAFFIC_PER_LAUNCH", {"ghost_geom": (9.15e6, h("ghost_geom"))})
    prof_ms, prof_n, algo = _profile({})
    r = bench.roofline_object(prof_ms, prof_n, algo, 6495.6, "measured", 148, 2032.0)
    assert r["kernel"] == "ghost_geom" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    ach = 11_876_551 / 0.0438e-3 / 1e12
    assert r["achieved"] == pytest.approx(ach)
    assert r["frac"] == pytest.approx(ach / bench.fp64_peak_tflops(148, 2032.0))
    assert r["traffic"] == 9.15e6
    assert r["hbm"]["unit"] == "GB/s" and r["hbm"]["frac"] == pytest.approx(
        algo["ghost_geom"] / 0.0438e-3 / 1e9 / 6495.6)
    assert r["per_kernel"]["tables"]["fp64_tflops"] > 0
    assert "fp64_tflops" not in r["per_kernel"]["fill_chain"]
    assert set(r["phases_ms"]) >= {"classify", "levels", "fill", "forces"}


def test_roofline_of_a_memory_bound_dominant_kernel():
    prof_ms, prof_n, algo = _profile({"fill_chain": 0.09, "gsrc": 0.03})
    r = bench.roofline_object(prof_ms, prof_n, algo, 6495.6, "measured", 148, 2032.0)
    assert r["kernel"] == "fill_chain" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(algo["fill_chain"] / 0.09e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6495.6)
    # per-launch figures divide by the launch count
    prof_ms, prof_n, algo = _profile({"gsrc": 0.3})
    r = bench.roofline_object(prof_ms, prof_n, algo, 6495.6, "measured", 148, 2032.0)
    assert r["kernel"] == "gsrc" and r["algo_bytes_per_launch"] == pytest.approx(algo["gsrc"] / 2)
    assert r["achieved"] == pytest.approx(algo["gsrc"] / 2 / (0.15e-3) / 1e9)


def test_counters_measured_on_other_source_are_null(monkeypatch):
    # a counter keyed to another version of the kernel's source is not used:
    # traffic null with the reason, and an FP64-bound kernel falls back to
    # the HBM roofline
    monkeypatch.setattr(bench, "FP64_FLOPS_PER_LAUNCH", {"ghost_geom": (11_876_551, "0" * 16)})
    monkeypatch.setattr(bench, "TRAFFIC_PER_LAUNCH", {"ghost_geom": (9.15e6, "0" * 16)})
    prof_ms, prof_n, algo = _profile({})
    r = bench.roofline_object(prof_ms, prof_n, algo, 6495.6, "measured", 148, 2032.0)
    assert r["traffic"] is None and "changed" in r["traffic_null_because"]
    assert r["bound"] == "hbm" and "changed" in r["fp64_flops_null_because"]
    assert r["source_hash"] == bench.kernel_source_hash("ghost_geom")
    # every profiled kernel name has a source file
    for ks in bench.PHASES.values():
        for k in ks:
            assert bench.kernel_source_hash(k) is not None, k


def test_cpu_samples_cover_the_whole_batch():
    order = bench.sample_order(256)
    assert sorted(order) == list(range(256))
    assert order[:20] != list(range(20))


def test_committed_counters_match_the_committed_sources():
    # every ncu figure the bench line can report names a profiled kernel and
    # was taken on the kernel source as it stands (a kernel changed after its
    # capture needs a new capture, or its figure removed)
    import re
    for table in (bench.TRAFFIC_PER_LAUNCH, bench.FP64_FLOPS_PER_LAUNCH):
        for kernel, (value, h) in table.items():
            assert re.fullmatch(r"[0-9a-f]{16}", h), (kernel, h)
            assert value > 0, kernel
            got, why = bench.counter(table, kernel)
            assert got == value, (kernel, why)
