"""Host logic of the launch-shape autotuner, with a stand-in for the library:
a fake context whose per-kernel step time is a known function of the block
size.  The search must find each kernel's minimum, leave kernels the step
never launches at their old shape, and round-trip its cache."""

import numpy as np
import pytest

from paper_2609_10165_b300 import autotune as A


class FakeCtx:
    """Mimics the Reconstructor calls the tuner uses; the 'time' of kernel k
    at block size T is cost[k][T] ms per step (plus a little seeded noise)."""

    def __init__(self, cost, launched):
        self.cost = cost
        self.launched = launched
        self.shape = {k: 128 for k in cost}
        self.prof = False
        self.rec = {}
        self.rng = np.random.default_rng(0)
        self.cell_offset = [0, 100, 250]
        self.n_ghosts = 42
        self.dim = 2

    def tunable_kernels(self):
        return list(self.cost)

    def set_block_size(self, k, t):
        if k not in self.shape or t % 32 or not 32 <= t <= 256:
            raise ValueError(k)
        self.shape[k] = t

    def block_size(self, k):
        return self.shape[k]

    def profile(self, on=True):
        self.prof = on
        if on:
            self.rec = {}

    def profile_read(self, keep=False):
        out = dict(self.rec)
        if not keep:
            self.rec = {}
        return out

    def step(self):
        if not self.prof:
            return
        for k in self.launched:
            t = self.cost[k][self.shape[k]] * (1.0 + 1e-3 * self.rng.standard_normal())
            ms, n = self.rec.get(k, (0.0, 0))
            self.rec[k] = (ms + t, n + 1)


COST = {
    "place": {64: 0.030, 128: 0.031, 256: 0.036},
    "tables": {64: 0.029, 128: 0.026, 256: 0.027},
    "adj_fluid": {64: 0.090, 128: 0.082, 256: 0.071},
    "gsrc": {64: 0.05, 128: 0.05, 256: 0.05},
}


def test_default_candidates_are_allowed_block_sizes():
    assert all(t % 32 == 0 and 32 <= t <= 256 for t in A.DEFAULT_CANDIDATES)


def test_choose_takes_the_minimum_and_breaks_ties_small():
    assert A.choose({64: 2.0, 128: 1.0, 256: 3.0}) == 128
    assert A.choose({256: 1.0, 64: 1.0, 128: 1.0}) == 64
    with pytest.raises(ValueError):
        A.choose({})


def test_search_finds_each_minimum_and_skips_unlaunched_kernels():
    R = FakeCtx(COST, launched=["place", "tables", "adj_fluid"])
    R.set_block_size("gsrc", 96)
    shapes, rep = A.autotune(R, R.step, candidates=(64, 128, 256), reps=5)
    assert shapes == {"place": 64, "tables": 128, "adj_fluid": 256, "gsrc": 96}
    assert R.shape == shapes
    assert rep["source"] == "search"
    assert set(rep["times_ms"]) == {"place", "tables", "adj_fluid"}
    assert rep["times_ms"]["adj_fluid"][256] == pytest.approx(0.071, rel=1e-2)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "shapes.json")
    R = FakeCtx(COST, launched=list(COST))
    key = A.workload_key(R, "f32", 3, "fake-gpu")
    shapes, rep = A.autotune(R, R.step, candidates=(64, 128, 256), reps=3, cache_path=path, key=key)
    assert rep["source"] == "search"
    R2 = FakeCtx(COST, launched=list(COST))
    shapes2, rep2 = A.autotune(R2, R2.step, candidates=(64, 128, 256), reps=3, cache_path=path, key=key)
    assert rep2["source"] == "cache" and shapes2 == shapes and R2.shape == shapes
    # another workload misses the cache
    R3 = FakeCtx(COST, launched=list(COST))
    R3.cell_offset = [0, 100, 251]
    assert A.workload_key(R3, "f32", 3, "fake-gpu") != key
