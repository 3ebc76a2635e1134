"""Tie audit of the workloads: no cell may sit within 1e-9 dx of a
classification threshold (psi = 0, |psi| = dn/2, an r_i ceiling, n_i = 0),
where two correct FP64 implementations could round to different tags.  The
workloads are checked here so the bit-exact GPU comparison is meaningful."""

import numpy as np
import pytest

import oracle as O
from paper_2609_10165_b300 import inputs as I


@pytest.mark.parametrize("name", ["cylinder_128", "airfoil_2048", "cylinder_1024", "sphere_256"])
@pytest.mark.parametrize("placement", ["HGC", "CGC", "CGC_ES"])
def test_workload_has_no_ties(name, placement):
    w = I.WORKLOADS[name]()
    c = O.classify(w["grid"], w["body"], placement)
    assert c.ties == []
    O.build_levels(c)     # acyclic, stencils valid


def test_whole_batch_has_no_ties():
    # all 256 geometries, in a spawn pool (the same worker the full-batch
    # GPU test uses for its bit-exact structure comparison)
    from tests.oracle_pool import batch_structure, start_pool
    n = 256
    with start_pool(n) as pool:
        res = pool.map_async(batch_structure, [(n, gi, "HGC") for gi in range(n)]).get(timeout=1200)
    assert [r[0] for r in res] == list(range(n))
    assert [r[0] for r in res if not r[1]] == []


def test_pool_worker_matches_a_direct_call():
    from tests.oracle_pool import batch_structure, start_pool
    args = [(256, 120, "HGC"), (256, 171, "CGC")]      # two of the smallest grids
    with start_pool(len(args)) as pool:
        got = pool.map_async(batch_structure, args).get(timeout=600)
    for a, r in zip(args, got):
        direct = batch_structure(a)
        assert r[0] == direct[0] and r[1] == direct[1]
        for x, y in zip(r[2:], direct[2:]):
            assert np.array_equal(x, y)
