"""Tie audit of the workloads: no cell may sit within 1e-9 dx of a
classification threshold (psi = 0, |psi| = dn/2, an r_i ceiling, n_i = 0),
where two correct FP64 implementations could round to different tags.  The
workloads are checked here so the bit-exact GPU comparison is meaningful."""

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


def test_batch_subset_has_no_ties():
    for k, gm in enumerate(I.batch()):
        if k % 8:
            continue
        c = O.classify(gm["grid"], gm["body"], "HGC")
        assert c.ties == [], k
        O.build_levels(c)
