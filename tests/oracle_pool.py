"""Process-pool workers that run the CPU oracle on geometries of the seeded
batch.  Host only: imports the oracle and the input generator, never torch
or the CUDA library, so that a pool started with `spawn` stays light and
never touches a GPU context."""

import multiprocessing as mp
import os

import oracle as O
from paper_2609_10165_b300 import inputs as I


def batch_structure(args):
    """(gi, tie-free, tags, canonical ghost cells, their levels, their r,
    their psi, normals and boundary points S, the smallest cell width) of
    geometry gi of the n_geoms-geometry batch, placed with `placement`."""
    n_geoms, gi, placement = args
    g = I.batch(n_geoms)[gi]
    c = O.classify(g["grid"], g["body"], placement)
    lev = O.build_levels(c)
    X = c.grid.centre(c.grid.unlin(c.idx))
    S = X + c.psi[:, None] * c.n
    return (gi, c.ties == [], c.tags, c.idx[lev.order], lev.level[lev.order], c.r[lev.order],
            c.psi[lev.order], c.n[lev.order], S[lev.order], min(c.grid.h))


def start_pool(n_tasks):
    """A spawn pool sized to the host's cores (at most 16, at most n_tasks)."""
    n = max(1, min(16, os.cpu_count() or 1, n_tasks))
    return mp.get_context("spawn").Pool(n)
