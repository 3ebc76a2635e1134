"""Sharding a batch of independent geometries over ranks (one GPU each).

The geometries of a batch share nothing (Sec. 3.2's levels are per ghost set;
the forces are per geometry), so a batch shards without any exchange on the
data path: each rank plans, levels, fills and differentiates its own
geometries.  The ranks are balanced by the work, which scales with the ghost
count times the fields; the ghost count of a geometry is estimated on the
host before any classification from the body's perimeter (surface area) over
the cell width: a ghost layer is about one cell thick along the boundary.
"""

import math

import numpy as np


def estimated_ghosts(g):
    """Ghosts of a geometry dict (grid, body), estimated: boundary length
    (area in 3D) over the cell size."""
    grid, body = g["grid"], g["body"]
    d = int(grid["dim"])
    h = [(grid["hi"][a] - grid["lo"][a]) / grid["n"][a] for a in range(d)]
    kind = body["kind"]
    if kind == "sphere":
        r = body["radii"][0]
        return 4.0 * math.pi * r * r / (h[0] * h[1])
    if kind == "circle":
        per = 2.0 * math.pi * body["radii"][0]
    elif kind == "ellipse":
        a, b = body["radii"][0], body["radii"][1]
        per = math.pi * (3 * (a + b) - math.sqrt((3 * a + b) * (a + 3 * b)))   # Ramanujan
    else:
        # the two surfaces of a thin section lying along x: about one ghost
        # per column of the section on each side
        return 2.04 * body["chord"] / h[0]
    return per / min(h)


def partition(geoms, n_ranks, fields=3):
    """Indices of the geometries of each rank: longest first to the rank with
    the least estimated work (ghosts x fields) so far; ties to the lower rank.
    Deterministic; every geometry in exactly one shard."""
    w = [estimated_ghosts(g) * fields for g in geoms]
    order = sorted(range(len(geoms)), key=lambda i: (-w[i], i))
    load = [0.0] * n_ranks
    shards = [[] for _ in range(n_ranks)]
    for i in order:
        r = min(range(n_ranks), key=lambda k: (load[k], k))
        shards[r].append(i)
        load[r] += w[i]
    return [sorted(s) for s in shards], load
