"""Ghost-cell dependency DAG and topological levels (oracle; test infrastructure).

Sec. 3.2: a ghost G depends on every stencil member that is itself a ghost and
carries a structurally non-zero reconstruction weight (a member offset along
an axis with n_i = 0 has weight zero, Secs. 4-5, so that edge is absent).
Level L_1 holds ghosts whose stencils contain no ghost; a ghost is in L_k when
all the ghosts it needs are in L_1..L_{k-1}, i.e. level(G) = 1 + max level of
its ghost dependencies (longest path from the fluid).  Computed here by a
memoised depth-first search, which detects cycles.  Within a level the order
is arbitrary (Sec. 3.2); the canonical order used for all data exchanged with
the library is (level, linear index).
"""

import sys

import numpy as np

from .classify import check_stencils, stencil_members, EBRError, E_CYCLE


class Levels:
    def __init__(self, level, order, level_ptr, deps, midx, active):
        self.level = level          # int64 [N_g], per ghost in linear-index order
        self.order = order          # int64 [N_g], canonical position -> ghost (index order)
        self.level_ptr = level_ptr  # int64 [n_levels + 1]
        self.deps = deps            # list per ghost of (k, ghost) dependencies
        self.midx = midx            # int64 [N_g, K] member cell indices
        self.active = active        # bool [N_g, K]

    @property
    def n_levels(self):
        return int(self.level_ptr.size - 1)

    def position(self):
        """Inverse of ``order``: ghost (index order) -> canonical position."""
        pos = np.empty_like(self.order)
        pos[self.order] = np.arange(self.order.size)
        return pos


def build_levels(cls):
    midx = check_stencils(cls)
    _, _, active = stencil_members(cls)
    ng = cls.n_ghosts
    pos = {int(c): g for g, c in enumerate(cls.idx)}
    deps = []
    for g in range(ng):
        dg = []
        for k in range(midx.shape[1]):
            m = int(midx[g, k])
            if active[g, k] and m in pos:
                dg.append((k, pos[m]))
        deps.append(dg)

    level = [0] * ng
    state = [0] * ng      # 0 unvisited, 1 on the DFS stack, 2 done
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 4 * ng + 1000))
    try:
        def visit(g):
            if state[g] == 2:
                return level[g]
            if state[g] == 1:
                raise EBRError(E_CYCLE, "ghost %d lies on a dependency cycle" % int(cls.idx[g]))
            state[g] = 1
            lv = 1
            for _, dgh in deps[g]:
                lv = max(lv, 1 + visit(dgh))
            level[g] = lv
            state[g] = 2
            return lv

        for g in range(ng):
            visit(g)
    finally:
        sys.setrecursionlimit(old)

    level = np.array(level, dtype=np.int64)
    order = np.lexsort((cls.idx, level)) if ng else np.zeros(0, dtype=np.int64)
    nl = int(level.max()) if ng else 0
    level_ptr = np.zeros(nl + 1, dtype=np.int64)
    for lv in range(1, nl + 1):
        level_ptr[lv] = level_ptr[lv - 1] + int(np.sum(level == lv))
    return Levels(level, order.astype(np.int64), level_ptr, deps, midx, active)
