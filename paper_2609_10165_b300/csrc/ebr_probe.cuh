// Cell-index helpers and the fixed-order probe of the (ghost, member) pairs
// that read a given cell (transposed stencil incidences), shared by the level
// builder and the adjoint.  Host-callable as well, so that the validation of
// ghost positions can be exercised on the CPU.
#pragma once

#include "ebr_device.cuh"

namespace ebr {

__host__ __device__ inline void cell_ijk3(const Geom& g, int cell, int ijk[3]) {
  ijk[0] = cell % g.n[0];
  int r = cell / g.n[0];
  ijk[1] = r % g.n[1];
  ijk[2] = r / g.n[1];
}

__host__ __device__ inline int cell_lin(const Geom& g, const int ijk[3]) {
  return ijk[0] + g.n[0] * (ijk[1] + g.n[1] * ijk[2]);
}

// fixed-trip loops over the three axes (predicated on the dimension) keep
// every index static, so the small arrays stay in registers
__host__ __device__ inline bool in_grid(const Geom& g, const int ijk[3]) {
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < g.dim && (ijk[a] < 0 || ijk[a] >= g.n[a])) ok = false;
  return ok;
}

// Position (in the ghost records rec_cell, pre-sort or canonical) of the
// ghost at linear cell `cell` of geometry g, or -1.  pcell (pos_of_cell of
// the geometry) is only meaningful at cells of this plan's ghosts; the
// position is accepted when it lies in the geometry's ghost range and its
// record names the same cell, so a ghost tag that the caller added to the
// tag buffer after planning never leads to an unchecked index.
__host__ __device__ inline int ghost_slot_of(const Geom& g, int cell, const int* pcell, const int* rec_cell) {
  const int q = pcell[cell];
  if (q < g.ghost_off || q >= g.ghost_off + g.n_ghost) return -1;
  return rec_cell[q] == cell ? q : -1;
}

// member k of a ghost at ijk with meta m
__host__ __device__ inline void member_ijk(const Geom& g, const int ijk[3], uint32_t m, int k, int out[3]) {
  int o[3];
  stencil_off(g.dim, k, o);
#pragma unroll
  for (int a = 0; a < 3; ++a) out[a] = ijk[a] + (a < g.dim ? o[a] * meta_r(m, a) * meta_e(m, a) : 0);
}

// ---------------------------------------------------------------------------
// transposed incidences: for a target cell T, the (ghost H, slot) pairs with
// member_slot(H) = T, found by probing H = T - delta over the box |delta_a| <= R
// in a fixed order.  Slot 0 (H = T itself) is listed first for ghost targets.
// ---------------------------------------------------------------------------
// One z-slab (dz fixed) of the reach-1 probe, in three rounds of independent
// loads (tags; positions; metas) before the ordered visit.  Returns false when
// the visitor stopped the probe.
template <typename Visit>
__host__ __device__ __forceinline__ bool probe_slab_r1(const Geom& g, const int tijk[3], int dz, const int8_t* tg,
                                              const int* pcell, const int* gcell, const uint32_t* g_meta,
                                              Visit& visit) {
  const int K = stencil_k(g.dim);
  int hc[9], q[9];
  uint32_t m[9];
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const int dx = b % 3 - 1, dy = b / 3 - 1;
    const int h[3] = {tijk[0] - dx, tijk[1] - dy, tijk[2] - dz};
    const bool ok = !(dx == 0 && dy == 0 && dz == 0) && in_grid(g, h);
    hc[b] = ok ? cell_lin(g, h) : -1;
  }
  int8_t t[9];
#pragma unroll
  for (int b = 0; b < 9; ++b) t[b] = hc[b] >= 0 ? tg[hc[b]] : (int8_t)0;
#pragma unroll
  for (int b = 0; b < 9; ++b) q[b] = (t[b] == 2 || t[b] == -2) ? pcell[hc[b]] : -1;
  // a position outside the geometry's ghost range, or whose record names
  // another cell, is not a ghost of this plan (ghost_slot_of)
#pragma unroll
  for (int b = 0; b < 9; ++b)
    if (q[b] < g.ghost_off || q[b] >= g.ghost_off + g.n_ghost) q[b] = -1;
  int qc[9];
#pragma unroll
  for (int b = 0; b < 9; ++b) qc[b] = q[b] >= 0 ? gcell[q[b]] : -1;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    if (q[b] >= 0 && qc[b] != hc[b]) q[b] = -1;
    m[b] = q[b] >= 0 ? g_meta[q[b]] : 0u;
  }
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    if (q[b] < 0) continue;
    const int dd[3] = {b % 3 - 1, b / 3 - 1, dz};
    for (int k = 0; k < K; ++k) {
      int o[3];
      stencil_off(g.dim, k, o);
      bool hit = true;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (a < g.dim && o[a] * meta_r(m[b], a) * meta_e(m[b], a) != dd[a]) hit = false;
      if (hit) { if (!visit(q[b], k + 1)) return false; }
    }
  }
  return true;
}

// pcell: pos_of_cell of the geometry (canonical positions); gcell: the
// canonical ghost records' cells (g_cell), used to validate each position.
template <typename Visit>
__host__ __device__ inline void probe_sources(const Geom& g, const int tijk[3], const int8_t* tg,
                                     const int* pcell, const int* gcell, const uint32_t* g_meta, int R,
                                     Visit visit) {
  if (R == 1) {
    // the usual reach: the 8 (2D) or 26 (3D) neighbours, same order as below
    if (g.dim == 3 && !probe_slab_r1(g, tijk, -1, tg, pcell, gcell, g_meta, visit)) return;
    if (!probe_slab_r1(g, tijk, 0, tg, pcell, gcell, g_meta, visit)) return;
    if (g.dim == 3) probe_slab_r1(g, tijk, 1, tg, pcell, gcell, g_meta, visit);
    return;
  }
  const int K = stencil_k(g.dim);
  int Rz = g.dim == 3 ? R : 0;
  for (int dz = -Rz; dz <= Rz; ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        if (dx == 0 && dy == 0 && dz == 0) continue;
        int hijk[3] = {tijk[0] - dx, tijk[1] - dy, tijk[2] - dz};
        if (!in_grid(g, hijk)) continue;
        int hc = cell_lin(g, hijk);
        int8_t t = tg[hc];
        if (t != 2 && t != -2) continue;
        const int q = ghost_slot_of(g, hc, pcell, gcell);
        if (q < 0) continue;
        uint32_t m = g_meta[q];
        int dd[3] = {dx, dy, dz};
        for (int k = 0; k < K; ++k) {
          int o[3];
          stencil_off(g.dim, k, o);
          bool hit = true;
#pragma unroll
          for (int a = 0; a < 3; ++a)
            if (a < g.dim && o[a] * meta_r(m, a) * meta_e(m, a) != dd[a]) hit = false;
          if (hit) { if (!visit(q, k + 1)) return; }
        }
      }
}

}  // namespace ebr
