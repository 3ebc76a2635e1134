// Level-by-level ghost fill (Sec. 3.2; closed forms of Secs. 4-5 through the
// per-ghost weight table).
//
// Two schedules:
//  * k_fill_level: one grid-wide launch per level of one geometry.
//  * k_fill_partial + k_fill_chain: everything that does not depend on
//    another ghost -- the boundary term and the fluid members of every ghost,
//    for every field -- is summed first by a grid-wide kernel (one thread per
//    ghost, all SMs); then one CTA per geometry loads those partial sums into
//    shared memory and runs the dependency chain level by level there,
//    separated by block barriers (warp barriers for the thin end).  Long
//    chains (an airfoil has ~60 levels) cost a few hundred cycles per level
//    instead of a kernel launch each.
// FP32 fields are combined in float with the weights rounded to float.
#include "ebr_kernels.cuh"

namespace ebr {

struct FieldSet {
  void* f[8];
  const void* bc[8];
  int kind[8];
};

// the weight table in the field type (FP32 fields: the float copy of the
// double table)
template <typename T>
__device__ inline T wload(const T* wtab, int ng, int bc, int slot, int p) {
  return wtab[(size_t)(bc * 8 + slot) * ng + p];
}

__device__ inline int member_cell(int dim, int cell, int nx, int ny, uint32_t m, int k) {
  int o[3];
  stencil_off(dim, k, o);
  int off = o[0] * meta_r(m, 0) * meta_e(m, 0) + nx * (o[1] * meta_r(m, 1) * meta_e(m, 1));
  if (dim == 3) off += nx * ny * (o[2] * meta_r(m, 2) * meta_e(m, 2));
  return cell + off;
}

// All loads of a ghost (weights, boundary data, member values of every
// field) are issued before its stores: the members of a level-L ghost are
// fluid cells or ghosts of lower levels, never written in this launch, so
// the loads may run ahead of the stores; the sums keep the order boundary
// term, then active members in member order.
template <typename T, int D>
__global__ void k_fill_level(FieldSet P, int F, long long cell_off, int p0, int p1,
                             const int* __restrict__ g_cell, const uint32_t* __restrict__ g_meta,
                             const T* __restrict__ wtab, int ng, int nx, int ny, int* status) {
  pdl_enter();
  constexpr int K = D == 2 ? 3 : 7;
  int p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= p1) return;
  const int cell = g_cell[p];
  const uint32_t m = g_meta[p];
  const uint32_t act = meta_active(m);
  int mc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) mc[k] = member_cell(D, cell, nx, ny, m, k);
  // weights of both boundary-condition kinds (selected per field below
  // without a dynamic index, so that they stay in registers)
  T w0[K + 1], w1[K + 1];
  w0[K] = wload<T>(wtab, ng, 0, 7, p);
  w1[K] = wload<T>(wtab, ng, 1, 7, p);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    w0[k] = wload<T>(wtab, ng, 0, k, p);
    w1[k] = wload<T>(wtab, ng, 1, k, p);
  }
  T val[8][K + 1];
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    if (f >= F) break;
    const T* fld = static_cast<const T*>(P.f[f]) + cell_off;
    val[f][K] = static_cast<const T*>(P.bc[f])[p];
#pragma unroll
    for (int k = 0; k < K; ++k) val[f][k] = (act >> k & 1u) ? fld[mc[k]] : T(0);
  }
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    if (f >= F) break;
    const bool neu = P.kind[f] != 0;
    T acc = (neu ? w1[K] : w0[K]) * val[f][K];
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act >> k & 1u) acc += (neu ? w1[k] : w0[k]) * val[f][k];
    static_cast<T*>(P.f[f])[cell_off + cell] = acc;
    if (!isfinite((double)acc)) set_status(status, S_ENONFINITE);
  }
}

void launch_fill_level(int dtype, int dim, int F, void* const* fields, const int* bc_kind,
                       const void* const* bc, long long cell_off, int p0, int p1, const int* g_cell,
                       const uint32_t* g_meta, const void* wtab, int ng_total, int nx, int ny,
                       int* status, cudaStream_t s) {
  if (p1 <= p0) return;
  FieldSet P;
  for (int f = 0; f < 8; ++f) {
    P.f[f] = f < F ? fields[f] : nullptr;
    P.bc[f] = f < F ? bc[f] : nullptr;
    P.kind[f] = f < F ? bc_kind[f] : 0;
  }
  int n = p1 - p0;
  int T = n < 128 ? 64 : 128;
  const unsigned nb = (unsigned)((n + T - 1) / T);
  if (dtype == 0 && dim == 2)
    launch(k_fill_level<float, 2>, nb, T, 0, s, P, F, cell_off, p0, p1, g_cell, g_meta, (const float*)wtab, ng_total, nx, ny, status);
  else if (dtype == 0)
    launch(k_fill_level<float, 3>, nb, T, 0, s, P, F, cell_off, p0, p1, g_cell, g_meta, (const float*)wtab, ng_total, nx, ny, status);
  else if (dim == 2)
    launch(k_fill_level<double, 2>, nb, T, 0, s, P, F, cell_off, p0, p1, g_cell, g_meta, (const double*)wtab, ng_total, nx, ny, status);
  else
    launch(k_fill_level<double, 3>, nb, T, 0, s, P, F, cell_off, p0, p1, g_cell, g_meta, (const double*)wtab, ng_total, nx, ny, status);
}

// Partial sum of every ghost and field: w_s b_G plus the fluid (non-
// dependency) members, in member order -- the first terms of the level fill,
// in the same order, so the chain that adds the dependency terms gives the
// same bits as summing everything in one place.
template <typename T>
__global__ void k_fill_partial(FieldSet P, int F, const Geom* __restrict__ G, const int* __restrict__ g_geo,
                               const int* __restrict__ g_cell, const uint32_t* __restrict__ g_meta,
                               const T* __restrict__ wtab, int ng, T* __restrict__ part) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  const Geom& g = G[g_geo[p]];
  const int dim = g.dim, K = stencil_k(dim), nx = g.n[0], ny = g.n[1];
  const int cell = g_cell[p];
  const uint32_t m = g_meta[p];
  const uint32_t act = meta_active(m), dm = meta_depmask(m);
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    if (f >= F) break;
    const T* fld = static_cast<const T*>(P.f[f]) + g.cell_off;
    const T* bc = static_cast<const T*>(P.bc[f]);
    const int kind = P.kind[f];
    T acc = wload<T>(wtab, ng, kind, 7, p) * bc[p];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      if (k >= K) break;
      if (!(act >> k & 1u) || (dm >> k & 1u)) continue;
      acc += wload<T>(wtab, ng, kind, k, p) * fld[member_cell(dim, cell, nx, ny, m, k)];
    }
    part[(size_t)f * ng + p] = acc;
  }
}

void launch_fill_partial(int dtype, int F, void* const* fields, const int* bc_kind, const void* const* bc,
                         const Geom* G, const int* g_geo, const int* g_cell, const uint32_t* g_meta,
                         const void* wtab, int ng, void* part, cudaStream_t s, int T) {
  if (ng <= 0) return;
  FieldSet P;
  for (int f = 0; f < 8; ++f) {
    P.f[f] = f < F ? fields[f] : nullptr;
    P.bc[f] = f < F ? bc[f] : nullptr;
    P.kind[f] = f < F ? bc_kind[f] : 0;
  }
  if (dtype == 0)
    launch(k_fill_partial<float>, (ng + T - 1) / T, T, 0, s, P, F, G, g_geo, g_cell, g_meta, (const float*)wtab, ng, (float*)part);
  else
    launch(k_fill_partial<double>, (ng + T - 1) / T, T, 0, s, P, F, G, g_geo, g_cell, g_meta, (const double*)wtab, ng, (double*)part);
}

constexpr int CH_T = 512;

size_t fill_chain_smem(int dtype, int dim, int F, int n) {
  size_t sz = dtype == 0 ? 4 : 8;
  int K = stencil_k(dim);
  // vals[F][n], weights of dependency members for both kinds [2][K][n],
  // positions [K][n], cells [n], level pointers [n + 1]
  return (size_t)n * (F * sz + 2 * K * sz + K * sizeof(int) + sizeof(int)) + (size_t)(n + 1) * sizeof(int) + 64;
}

// The dependency chain of geometry g in one CTA (CH_T threads), on the
// dynamic shared memory of fill_chain_smem.
template <typename T>
__device__ inline void chain_walk(const FieldSet& P, int F, const Geom& g, const int* __restrict__ g_cell,
                                  const uint32_t* __restrict__ g_meta, const int* __restrict__ g_dep,
                                  const int* __restrict__ lev_ptr, const T* __restrict__ wtab, int ng,
                                  const T* __restrict__ part, int* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = g.n_ghost, g0 = g.ghost_off, dim = g.dim;
  // geometry fields in registers: the loops below store to global memory,
  // after which a read through g would have to be repeated
  const int n_levels = g.n_levels;
  const long long cell_off = g.cell_off;
  const int K = stencil_k(dim);
  T* vals = reinterpret_cast<T*>(smem);                 // [F][n]
  T* wdep = vals + (size_t)F * n;                       // [2][K][n]
  int* dpos = reinterpret_cast<int*>(wdep + (size_t)2 * K * n);  // [K][n]
  int* cellv = dpos + (size_t)K * n;                             // [n]
  int* lps = cellv + n;                                          // [n_levels + 1]
  const int* lp = lev_ptr + g.lev_off;
  for (int q = threadIdx.x; q <= n_levels; q += CH_T) lps[q] = lp[q] - g0;
  // phase 1: the partial sums (boundary term + fluid members) of the
  // geometry's ghosts; dependency weights and positions.  U ghosts per
  // thread at a time: their cells, metas and partials are loaded together,
  // then (the meta tells which members are dependencies) their dependency
  // positions and weights
  constexpr int U = 4;
  for (int s0 = threadIdx.x; s0 < n; s0 += CH_T * U) {
    uint32_t dm[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 + u * CH_T;
      dm[u] = 0u;
      if (s >= n) continue;
      const int p = g0 + s;
      cellv[s] = g_cell[p];
      dm[u] = meta_depmask(g_meta[p]);
#pragma unroll
      for (int f = 0; f < 8; ++f)
        if (f < F) vals[(size_t)f * n + s] = part[(size_t)f * ng + p];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 + u * CH_T;
      if (s >= n) continue;
      const int p = g0 + s;
      for (int k = 0; k < K; ++k) {
        const bool d = dm[u] >> k & 1u;
        dpos[(size_t)k * n + s] = d ? g_dep[(size_t)k * ng + p] - g0 : -1;
        wdep[(size_t)k * n + s] = d ? wload<T>(wtab, ng, 0, k, p) : T(0);
        wdep[(size_t)(K + k) * n + s] = d ? wload<T>(wtab, ng, 1, k, p) : T(0);
      }
    }
  }
  __syncthreads();
  // phase 2: the dependency chain, level by level, on shared memory only
  // every field's sum in registers, the dependencies walked once: the loads
  // of all fields are issued together and no store intervenes (each field
  // still adds its dependencies in member order, so the bits are the same)
  auto relax = [&](int s) {
    const int cell = cellv[s];
    T v[8];
#pragma unroll
    for (int f = 0; f < 8; ++f)
      if (f < F) v[f] = vals[(size_t)f * n + s];
    for (int k = 0; k < K; ++k) {
      const int d = dpos[(size_t)k * n + s];
      if (d < 0) continue;
      const T w0 = wdep[(size_t)k * n + s], w1 = wdep[(size_t)(K + k) * n + s];
#pragma unroll
      for (int f = 0; f < 8; ++f)
        if (f < F) v[f] += (P.kind[f] ? w1 : w0) * vals[(size_t)f * n + d];
    }
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      if (f >= F) break;
      vals[(size_t)f * n + s] = v[f];
      static_cast<T*>(P.f[f])[cell_off + cell] = v[f];
      if (!isfinite(v[f])) set_status(status, S_ENONFINITE);
    }
  };
  // levels lw.. hold at most 32 ghosts each (the thin end of the chains):
  // one warp walks them with warp barriers instead of block barriers
  int lw = n_levels + 1;
  while (lw > 1 && lps[lw - 1] - lps[lw - 2] <= 32) --lw;
  for (int lv = 1; lv < lw; ++lv) {
    int a = lps[lv - 1], b = lps[lv];
    for (int s = a + threadIdx.x; s < b; s += CH_T) relax(s);
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    for (int lv = lw; lv <= n_levels; ++lv) {
      const int s = lps[lv - 1] + threadIdx.x;
      if (s < lps[lv]) relax(s);
      __syncwarp();
    }
  }
}


template <typename T>
__global__ void __launch_bounds__(CH_T) k_fill_chain(FieldSet P, int F, const Geom* __restrict__ G,
                                                     const int* __restrict__ geo_list,
                                                     const int* __restrict__ g_cell,
                                                     const uint32_t* __restrict__ g_meta,
                                                     const int* __restrict__ g_dep,
                                                     const int* __restrict__ lev_ptr,
                                                     const T* __restrict__ wtab, int ng,
                                                     const T* __restrict__ part, int* status) {
  pdl_enter();
  chain_walk<T>(P, F, G[geo_list[blockIdx.x]], g_cell, g_meta, g_dep, lev_ptr, wtab, ng, part, status);
}

void launch_fill_chain(int dtype, int dim, int F, void* const* fields, const int* bc_kind,
                       const void* const* bc, const Geom* G, const int* geo_list, int n_list,
                       const int* g_cell, const uint32_t* g_meta, const int* g_dep,
                       const int* lev_ptr, const void* wtab, int ng_total, size_t smem,
                       const void* part, int* status, cudaStream_t s) {
  (void)dim;
  if (n_list <= 0) return;
  FieldSet P;
  for (int f = 0; f < 8; ++f) {
    P.f[f] = f < F ? fields[f] : nullptr;
    P.bc[f] = f < F ? bc[f] : nullptr;
    P.kind[f] = f < F ? bc_kind[f] : 0;
  }
  if (dtype == 0) {
    smem_raise<k_fill_chain<float>>(smem);
    launch(k_fill_chain<float>, n_list, CH_T, smem, s, P, F, G, geo_list, g_cell, g_meta, g_dep, lev_ptr, (const float*)wtab, ng_total, (const float*)part, status);
  } else {
    smem_raise<k_fill_chain<double>>(smem);
    launch(k_fill_chain<double>, n_list, CH_T, smem, s, P, F, G, geo_list, g_cell, g_meta, g_dep, lev_ptr, (const double*)wtab, ng_total, (const double*)part, status);
  }
}

}  // namespace ebr
