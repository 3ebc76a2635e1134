// Many-field reconstruction in the field-minor ("packed") layout: one array
// [cells][F] whose F values of a cell are contiguous, so that the stencil
// gather of one ghost reads F consecutive values per member (a 128-byte line
// per 32 FP32 fields) instead of one 4-byte value per field array.
//
// Forward (Sec. 3.2 level order, closed forms of Secs. 4-5 through the weight
// table): one CTA per (geometry, chunk of 32 fields), a warp per ghost and a
// lane per field.  Fields are independent, so chunks never wait on each other;
// inside a CTA the dependency chain is ordered by block barriers.
//   phase 1: every ghost, in parallel: boundary term + fluid members, written
//            in place (final for ghosts without a ghost member);
//   phase 2: levels 2.. in order: add the terms of the ghost members.
//
// Adjoint (vector-Jacobian product of the in-place fill, field-minor).  On
// entry cot holds dJ/d(field after the fill); on exit dJ/d(field before the
// fill): ghost entries 0 (the fill overwrites them), fluid entries
// incremented by the transposed weights, and grad_bc = dJ/d(boundary data).
//   chain: reverse levels, lambda_G = cot_G + sum over consumers (H, k) of
//          w_(H,k) lambda_H, from the per-ghost source lists;
//   fluid: for every active (ghost, member) incidence with a fluid member T,
//          the warp probes the ghosts that read T (lane per probe cell, fixed
//          order); the first active incidence owns T and adds all of them,
//          so every target is written once, without atomics.
#include "ebr_kernels.cuh"
#include "ebr_probe.cuh"

namespace ebr {

constexpr int PK_T = 256;        // 8 warps per CTA
constexpr int PK_BATCH = 4;      // ghosts per warp per step of phase 1 (loads in flight)

__device__ __forceinline__ int kind_of(const KindBits& kb, int f) {
  return (kb.w[f >> 5] >> (f & 31)) & 1u;
}

__device__ __forceinline__ long long member_lin(const Geom& g, int cell, uint32_t m, int k) {
  int o[3];
  stencil_off(g.dim, k, o);
  long long off = (long long)o[0] * meta_r(m, 0) * meta_e(m, 0) +
                  (long long)g.n[0] * (o[1] * meta_r(m, 1) * meta_e(m, 1));
  if (g.dim == 3) off += (long long)g.n[0] * g.n[1] * (o[2] * meta_r(m, 2) * meta_e(m, 2));
  return cell + off;
}

template <typename T, int K>
__device__ __forceinline__ void pfill_body(const Geom& g, T* __restrict__ fld, const T* __restrict__ bc,
                                           int F, const KindBits& kb,
                                           const int* __restrict__ g_cell,
                                           const uint32_t* __restrict__ g_meta,
                                           const int* __restrict__ lev_ptr,
                                           const double* __restrict__ wtab, int ng, int* status) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = PK_T / 32;
  const int f = blockIdx.y * 32 + lane;
  const bool on = f < F;
  const int fo = on ? f : 0;
  const int kind = on ? kind_of(kb, f) : 0;
  const int n = g.n_ghost, g0 = g.ghost_off;
  T* base = fld + g.cell_off * (long long)F + fo;
  bool bad = false;
  // phase 1: boundary term + fluid members of every ghost
  for (int s0 = warp; s0 < n; s0 += nw * PK_BATCH) {
    T acc[PK_BATCH];
    long long dst[PK_BATCH];
#pragma unroll
    for (int u = 0; u < PK_BATCH; ++u) {
      int s = s0 + u * nw;
      acc[u] = T(0);
      dst[u] = -1;
      if (s < n) {
        int p = g0 + s;
        int cell = g_cell[p];
        uint32_t m = g_meta[p];
        uint32_t act = meta_active(m) & ~meta_depmask(m);
        T a = (T)wtab[(size_t)(kind * 8 + 7) * ng + p] * bc[(long long)p * F + fo];
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (act >> k & 1u)
            a += (T)wtab[(size_t)(kind * 8 + k) * ng + p] * base[member_lin(g, cell, m, k) * F];
        acc[u] = a;
        dst[u] = (long long)cell * F;
      }
    }
#pragma unroll
    for (int u = 0; u < PK_BATCH; ++u)
      if (dst[u] >= 0 && on) {
        base[dst[u]] = acc[u];
        if (!isfinite((double)acc[u])) bad = true;
      }
  }
  __syncthreads();
  // phase 2: ghost members, level by level
  const int* lp = lev_ptr + g.lev_off;
  for (int lv = 2; lv <= g.n_levels; ++lv) {
    int a = lp[lv - 1], b = lp[lv];
    for (int p = a + warp; p < b; p += nw) {
      int cell = g_cell[p];
      uint32_t m = g_meta[p];
      uint32_t dm = meta_depmask(m) & meta_active(m);
      T v = base[(long long)cell * F];
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (dm >> k & 1u)
          v += (T)wtab[(size_t)(kind * 8 + k) * ng + p] * base[member_lin(g, cell, m, k) * F];
      if (on) {
        base[(long long)cell * F] = v;
        if (!isfinite((double)v)) bad = true;
      }
    }
    __syncthreads();
  }
  if (bad) set_status(status, S_ENONFINITE);
}

template <typename T>
__global__ void __launch_bounds__(PK_T) k_pfill(T* __restrict__ fld, const T* __restrict__ bc, int F,
                                                const __grid_constant__ KindBits kb,
                                                const Geom* __restrict__ G,
                                                const int* __restrict__ geo_list,
                                                const int* __restrict__ g_cell,
                                                const uint32_t* __restrict__ g_meta,
                                                const int* __restrict__ lev_ptr,
                                                const double* __restrict__ wtab, int ng,
                                                int* status) {
  const Geom& g = G[geo_list[blockIdx.x]];
  if (g.dim == 2) pfill_body<T, 3>(g, fld, bc, F, kb, g_cell, g_meta, lev_ptr, wtab, ng, status);
  else pfill_body<T, 7>(g, fld, bc, F, kb, g_cell, g_meta, lev_ptr, wtab, ng, status);
}

void launch_pfill(int dtype, int F, void* fld, const void* bc, const KindBits& kb, const Geom* G,
                  const int* geo_list, int n_list, const int* g_cell, const uint32_t* g_meta,
                  const int* lev_ptr, const double* wtab, int ng, int* status, cudaStream_t s) {
  if (n_list <= 0 || F <= 0) return;
  dim3 grid(n_list, (F + 31) / 32);
  if (dtype == 0)
    k_pfill<float><<<grid, PK_T, 0, s>>>((float*)fld, (const float*)bc, F, kb, G, geo_list, g_cell,
                                          g_meta, lev_ptr, wtab, ng, status);
  else
    k_pfill<double><<<grid, PK_T, 0, s>>>((double*)fld, (const double*)bc, F, kb, G, geo_list, g_cell,
                                           g_meta, lev_ptr, wtab, ng, status);
}

// reverse levels: lambda of every ghost (lamP [ng][F]), ghost cotangents
// cleared, boundary-data gradients
template <typename T>
__global__ void __launch_bounds__(PK_T) k_padj_chain(T* __restrict__ cot, T* __restrict__ lamP,
                                                     T* __restrict__ gbc, int F,
                                                     const __grid_constant__ KindBits kb,
                                                     const Geom* __restrict__ G,
                                                     const int* __restrict__ geo_list,
                                                     const int* __restrict__ g_cell,
                                                     const uint32_t* __restrict__ g_meta,
                                                     const int* __restrict__ lev_ptr,
                                                     const int* __restrict__ gsrc_ptr,
                                                     const int* __restrict__ gsrc,
                                                     const double* __restrict__ wtab, int ng) {
  const Geom& g = G[geo_list[blockIdx.x]];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = PK_T / 32;
  const int f = blockIdx.y * 32 + lane;
  const bool on = f < F;
  const int fo = on ? f : 0;
  const int kind = on ? kind_of(kb, f) : 0;
  T* cbase = cot + g.cell_off * (long long)F + fo;
  const int* lp = lev_ptr + g.lev_off;
  for (int lv = g.n_levels; lv >= 1; --lv) {
    int a = lp[lv - 1], b = lp[lv];
    for (int p = a + warp; p < b; p += nw) {
      long long c = (long long)g_cell[p] * F;
      T lam = cbase[c];
      for (int j = gsrc_ptr[p]; j < gsrc_ptr[p + 1]; ++j) {
        int e = gsrc[j];
        int q = e >> 3, sl = e & 7;
        if (sl > 0 && (meta_active(g_meta[q]) >> (sl - 1) & 1u))
          lam += (T)wtab[(size_t)(kind * 8 + sl - 1) * ng + q] * lamP[(long long)q * F + fo];
      }
      if (on) {
        lamP[(long long)p * F + f] = lam;
        gbc[(long long)p * F + f] = (T)wtab[(size_t)(kind * 8 + 7) * ng + p] * lam;
        cbase[c] = T(0);
      }
    }
    __syncthreads();
  }
}

// fluid targets: a warp per (ghost, member) incidence over all geometries
template <typename T>
__global__ void __launch_bounds__(PK_T) k_padj_fluid(T* __restrict__ cot, const T* __restrict__ lamP,
                                                     int F, const __grid_constant__ KindBits kb,
                                                     int ng, int kmax,
                                                     const Geom* __restrict__ G,
                                                     const int* __restrict__ g_geo,
                                                     const int* __restrict__ g_cell,
                                                     const uint32_t* __restrict__ g_meta,
                                                     const int8_t* __restrict__ tags,
                                                     const int* __restrict__ pos_of_cell, int R,
                                                     const double* __restrict__ wtab) {
  const int lane = threadIdx.x & 31;
  const long long inc = ((long long)blockIdx.x * PK_T + threadIdx.x) >> 5;
  if (inc >= (long long)ng * kmax) return;
  const int p = (int)(inc / kmax), k = (int)(inc - (long long)p * kmax);
  const Geom& g = G[g_geo[p]];
  if (k >= stencil_k(g.dim)) return;
  const uint32_t mp = g_meta[p];
  if (!(meta_active(mp) >> k & 1u)) return;
  int gijk[3], tijk[3];
  cell_ijk3(g, g_cell[p], gijk);
  member_ijk(g, gijk, mp, k, tijk);
  const int8_t* tg = tags + g.cell_off;
  const int* pc = pos_of_cell + g.cell_off;
  if (!in_grid(g, tijk) || tg[cell_lin(g, tijk)] != 0) return;
  // probe cells in the fixed order dz, dy, dx (outer to inner), lane per cell
  const int Rz = g.dim == 3 ? R : 0;
  const int wx = 2 * R + 1, wy = 2 * R + 1, nbox = wx * wy * (2 * Rz + 1);
  const int K = stencil_k(g.dim);
  // fields in groups of 128 (4 per lane); the probe is repeated per group
  for (int f0 = 0; f0 < F; f0 += 128) {
    const int nchunk = min(4, (F - f0 + 31) / 32);
    T acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = T(0);
    bool decided = false;
    for (int b0 = 0; b0 < nbox; b0 += 32) {
      int bi = b0 + lane;
      int q = -1, slot = 0;
      if (bi < nbox) {
        int dx = bi % wx - R, r1 = bi / wx;
        int dy = r1 % wy - R, dz = r1 / wy - Rz;
        if (dx != 0 || dy != 0 || dz != 0) {
          int hijk[3] = {tijk[0] - dx, tijk[1] - dy, tijk[2] - dz};
          if (in_grid(g, hijk)) {
            int hc = cell_lin(g, hijk);
            int8_t t = tg[hc];
            if (t == 2 || t == -2) {
              int qq = pc[hc];
              uint32_t m = g_meta[qq];
              int dd[3] = {dx, dy, dz};
              for (int kk = 0; kk < K; ++kk) {
                int o[3];
                stencil_off(g.dim, kk, o);
                bool hit = true;
                for (int a = 0; a < g.dim; ++a)
                  if (o[a] * meta_r(m, a) * meta_e(m, a) != dd[a]) hit = false;
                if (hit && (meta_active(m) >> kk & 1u)) { q = qq; slot = kk + 1; }
              }
            }
          }
        }
      }
      unsigned hits = __ballot_sync(0xffffffffu, q >= 0);
      if (!decided && hits) {
        int first = __ffs(hits) - 1;
        int q0 = __shfl_sync(0xffffffffu, q, first), s0 = __shfl_sync(0xffffffffu, slot, first);
        if (q0 != p || s0 != k + 1) return;     // another incidence owns T (warp-uniform)
        decided = true;
      }
      while (hits) {
        int h = __ffs(hits) - 1;
        hits &= hits - 1;
        int qh = __shfl_sync(0xffffffffu, q, h), sh = __shfl_sync(0xffffffffu, slot, h);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          int f = f0 + c * 32 + lane;
          if (c < nchunk && f < F) {
            int kd = kind_of(kb, f);
            acc[c] += (T)wtab[(size_t)(kd * 8 + sh - 1) * ng + qh] * lamP[(long long)qh * F + f];
          }
        }
      }
    }
    if (!decided) return;
    T* dst = cot + (g.cell_off + cell_lin(g, tijk)) * (long long)F;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int f = f0 + c * 32 + lane;
      if (c < nchunk && f < F) dst[f] += acc[c];
    }
  }
}

void launch_padj(int dtype, int F, void* cot, void* lamP, void* gbc, const KindBits& kb,
                 const Geom* G, const int* geo_list, int n_list, int ng, int kmax, const int* g_geo,
                 const int* g_cell, const uint32_t* g_meta, const int* lev_ptr, const int* gsrc_ptr,
                 const int* gsrc, const int8_t* tags, const int* pos_of_cell, int R,
                 const double* wtab, cudaStream_t s, int phase) {
  if (F <= 0 || ng <= 0) return;
  if (phase == 0) {
    if (n_list <= 0) return;
    dim3 grid(n_list, (F + 31) / 32);
    if (dtype == 0)
      k_padj_chain<float><<<grid, PK_T, 0, s>>>((float*)cot, (float*)lamP, (float*)gbc, F, kb, G,
                                                geo_list, g_cell, g_meta, lev_ptr, gsrc_ptr, gsrc,
                                                wtab, ng);
    else
      k_padj_chain<double><<<grid, PK_T, 0, s>>>((double*)cot, (double*)lamP, (double*)gbc, F, kb, G,
                                                 geo_list, g_cell, g_meta, lev_ptr, gsrc_ptr, gsrc,
                                                 wtab, ng);
  } else {
    long long warps = (long long)ng * kmax;
    long long blocks = (warps * 32 + PK_T - 1) / PK_T;
    if (dtype == 0)
      k_padj_fluid<float><<<(unsigned)blocks, PK_T, 0, s>>>((float*)cot, (const float*)lamP, F, kb, ng,
                                                           kmax, G, g_geo, g_cell, g_meta, tags,
                                                           pos_of_cell, R, wtab);
    else
      k_padj_fluid<double><<<(unsigned)blocks, PK_T, 0, s>>>((double*)cot, (const double*)lamP, F, kb,
                                                            ng, kmax, G, g_geo, g_cell, g_meta, tags,
                                                            pos_of_cell, R, wtab);
  }
}

}  // namespace ebr
