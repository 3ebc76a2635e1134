// Adjoint of the fill and the forces: gradient of
// J = sum_b seed_b0 drag_b + seed_b1 lift_b with respect to the fluid field
// values and the boundary data.  For fixed geometry the path is linear, so
// J = sum_(ghost H, slot s, field f) c[f][s][H] * value_f(slot s of H) where
// the force coefficients c follow from the Sec. 6 relations (phi_s and grad
// coefficients in ftab):
//   pressure:     c = -w_H (q . n) alpha_s
//   velocity u_m: c = w_H mu (q_m (beta_s . n) + n_m (q . beta_s))
// with q = seed_0 e_drag + seed_1 e_lift.  With lambda_G = dJ / d phi_G:
//   lambda_G = sum over incidences (H, s) whose slot s is G of
//              c[f][s][H] + [s > 0 and member active] w_(H, s-1) lambda_H,
// processed in reverse level order (consumers H sit in higher levels) from
// per-ghost source lists; then dJ/dx_T is the same sum for a fluid cell T,
// found by probing the ghosts that read T in a fixed order, and
// dJ/db_G = w_(G, s) lambda_G.  Every target sums its sources in a fixed
// order and is written once: no atomics, bitwise reproducible.
#include "ebr_kernels.cuh"
#include "ebr_probe.cuh"

namespace ebr {

struct AdjSet {
  int kind[8];
  void* grad[8];
  void* gbc[8];
};

// The force coefficients in the field type (FP32 fields: from the
// coefficients rounded to float, as the forward forces take them).
template <typename T, int D>
__global__ void k_adj_seed(int F, int4 role, double mu, double dd0, double dd1, double dd2,
                           double dl0, double dl1, double dl2, const double* __restrict__ seed,
                           int ng, const int* __restrict__ g_geo, const double* __restrict__ g_n,
                           const T* __restrict__ ftab, T* __restrict__ sv) {
  pdl_enter();
  constexpr int K = D == 2 ? 3 : 7;
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  int b = g_geo[p];
  const T s0 = (T)seed[2 * b], s1 = (T)seed[2 * b + 1];
  const T dd[3] = {(T)dd0, (T)dd1, (T)dd2}, dl[3] = {(T)dl0, (T)dl1, (T)dl2};
  T q[D], n[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    q[a] = s0 * dd[a] + s1 * dl[a];
    n[a] = (T)g_n[(size_t)a * ng + p];
  }
  const T wG = (T)ftab[p];
  const T muT = (T)mu;
  T qn = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) qn += q[a] * n[a];
  const int vel[3] = {role.x, role.y, role.z};
  const int pidx = role.w;
  for (int f = 0; f < F; ++f) {
    // velocity component of field f (if any), selected without indexing
    bool isv = false;
    T qm = T(0), nm = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (vel[a] == f) { isv = true; qm = q[a]; nm = n[a]; }
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      T c = T(0);
      if (s <= K) {
        if (f == pidx) {
          c = -wG * qn * (T)ftab[(size_t)(1 + s) * ng + p];
        } else if (isv) {
          T bn = T(0), qb = T(0);
#pragma unroll
          for (int a = 0; a < D; ++a) {
            const T beta = (T)ftab[(size_t)(9 + 8 * a + s) * ng + p];
            bn += beta * n[a];
            qb += beta * q[a];
          }
          c = wG * muT * (qm * bn + nm * qb);
        }
      }
      sv[(size_t)(f * 8 + s) * ng + p] = c;
    }
  }
}

void launch_adj_seed(int dtype, int dim, int F, const int* role, double mu, const double* dirs,
                     const double* seed, int ng, const int* g_geo, const double* g_n,
                     const void* ftab, void* sv, cudaStream_t s, int T) {
  if (ng <= 0) return;
  int4 r = make_int4(role[0], role[1], role[2], role[3]);
  double dd[3] = {0, 0, 0}, dl[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) { dd[a] = dirs[a]; dl[a] = dirs[dim + a]; }
  const unsigned nb = (unsigned)((ng + T - 1) / T);
  if (dtype == 0 && dim == 2)
    launch(k_adj_seed<float, 2>, nb, T, 0, s, F, r, mu, dd[0], dd[1], dd[2], dl[0], dl[1], dl[2], seed, ng,
           g_geo, g_n, (const float*)ftab, (float*)sv);
  else if (dtype == 0)
    launch(k_adj_seed<float, 3>, nb, T, 0, s, F, r, mu, dd[0], dd[1], dd[2], dl[0], dl[1], dl[2], seed, ng,
           g_geo, g_n, (const float*)ftab, (float*)sv);
  else if (dim == 2)
    launch(k_adj_seed<double, 2>, nb, T, 0, s, F, r, mu, dd[0], dd[1], dd[2], dl[0], dl[1], dl[2], seed, ng,
           g_geo, g_n, (const double*)ftab, (double*)sv);
  else
    launch(k_adj_seed<double, 3>, nb, T, 0, s, F, r, mu, dd[0], dd[1], dd[2], dl[0], dl[1], dl[2], seed, ng,
           g_geo, g_n, (const double*)ftab, (double*)sv);
}

template <typename T>
__device__ inline T pull_sum(int f, int kind, int j0, int j1, const int* __restrict__ src,
                             const uint32_t* __restrict__ g_meta, const T* __restrict__ wtab,
                             const T* __restrict__ sv, int ng, const T* __restrict__ lam) {
  T acc = T(0);
  for (int j = j0; j < j1; ++j) {
    int e = src[j];
    int q = e >> 3, s = e & 7;
    acc += sv[(size_t)(f * 8 + s) * ng + q];
    if (s > 0 && (meta_active(g_meta[q]) >> (s - 1) & 1u))
      acc += (T)wtab[(size_t)(kind * 8 + s - 1) * ng + q] * lam[(size_t)f * ng + q];
  }
  return acc;
}

template <typename T>
__global__ void k_adj_level(AdjSet A, int F, int p0, int p1, const int* __restrict__ gsrc_ptr,
                            const int* __restrict__ gsrc, const uint32_t* __restrict__ g_meta,
                            const T* __restrict__ wtab, const T* __restrict__ sv, int ng,
                            T* __restrict__ lam) {
  pdl_enter();
  int p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= p1) return;
  for (int f = 0; f < F; ++f)
    lam[(size_t)f * ng + p] = pull_sum<T>(f, A.kind[f], gsrc_ptr[p], gsrc_ptr[p + 1], gsrc, g_meta,
                                          wtab, sv, ng, lam);
}

void launch_adj_level(int dtype, int dim, int F, const int* bc_kind, int p0, int p1,
                      const int* gsrc_ptr, const int* gsrc, const uint32_t* g_meta,
                      const void* wtab, const void* sv, int ng_total, void* lam, cudaStream_t s) {
  (void)dim;
  if (p1 <= p0) return;
  AdjSet A{};
  for (int f = 0; f < F && f < 8; ++f) A.kind[f] = bc_kind[f];
  int n = p1 - p0, T = n < 128 ? 64 : 128;
  if (dtype == 0)
    launch(k_adj_level<float>, (n + T - 1) / T, T, 0, s, A, F, p0, p1, gsrc_ptr, gsrc, g_meta, (const float*)wtab, (const float*)sv, ng_total, (float*)lam);
  else
    launch(k_adj_level<double>, (n + T - 1) / T, T, 0, s, A, F, p0, p1, gsrc_ptr, gsrc, g_meta, (const double*)wtab, (const double*)sv, ng_total, (double*)lam);
}

// Per ghost, grid-wide (one thread per ghost): lambda's start value, the sum
// of the force coefficients of all incidences (in source-list order), and,
// per incidence of the source list, the consumer it stands for (global ghost
// position, -1 when it is the ghost itself or an inactive member) with its
// weights of both kinds.
template <typename T>
__global__ void k_adj_part(int F, int ng, const int* __restrict__ gsrc_ptr, const int* __restrict__ gsrc,
                           const uint32_t* __restrict__ g_meta, const T* __restrict__ wtab,
                           const T* __restrict__ sv, T* __restrict__ lpart, int* __restrict__ cq_g,
                           T* __restrict__ cw_g, int n_src) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  const int j0 = gsrc_ptr[p], j1 = gsrc_ptr[p + 1];
  // every field's sum in registers, each source word read once (each field
  // still adds its sources in list order)
  T acc[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) acc[f] = T(0);
  for (int j = j0; j < j1; ++j) {
    const int e = gsrc[j];
    const size_t col = (size_t)(e & 7) * ng + (e >> 3);
#pragma unroll
    for (int f = 0; f < 8; ++f)
      if (f < F) acc[f] += sv[(size_t)f * 8 * ng + col];
  }
#pragma unroll
  for (int f = 0; f < 8; ++f)
    if (f < F) lpart[(size_t)f * ng + p] = acc[f];
  for (int j = j0; j < j1; ++j) {
    const int e = gsrc[j];
    const int q = e >> 3, sl = e & 7;
    const bool c = sl > 0 && (meta_active(g_meta[q]) >> (sl - 1) & 1u);
    cq_g[j] = c ? q : -1;
    cw_g[j] = c ? (T)wtab[(size_t)(sl - 1) * ng + q] : T(0);
    cw_g[(size_t)n_src + j] = c ? (T)wtab[(size_t)(8 + sl - 1) * ng + q] : T(0);
  }
}

void launch_adj_part(int dtype, int F, int ng, const int* gsrc_ptr, const int* gsrc, const uint32_t* g_meta,
                     const void* wtab, const void* sv, void* lpart, int* cq_g, void* cw_g, int n_src,
                     cudaStream_t s, int T) {
  if (ng <= 0) return;
  if (dtype == 0)
    launch(k_adj_part<float>, (ng + T - 1) / T, T, 0, s, F, ng, gsrc_ptr, gsrc, g_meta, (const float*)wtab, (const float*)sv, (float*)lpart,
                                                     cq_g, (float*)cw_g, n_src);
  else
    launch(k_adj_part<double>, (ng + T - 1) / T, T, 0, s, F, ng, gsrc_ptr, gsrc, g_meta, (const double*)wtab, (const double*)sv, (double*)lpart,
                                                      cq_g, (double*)cw_g, n_src);
}

// One CTA per geometry.  Phase 1: lambda's start values and the geometry's
// slice of the incidence records (from k_adj_part) are copied into shared
// memory.  Phase 2: reverse levels on shared memory only, each ghost adding
// w lambda over its consumers in source-list order.
constexpr int AC_T = 512;

size_t adj_chain_smem(int dtype, int F, int n, int n_src) {
  size_t sz = dtype == 0 ? 4 : 8;
  return (size_t)F * n * sz + (size_t)(2 * n + 2) * sizeof(int) + (size_t)n_src * (sizeof(int) + 2 * sz) + 64;
}

template <typename T>
__global__ void __launch_bounds__(AC_T) k_adj_chain(AdjSet A, int F, const Geom* __restrict__ G,
                                                    const int* __restrict__ geo_list,
                                                    const int* __restrict__ lev_ptr,
                                                    const int* __restrict__ gsrc_ptr,
                                                    const T* __restrict__ lpart,
                                                    const int* __restrict__ cq_g,
                                                    const T* __restrict__ cw_g, int n_src, int ng,
                                                    T* __restrict__ lam) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem[];
  const Geom& g = G[geo_list[blockIdx.x]];
  const int n = g.n_ghost, g0 = g.ghost_off;
  const int n_levels = g.n_levels;     // in a register: the kernel stores to global memory
  const int j0g = gsrc_ptr[g0];
  const int nsrc = gsrc_ptr[g0 + n] - j0g;
  T* L = reinterpret_cast<T*>(smem);                         // [F][n]
  T* cw = L + (size_t)F * n;                                 // [2][nsrc]
  int* cq = reinterpret_cast<int*>(cw + (size_t)2 * nsrc);   // [nsrc] local consumer or -1
  int* cptr = cq + nsrc;                                     // [n + 1]
  int* lps = cptr + n + 1;                                   // [n_levels + 1]
  {
    const int* lp = lev_ptr + g.lev_off;
    for (int q = threadIdx.x; q <= n_levels; q += AC_T) lps[q] = lp[q] - g0;
  }
  // phase 1: start values, source offsets and the incidence records (the
  // loops unrolled so that several items' loads are in flight together)
#pragma unroll 4
  for (int s = threadIdx.x; s < n; s += AC_T) {
    const int p = g0 + s;
    cptr[s] = gsrc_ptr[p] - j0g;
#pragma unroll
    for (int f = 0; f < 8; ++f)
      if (f < F) L[(size_t)f * n + s] = lpart[(size_t)f * ng + p];
  }
  if (threadIdx.x == 0) cptr[n] = nsrc;
#pragma unroll 4
  for (int o = threadIdx.x; o < nsrc; o += AC_T) {
    const int q = cq_g[j0g + o];
    cq[o] = q >= 0 ? q - g0 : -1;
    cw[o] = cw_g[j0g + o];
    cw[nsrc + o] = cw_g[(size_t)n_src + j0g + o];
  }
  __syncthreads();
  // phase 2: reverse levels
  // every field's sum in registers, the sources walked once: the loads of
  // all fields are issued together and no store intervenes (each field
  // still sums its sources in the same order, so the bits are the same)
  auto relax = [&](int s) {
    T v[8];
#pragma unroll
    for (int f = 0; f < 8; ++f)
      if (f < F) v[f] = L[(size_t)f * n + s];
    for (int o = cptr[s]; o < cptr[s + 1]; ++o) {
      const int q = cq[o];
      if (q < 0) continue;
      const T w0 = cw[o], w1 = cw[(size_t)nsrc + o];
#pragma unroll
      for (int f = 0; f < 8; ++f)
        if (f < F) v[f] += (A.kind[f] ? w1 : w0) * L[(size_t)f * n + q];
    }
#pragma unroll
    for (int f = 0; f < 8; ++f)
      if (f < F) L[(size_t)f * n + s] = v[f];
  };
  // the deepest levels (lw.., at most 32 ghosts each) come first: one warp
  // walks them with warp barriers, then the block takes the wide levels
  int lw = n_levels + 1;
  while (lw > 1 && lps[lw - 1] - lps[lw - 2] <= 32) --lw;
  if (threadIdx.x < 32) {
    for (int lv = n_levels; lv >= lw; --lv) {
      const int s = lps[lv - 1] + threadIdx.x;
      if (s < lps[lv]) relax(s);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int lv = lw - 1; lv >= 1; --lv) {
    int a = lps[lv - 1], b = lps[lv];
    for (int s = a + threadIdx.x; s < b; s += AC_T) relax(s);
    __syncthreads();
  }
  for (int s = threadIdx.x; s < n; s += AC_T)
    for (int f = 0; f < F; ++f) lam[(size_t)f * ng + g0 + s] = L[(size_t)f * n + s];
}

void launch_adj_chain(int dtype, int dim, int F, const int* bc_kind, const Geom* G,
                      const int* geo_list, int n_list, const int* lev_ptr, const int* gsrc_ptr,
                      const void* lpart, const int* cq_g, const void* cw_g, int n_src,
                      int ng_total, void* lam, size_t smem, cudaStream_t s) {
  (void)dim;
  if (n_list <= 0) return;
  AdjSet A{};
  for (int f = 0; f < F && f < 8; ++f) A.kind[f] = bc_kind[f];
  if (dtype == 0) {
    smem_raise<k_adj_chain<float>>(smem);
    launch(k_adj_chain<float>, n_list, AC_T, smem, s, A, F, G, geo_list, lev_ptr, gsrc_ptr, (const float*)lpart, cq_g,
                                                  (const float*)cw_g, n_src, ng_total, (float*)lam);
  } else {
    smem_raise<k_adj_chain<double>>(smem);
    launch(k_adj_chain<double>, n_list, AC_T, smem, s, A, F, G, geo_list, lev_ptr, gsrc_ptr, (const double*)lpart,
                                                   cq_g, (const double*)cw_g, n_src, ng_total, (double*)lam);
  }
}

// Gradient of the fluid cells.  Incidence (ghost p, member k) with a fluid
// member T probes the ghosts that read T in a fixed order; only the first of
// them owns T and pulls every source (force coefficient + weight x lambda) in
// that order, so each fluid cell is written once, without atomics, bitwise
// reproducibly.
template <typename T>
__global__ void k_adj_fluid(AdjSet A, int F, int ng, const Geom* __restrict__ G,
                            const int* __restrict__ g_geo, const int* __restrict__ g_cell,
                            const uint32_t* __restrict__ g_meta, const int8_t* __restrict__ tags,
                            const int* __restrict__ pos_of_cell, int rmax,
                            const T* __restrict__ wtab, const T* __restrict__ sv,
                            const T* __restrict__ lam, int accumulate, int kmax) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int p = i / kmax, k = i - p * kmax;
  if (p >= ng) return;
  const Geom& g = G[g_geo[p]];
  if (k >= stencil_k(g.dim)) return;
  int gijk[3], tijk[3];
  cell_ijk3(g, g_cell[p], gijk);
  member_ijk(g, gijk, g_meta[p], k, tijk);
  const int8_t* tg = tags + g.cell_off;
  const int* pc = pos_of_cell + g.cell_off;
  if (!in_grid(g, tijk) || tg[cell_lin(g, tijk)] != 0) return;
  // one pass: the first source met decides ownership; a non-owner stops there
  // fields up to 8: fixed-trip loops keep acc[] in registers
  T acc[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) acc[f] = T(0);
  bool first = true, owner = false;
  probe_sources(g, tijk, tg, pc, g_cell, g_meta, rmax, [&](int q, int slot) {
    if (first) {
      first = false;
      owner = (q == p && slot == k + 1);
      if (!owner) return false;
    }
    bool act = meta_active(g_meta[q]) >> (slot - 1) & 1u;
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      if (f < F) {
        acc[f] += sv[(size_t)(f * 8 + slot) * ng + q];
        if (act) acc[f] += (T)wtab[(size_t)(A.kind[f] * 8 + slot - 1) * ng + q] * lam[(size_t)f * ng + q];
      }
    }
    return true;
  });
  if (!owner) return;
  long long c = g.cell_off + cell_lin(g, tijk);
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    if (f < F) {
      T* gr = static_cast<T*>(A.grad[f]);
      if (accumulate) gr[c] += acc[f]; else gr[c] = acc[f];
    }
  }
}

void launch_adj_fluid(int dtype, int F, const int* bc_kind, int ng, const Geom* G, const int* g_geo,
                      const int* g_cell, const uint32_t* g_meta, const int8_t* tags,
                      const int* pos_of_cell, int rmax, const void* wtab, const void* sv,
                      const void* lam, void* const* grad, int accumulate, int kmax, cudaStream_t s, int T) {
  if (ng <= 0) return;
  AdjSet A{};
  for (int f = 0; f < F && f < 8; ++f) { A.kind[f] = bc_kind[f]; A.grad[f] = grad[f]; }
  // one thread per (ghost, member): K = 3 in 2D, 7 in 3D (kmax covers both)
  int n = ng * kmax;
  if (dtype == 0)
    launch(k_adj_fluid<float>, (n + T - 1) / T, T, 0, s, A, F, ng, G, g_geo, g_cell, g_meta, tags, pos_of_cell, rmax, (const float*)wtab, (const float*)sv, (const float*)lam, accumulate, kmax);
  else
    launch(k_adj_fluid<double>, (n + T - 1) / T, T, 0, s, A, F, ng, G, g_geo, g_cell, g_meta, tags, pos_of_cell, rmax, (const double*)wtab, (const double*)sv, (const double*)lam, accumulate, kmax);
}

// Fluid targets in two passes at reach 1: the probe needs no lambda, so it
// can run beside the seed and chain kernels; the pull then sums in the
// probe's order, which gives the same bits as the one-pass kernel above.
// Per incidence i = (ghost p, member k): fcnt[i] = sources recorded when the
// incidence owns its target (the first source in probe order), else 0;
// fcell[i] = the target's global cell; fsrc[i * cap + e] = q << 4 | slot << 1
// | active, in probe order.
__global__ void k_adj_fprobe(int ng, const Geom* __restrict__ G, const int* __restrict__ g_geo,
                             const int* __restrict__ g_cell, const uint32_t* __restrict__ g_meta,
                             const int8_t* __restrict__ tags, const int* __restrict__ pos_of_cell, int kmax,
                             int cap, int* __restrict__ fcnt, int* __restrict__ fcell, int* __restrict__ fsrc,
                             int* status) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = i / kmax, k = i - p * kmax;
  if (p >= ng) return;
  const Geom& g = G[g_geo[p]];
  int n = 0;
  if (k < stencil_k(g.dim)) {
    int gijk[3], tijk[3];
    cell_ijk3(g, g_cell[p], gijk);
    member_ijk(g, gijk, g_meta[p], k, tijk);
    const int8_t* tg = tags + g.cell_off;
    const int* pc = pos_of_cell + g.cell_off;
    if (in_grid(g, tijk) && tg[cell_lin(g, tijk)] == 0) {
      bool first = true, owner = false;
      int* out = fsrc + (size_t)i * cap;
      probe_sources(g, tijk, tg, pc, g_cell, g_meta, 1, [&](int q, int slot) {
        if (first) {
          first = false;
          owner = (q == p && slot == k + 1);
          if (!owner) return false;
        }
        const int act = (int)((meta_active(g_meta[q]) >> (slot - 1)) & 1u);
        if (n < cap) out[n] = (q << 4) | (slot << 1) | act;
        ++n;
        return true;
      });
      if (!owner) n = 0;
      if (n > cap) {
        set_status(status, S_EINVAL);
        n = cap;
      }
      if (n > 0) fcell[i] = (int)(g.cell_off + cell_lin(g, tijk));
    }
  }
  fcnt[i] = n;
}

template <typename T>
__global__ void k_adj_fpull(AdjSet A, int F, int ng, int n_inc, int cap, const int* __restrict__ fcnt,
                            const int* __restrict__ fcell, const int* __restrict__ fsrc,
                            const T* __restrict__ wtab, const T* __restrict__ sv,
                            const T* __restrict__ lam, int accumulate) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inc) return;
  const int n = fcnt[i];
  if (n <= 0) return;
  T acc[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) acc[f] = T(0);
  const int* src = fsrc + (size_t)i * cap;
  for (int e = 0; e < n; ++e) {
    const int w = src[e];
    const int q = w >> 4, slot = (w >> 1) & 7;
    const bool act = w & 1;
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      if (f < F) {
        acc[f] += sv[(size_t)(f * 8 + slot) * ng + q];
        if (act) acc[f] += (T)wtab[(size_t)(A.kind[f] * 8 + slot - 1) * ng + q] * lam[(size_t)f * ng + q];
      }
    }
  }
  const long long c = fcell[i];
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    if (f < F) {
      T* gr = static_cast<T*>(A.grad[f]);
      if (accumulate) gr[c] += acc[f]; else gr[c] = acc[f];
    }
  }
}

int adj_fluid_cap(int dim) { return dim == 2 ? 8 : 26; }

void launch_adj_fprobe(int ng, const Geom* G, const int* g_geo, const int* g_cell, const uint32_t* g_meta,
                       const int8_t* tags, const int* pos_of_cell, int kmax, int cap, int* fcnt, int* fcell,
                       int* fsrc, int* status, cudaStream_t s, int T) {
  if (ng <= 0) return;
  const int n = ng * kmax;
  launch(k_adj_fprobe, (n + T - 1) / T, T, 0, s, ng, G, g_geo, g_cell, g_meta, tags, pos_of_cell, kmax, cap, fcnt,
                                             fcell, fsrc, status);
}

void launch_adj_fpull(int dtype, int F, const int* bc_kind, int ng, int kmax, int cap, const int* fcnt,
                      const int* fcell, const int* fsrc, const void* wtab, const void* sv, const void* lam,
                      void* const* grad, int accumulate, cudaStream_t s, int T) {
  if (ng <= 0) return;
  AdjSet A{};
  for (int f = 0; f < F && f < 8; ++f) { A.kind[f] = bc_kind[f]; A.grad[f] = grad[f]; }
  const int n = ng * kmax;
  if (dtype == 0)
    launch(k_adj_fpull<float>, (n + T - 1) / T, T, 0, s, A, F, ng, n, cap, fcnt, fcell, fsrc, (const float*)wtab,
           (const float*)sv, (const float*)lam, accumulate);
  else
    launch(k_adj_fpull<double>, (n + T - 1) / T, T, 0, s, A, F, ng, n, cap, fcnt, fcell, fsrc, (const double*)wtab,
           (const double*)sv, (const double*)lam, accumulate);
}

template <typename T>
__global__ void k_adj_bc(AdjSet A, int F, int ng, const Geom* __restrict__ G,
                         const int* __restrict__ g_geo, const int* __restrict__ g_cell,
                         const T* __restrict__ wtab, const T* __restrict__ lam, int accumulate) {
  pdl_enter();
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  long long c = G[g_geo[p]].cell_off + g_cell[p];
  for (int f = 0; f < F; ++f) {
    T v = (T)wtab[(size_t)(A.kind[f] * 8 + 7) * ng + p] * lam[(size_t)f * ng + p];
    T* gb = static_cast<T*>(A.gbc[f]);
    if (accumulate) gb[p] += v; else gb[p] = v;
    if (!accumulate) static_cast<T*>(A.grad[f])[c] = T(0);
  }
}

void launch_adj_bc(int dtype, int F, const int* bc_kind, int ng, const Geom* G, const int* g_geo,
                   const int* g_cell, const void* wtab, const void* lam, void* const* grad_bc,
                   void* const* grad, int accumulate, cudaStream_t s, int T) {
  if (ng <= 0) return;
  AdjSet A{};
  for (int f = 0; f < F && f < 8; ++f) { A.kind[f] = bc_kind[f]; A.gbc[f] = grad_bc[f]; A.grad[f] = grad[f]; }
  if (dtype == 0)
    launch(k_adj_bc<float>, (ng + T - 1) / T, T, 0, s, A, F, ng, G, g_geo, g_cell, (const float*)wtab, (const float*)lam, accumulate);
  else
    launch(k_adj_bc<double>, (ng + T - 1) / T, T, 0, s, A, F, ng, G, g_geo, g_cell, (const double*)wtab, (const double*)lam, accumulate);
}

}  // namespace ebr
