// Dependency DAG, topological levels and canonical order (Sec. 3.2); per-ghost
// coefficient tables (Secs. 4-6); transposed incidence lists for the adjoint.
#include "ebr_kernels.cuh"
#include "ebr_probe.cuh"

namespace ebr {

// position of every ghost cell in the ghost arrays; src_cnt (optional): the
// ghost-source counts set to 1 (each ghost is its own first source);
// iface_tag (optional): the final tag of every interface cell, written to the
// tag array
__global__ void k_poscell(const Geom* __restrict__ G, int ng, const int* __restrict__ cell,
                          const int* __restrict__ geo, const int* __restrict__ pos_of,
                          int* __restrict__ pos_of_cell, int* __restrict__ src_cnt, int n_iface,
                          const int* __restrict__ iface_cell, const int* __restrict__ iface_geo,
                          const int8_t* __restrict__ iface_tag, int8_t* __restrict__ tags) {
  pdl_enter();
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (iface_tag && s < n_iface) tags[G[iface_geo[s]].cell_off + iface_cell[s]] = iface_tag[s];
  if (s >= ng) return;
  pos_of_cell[G[geo[s]].cell_off + cell[s]] = pos_of ? pos_of[s] : s;
  if (src_cnt) src_cnt[s] = 1;
}

void launch_poscell(const Geom* G, int ng, const int* cell, const int* geo, const int* pos_of,
                    int* pos_of_cell, int* src_cnt, cudaStream_t s, int n_iface, const int* iface_cell,
                    const int* iface_geo, const int8_t* iface_tag, int8_t* tags) {
  const int n = std::max(ng, iface_tag ? n_iface : 0);
  if (n <= 0) return;
  launch(k_poscell, (n + 255) / 256, 256, 0, s, G, ng, cell, geo, pos_of, pos_of_cell, src_cnt, n_iface,
         iface_cell, iface_geo, iface_tag, tags);
}

// Stencil members: validate (inside the grid, not tag 1), active mask (the
// structurally active members of the meta word -- n_i != 0 along every offset
// axis -- that lie in the grid), dependencies on ghost members.  A member
// tagged +-2 in the caller's tag buffer is a dependency only when it is a
// ghost of this plan (ghost_slot_of); any other +-2 tag (the buffer was
// edited after planning) sets EBR_ESHAPE and adds no edge, so no position
// read from pos_of_cell is used unchecked.
__global__ void k_deps(const Geom* __restrict__ G, int ng, const int* __restrict__ gs_cell,
                       const int* __restrict__ gs_geo, uint32_t* __restrict__ gs_meta,
                       const int8_t* __restrict__ tags, const int* __restrict__ pos_of_cell,
                       int* __restrict__ dep, int* status) {
  pdl_enter();
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ng) return;
  const Geom& g = G[gs_geo[s]];
  int ijk[3];
  cell_ijk3(g, gs_cell[s], ijk);
  const uint32_t m0 = gs_meta[s];
  const uint32_t pre = meta_active(m0);
  uint32_t m = m0 & ~((127u << 15) | (127u << 23));
  const int K = stencil_k(g.dim);
  uint32_t active = 0, depm = 0;
  for (int k = 0; k < MAXK; ++k) {
    int d = -1;
    if (k < K) {
      int mijk[3];
      member_ijk(g, ijk, m, k, mijk);
      if (!in_grid(g, mijk)) {
        set_status(status, S_ESTENCIL_OOB);
      } else {
        const bool act = pre >> k & 1u;
        long long mc = g.cell_off + cell_lin(g, mijk);
        int8_t t = tags[mc];
        if (t == 1) set_status(status, S_ESTENCIL_SOLID);
        if (act) active |= 1u << k;
        if (act && (t == 2 || t == -2)) {
          d = ghost_slot_of(g, cell_lin(g, mijk), pos_of_cell + g.cell_off, gs_cell);
          if (d >= 0) depm |= 1u << k;
          else set_status(status, S_ESHAPE);
        }
      }
    }
    dep[(size_t)k * ng + s] = d;
  }
  gs_meta[s] = m | (active << 15) | (depm << 23);
}

void launch_deps(const Geom* G, int ng, const int* gs_cell, const int* gs_geo, uint32_t* gs_meta,
                 const int8_t* tags, const int* pos_of_cell, int* dep, int* status, cudaStream_t s, int T) {
  if (ng <= 0) return;
  launch(k_deps, (ng + T - 1) / T, T, 0, s, G, ng, gs_cell, gs_geo, gs_meta, tags, pos_of_cell, dep, status);
}

// One CTA per geometry, integer arithmetic only.  Geometries whose arrays fit
// in shared memory run a layered topological sort there: consumer lists from
// the dependencies, in-degree counters, and one frontier per level (a ghost
// enters level L + 1 when the last of its dependencies is placed in level L,
// so its level is 1 + the largest level among its dependencies, whatever the
// thread schedule); each level touches only its frontier.  Larger geometries
// sweep on global memory: in sweep L a ghost whose dependencies all carry
// levels in [1, L-1] receives level L (a level written in the same sweep
// reads as "not ready").  Then a stable counting sort by level gives the
// canonical position (level, index) of every ghost: in shared memory one
// pass per chunk (warps in order, __match_any_sync within a warp), else one
// block scan per level.
constexpr int LV_T = 1024;
constexpr int LV_W = LV_T / 32;  // warps per CTA
constexpr int LV_NL = 64;        // levels ranked with per-warp counts (more: warp by warp)

// shared-memory ints of the fast path: levels, local dependencies [K][n],
// in-degrees, consumer offsets [n + 1], consumers [K][n], two frontiers
__host__ __device__ inline long long levels_smem_ints(int K, int n) { return (long long)(2 * K + 5) * n + 1; }

size_t levels_smem(int dim, int n) {
  return (size_t)levels_smem_ints(stencil_k(dim), n) * sizeof(int) + 64;
}

__global__ void __launch_bounds__(LV_T, 2) k_levels(const Geom* __restrict__ G, int B,
                                                 const int* __restrict__ dep, int ng_total,
                                                 int* __restrict__ level, int* __restrict__ order_pos,
                                                 int* __restrict__ lev_ptr, int* __restrict__ n_levels,
                                                 int smem_ints, int* status) {
  pdl_enter();
  extern __shared__ int sm[];
  __shared__ int sh_cnt3[3];
  __shared__ int sh_warp[32];
  __shared__ int sh_wl[LV_W][LV_NL];          // per-warp counts of each level (ranking)
  __shared__ int sh_tot[LV_NL];               // chunk total of each level
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    const Geom& g = G[b];
    const int g0 = g.ghost_off, n = g.n_ghost;
    const int K = stencil_k(g.dim);
    const bool fast = levels_smem_ints(K, n) <= smem_ints;
    int* lp = lev_ptr + g.lev_off;
    int* lvl = fast ? sm : level + g0;
    int* dl = sm + n;                          // [K][n] local dependencies (fast path)
#pragma unroll 4
    for (int s = threadIdx.x; s < n; s += LV_T) {
      lvl[s] = 0;
      if (fast)
        for (int k = 0; k < K; ++k) {
          // k_deps only writes positions of this geometry's ghosts; the range
          // check keeps every shared-memory index in [0, n) regardless
          int d = dep[(size_t)k * ng_total + g0 + s];
          const bool in = d >= g0 && d < g0 + n;
          if (d >= 0 && !in) set_status(status, S_ESHAPE);
          dl[(size_t)k * n + s] = in ? d - g0 : -1;
        }
    }
    if (threadIdx.x == 0) {
      lp[0] = g0;
      sh_cnt3[0] = sh_cnt3[1] = sh_cnt3[2] = 0;
    }
    __syncthreads();
    int remaining = n, L = 0, run = 0;     // run: ghosts levelled so far (register, not lp[])
    if (fast) {
      // layered topological sort: a ghost joins level L + 1 when its last
      // dependency is placed in level L, i.e. level = 1 + max over its
      // dependencies (Sec. 3.2); each level touches only its own frontier
      int* indeg = dl + (size_t)K * n;         // [n]
      int* cptr = indeg + n;                   // [n + 1] consumer offsets
      int* cons = cptr + n + 1;                // [K][n] consumers
      int* fr0 = cons + (size_t)K * n;         // [n] frontiers of odd levels
      int* fr1 = fr0 + n;                      // [n] frontiers of even levels (first: cursors)
      for (int q = threadIdx.x; q <= n; q += LV_T) cptr[q] = 0;
      __syncthreads();
      for (int q = threadIdx.x; q < n; q += LV_T) {
        int c = 0;
        for (int k = 0; k < K; ++k) {
          const int d = dl[(size_t)k * n + q];
          if (d >= 0) { ++c; atomicAdd(&cptr[d], 1); }
        }
        indeg[q] = c;
      }
      __syncthreads();
      {
        // exclusive scan of the consumer counts, a contiguous segment per thread
        const int per = (n + LV_T - 1) / LV_T;
        const int q0 = min(n, (int)threadIdx.x * per), q1 = min(n, q0 + per);
        int loc = 0;
        for (int q = q0; q < q1; ++q) loc += cptr[q];
        int x = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        if (lane == 31) sh_warp[w] = x;
        __syncthreads();
        if (w == 0) {
          int v = lane < LV_W ? sh_warp[lane] : 0;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
          }
          if (lane < LV_W) sh_warp[lane] = v;
        }
        __syncthreads();
        int ex = (w > 0 ? sh_warp[w - 1] : 0) + x - loc;
        for (int q = q0; q < q1; ++q) {
          const int c = cptr[q];
          cptr[q] = ex;
          ex += c;
        }
        if (threadIdx.x == LV_T - 1) cptr[n] = sh_warp[LV_W - 1];
        __syncthreads();
      }
      for (int q = threadIdx.x; q < n; q += LV_T) fr1[q] = cptr[q];
      __syncthreads();
      for (int q = threadIdx.x; q < n; q += LV_T)
        for (int k = 0; k < K; ++k) {
          const int d = dl[(size_t)k * n + q];
          if (d >= 0) cons[atomicAdd(&fr1[d], 1)] = q;
        }
      __syncthreads();
      for (int q = threadIdx.x; q < n; q += LV_T)
        if (indeg[q] == 0) {
          lvl[q] = 1;
          fr0[atomicAdd(&sh_cnt3[1], 1)] = q;
        }
      __syncthreads();
      // frontier counts: level L in sh_cnt3[L % 3]; thread 0 clears the slot
      // of level L + 2 while level L is processed (last read two levels ago)
      int nf = sh_cnt3[1];
      if (nf > 0) {
        L = 1;
        run = nf;
        if (threadIdx.x == 0) lp[1] = g0 + run;
      }
      while (nf > 0) {
        if (threadIdx.x == 0) sh_cnt3[(L + 2) % 3] = 0;
        const int* cur = (L & 1) ? fr0 : fr1;
        int* nxt = (L & 1) ? fr1 : fr0;
        for (int i = threadIdx.x; i < nf; i += LV_T) {
          const int q = cur[i];
          for (int e = cptr[q]; e < cptr[q + 1]; ++e) {
            const int c = cons[e];
            if (atomicSub(&indeg[c], 1) == 1) {
              lvl[c] = L + 1;
              nxt[atomicAdd(&sh_cnt3[(L + 1) % 3], 1)] = c;
            }
          }
        }
        __syncthreads();
        nf = sh_cnt3[(L + 1) % 3];
        if (nf == 0) break;
        ++L;
        run += nf;
        if (threadIdx.x == 0) lp[L] = g0 + run;
      }
      remaining = n - run;
      if (remaining > 0 && threadIdx.x == 0) set_status(status, S_ECYCLE);
    } else {
      // one barrier per sweep: the count of sweep L lives in sh_cnt3[L % 3];
      // thread 0 clears the slot of sweep L + 1, last read in sweep L - 2
      while (remaining > 0) {
        ++L;
        if (threadIdx.x == 0) sh_cnt3[(L + 1) % 3] = 0;
        int mine = 0;
        for (int s = threadIdx.x; s < n; s += LV_T) {
          if (lvl[s] != 0) continue;
          bool ok = true;
          for (int k = 0; k < K && ok; ++k) {
            int d = fast ? dl[(size_t)k * n + s] : dep[(size_t)k * ng_total + g0 + s] - g0;
            if (d >= n) d = -1;              // outside the geometry (never written by k_deps)
            if (d >= 0) {
              int lv = ((volatile int*)lvl)[d];
              if (lv == 0 || lv >= L) ok = false;
            }
          }
          if (ok) { lvl[s] = L; ++mine; }
        }
        // one shared-memory atomic per warp (same-address atomics serialise)
        mine = __reduce_add_sync(0xffffffffu, mine);
        if (lane == 0 && mine) atomicAdd(&sh_cnt3[L % 3], mine);
        __syncthreads();
        const int cnt = sh_cnt3[L % 3];
        if (cnt == 0) {
          if (threadIdx.x == 0) set_status(status, S_ECYCLE);
          break;
        }
        remaining -= cnt;
        run += cnt;
        if (threadIdx.x == 0) lp[L] = g0 + run;
      }
    }
    __syncthreads();
    int nl = remaining > 0 ? 0 : L;
    if (threadIdx.x == 0) n_levels[b] = nl;
    __syncthreads();
    if (remaining > 0) continue;
    if (fast && nl < LV_NL) {
      // stable counting sort by level: pos[L] = next free canonical slot of
      // level L (the dependency area is free now); per chunk of LV_T ghosts,
      // slot = pos[L] + (same-level ghosts of earlier warps in the chunk) +
      // (same-level lanes before it in its warp)
      int* pos = sm + n;
      for (int q = threadIdx.x; q < nl; q += LV_T) pos[q + 1] = lp[q];
      for (int base = 0; base < n; base += LV_T) {
        for (int q = threadIdx.x; q < (LV_T / 32) * LV_NL; q += LV_T) (&sh_wl[0][0])[q] = 0;
        __syncthreads();
        const int s = base + threadIdx.x;
        const int L2 = s < n ? lvl[s] : 0;
        const unsigned peers = __match_any_sync(0xffffffffu, L2);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (s < n && lane == __ffs(peers) - 1) sh_wl[w][L2] = __popc(peers);
        __syncthreads();
        // exclusive prefix over the warps, one thread per level
        for (int q = threadIdx.x; q <= nl; q += LV_T) {
          int acc = 0;
          for (int ww = 0; ww < LV_T / 32; ++ww) {
            const int v = sh_wl[ww][q];
            sh_wl[ww][q] = acc;
            acc += v;
          }
          sh_tot[q] = acc;
        }
        __syncthreads();
        if (s < n) order_pos[g0 + s] = pos[L2] + sh_wl[w][L2] + rank;
        __syncthreads();
        for (int q = threadIdx.x + 1; q <= nl; q += LV_T) pos[q] += sh_tot[q];
      }
      __syncthreads();
      for (int s = threadIdx.x; s < n; s += LV_T) level[g0 + s] = lvl[s];
    } else if (fast) {
      // more than LV_NL - 1 levels: warps in order, one at a time
      int* pos = sm + n;
      for (int q = threadIdx.x; q < nl; q += LV_T) pos[q + 1] = lp[q];
      __syncthreads();
      for (int base = 0; base < n; base += LV_T) {
        int s = base + threadIdx.x;
        int L2 = s < n ? lvl[s] : 0;
        unsigned peers = __match_any_sync(0xffffffffu, L2);
        int rank = __popc(peers & ((1u << lane) - 1u));
        bool leader = lane == __ffs(peers) - 1;
        for (int ww = 0; ww < LV_T / 32; ++ww) {
          int slot = 0;
          if (w == ww && s < n) slot = pos[L2] + rank;
          __syncwarp();
          if (w == ww && s < n) {
            order_pos[g0 + s] = slot;
            if (leader) pos[L2] += __popc(peers);
          }
          __syncthreads();
        }
      }
      for (int s = threadIdx.x; s < n; s += LV_T) level[g0 + s] = lvl[s];
    } else {
      // one block scan per level over the index order
      for (int lv = 1; lv <= nl; ++lv) {
        int carry = lp[lv - 1];
        for (int base = 0; base < n; base += LV_T) {
          int s = base + threadIdx.x;
          int f = (s < n && lvl[s] == lv) ? 1 : 0;
          unsigned bal = __ballot_sync(0xffffffffu, f);
          int inwarp = __popc(bal & ((1u << lane) - 1u));
          if (lane == 0) sh_warp[w] = __popc(bal);
          __syncthreads();
          if (w == 0) {
            int v = lane < LV_W ? sh_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              int y = __shfl_up_sync(0xffffffffu, v, o);
              if (lane >= o) v += y;
            }
            if (lane < LV_W) sh_warp[lane] = v;
          }
          __syncthreads();
          int before = (w > 0 ? sh_warp[w - 1] : 0);
          if (f) order_pos[g0 + s] = carry + before + inwarp;
          int tot = sh_warp[LV_W - 1];
          __syncthreads();
          carry += tot;
        }
      }
    }
    __syncthreads();
  }
}

void launch_levels(const Geom* G, int B, const int* dep, int ng_total, int* level, int* order_pos,
                   int* lev_ptr, int* n_levels, size_t smem, int* status, cudaStream_t s) {
  if (B <= 0) return;
  smem_raise<k_levels>(smem);
  launch(k_levels, B, LV_T, smem, s, G, B, dep, ng_total, level, order_pos, lev_ptr, n_levels,
                                 (int)(smem / sizeof(int)) - 16, status);
}

// canonical reorder of the ghost records; also the position of each ghost
// cell in the canonical order (pos_of_cell; no kernel of this launch reads it)
__global__ void k_reorder(const Geom* __restrict__ G, int* __restrict__ pos_of_cell, int ng,
                          const int* __restrict__ order_pos, const int* __restrict__ gs_cell,
                          const int* __restrict__ gs_geo, const double* __restrict__ gs_psi,
                          const double* __restrict__ gs_n, const uint32_t* __restrict__ gs_meta,
                          const int* __restrict__ dep, const int* __restrict__ level,
                          int* __restrict__ g_cell, int* __restrict__ g_geo, double* __restrict__ g_psi,
                          double* __restrict__ g_n, uint32_t* __restrict__ g_meta,
                          int* __restrict__ g_dep, int* __restrict__ g_level, const PlanCheck chk,
                          int* status) {
  pdl_enter();
  plan_check(G, chk, status);
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ng) return;
  int p = order_pos[s];
  g_cell[p] = gs_cell[s];
  g_geo[p] = gs_geo[s];
  g_psi[p] = gs_psi[s];
  for (int a = 0; a < 3; ++a) g_n[(size_t)a * ng + p] = gs_n[(size_t)a * ng + s];
  g_meta[p] = gs_meta[s];
  g_level[p] = level[s];
  for (int k = 0; k < MAXK; ++k) {
    int d = dep[(size_t)k * ng + s];
    g_dep[(size_t)k * ng + p] = d >= 0 ? order_pos[d] : -1;
  }
  pos_of_cell[G[gs_geo[s]].cell_off + gs_cell[s]] = p;
}

void launch_reorder(const Geom* G, int* pos_of_cell, int ng, const int* order_pos, const int* gs_cell,
                    const int* gs_geo,
                    const double* gs_psi, const double* gs_n, const uint32_t* gs_meta,
                    const int* dep, const int* level, int* g_cell, int* g_geo, double* g_psi,
                    double* g_n, uint32_t* g_meta, int* g_dep, int* g_level, cudaStream_t s,
                    const PlanCheck& chk, int* status) {
  if (ng <= 0) return;
  launch(k_reorder, (ng + 255) / 256, 256, 0, s, G, pos_of_cell, ng, order_pos, gs_cell, gs_geo, gs_psi, gs_n,
         gs_meta, dep, level, g_cell, g_geo, g_psi, g_n, g_meta, g_dep, g_level, chk, status);
}

// ---------------------------------------------------------------------------
// Per-ghost coefficient tables, evaluated once in double (the B300 FP64 pipe
// is narrow, so each closed form is evaluated once per geometry by all SMs):
//   wtab[(bc * 8 + slot) * ng + p]: weights on P_1..P_K (slots 0..K-1) and on
//     the boundary datum (slot 7), Eqs. phi_G_Dir_2d/_3d (bc 0) and
//     phi_G_Neu_2d/_3d (bc 1), local coordinates with the origin at G.
//   ftab[q * ng + p]: q = 0 surface weight w_G; q = 1 + slot: coefficient of the
//     slot value in phi_s (the Dirichlet relation solved for phi_s); q = 9 +
//     8 a + slot: coefficient in d phi / d x_a at S (Eq. derivative_bilinear,
//     Eqs. derivative_trilinear_x/y/z).  Slot 0 is G itself, slot k the member P_k.
// ---------------------------------------------------------------------------
__device__ void dirichlet_w(int dim, const double X2[3], const double Xs[3], double w[8]) {
  // w_a = (x_1 - x_s) / (x_2 - x_s) with x_1 = 0 (Eqs. phi_G_Dir_2d / _3d)
  double om[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < dim) om[a] = -Xs[a] / (X2[a] - Xs[a]);
  for (int q = 0; q < 8; ++q) w[q] = 0.0;
  if (dim == 2) {
    w[0] = om[0]; w[1] = om[1]; w[2] = -om[0] * om[1];
    w[7] = (1.0 - om[0]) * (1.0 - om[1]);
  } else {
    w[0] = om[0]; w[1] = om[1]; w[2] = om[2];
    w[3] = -om[0] * om[1]; w[4] = -om[1] * om[2]; w[5] = -om[0] * om[2];
    w[6] = om[0] * om[1] * om[2];
    w[7] = (1.0 - om[0]) * (1.0 - om[1]) * (1.0 - om[2]);
  }
}

__device__ void neumann_w(int dim, const double X2[3], const double Xs[3], const double n[3],
                          double w[8]) {
  for (int q = 0; q < 8; ++q) w[q] = 0.0;
  if (dim == 2) {
    // Eq. phi_G_Neu_2d with x_1 = y_1 = 0; one reciprocal of the common denominator
    double a1 = n[0] * (0.0 - Xs[1]), a2 = n[0] * (X2[1] - Xs[1]);
    double b1 = n[1] * (0.0 - Xs[0]), b2 = n[1] * (X2[0] - Xs[0]);
    double rden = 1.0 / (a2 + b2);
    double w1 = (a2 + b1) * rden, w2 = (a1 + b2) * rden;
    w[0] = w1; w[1] = w2; w[2] = 1.0 - w1 - w2;
    w[7] = -(X2[0] * X2[1]) * rden;
    return;
  }
  // Eq. phi_G_Neu_3d with a_ij = n_x (y_i - y_s)(z_j - z_s) etc., x_1 = 0
  const double xi[2] = {0.0 - Xs[0], X2[0] - Xs[0]};
  const double yi[2] = {0.0 - Xs[1], X2[1] - Xs[1]};
  const double zi[2] = {0.0 - Xs[2], X2[2] - Xs[2]};
  auto A = [&](int i, int j) { return n[0] * yi[i - 1] * zi[j - 1]; };
  auto Bf = [&](int i, int j) { return n[1] * xi[i - 1] * zi[j - 1]; };
  auto C = [&](int i, int j) { return n[2] * xi[i - 1] * yi[j - 1]; };
  double rden = 1.0 / (A(2, 2) + Bf(2, 2) + C(2, 2));
  w[0] = (A(2, 2) + Bf(1, 2) + C(1, 2)) * rden;
  w[1] = (A(1, 2) + Bf(2, 2) + C(2, 1)) * rden;
  w[2] = (A(2, 1) + Bf(2, 1) + C(2, 2)) * rden;
  w[3] = -(A(1, 2) + Bf(1, 2) + C(1, 1)) * rden;
  w[4] = -(A(1, 1) + Bf(2, 1) + C(2, 1)) * rden;
  w[5] = -(A(2, 1) + Bf(1, 1) + C(1, 2)) * rden;
  w[6] = (A(1, 1) + Bf(1, 1) + C(1, 1)) * rden;
  w[7] = -(X2[0] * X2[1] * X2[2]) * rden;
}

__global__ void k_tables(const Geom* __restrict__ G, int ng, const int* __restrict__ g_cell,
                         const int* __restrict__ g_geo, const double* __restrict__ g_psi,
                         const double* __restrict__ g_n, const uint32_t* __restrict__ g_meta,
                         const int8_t* __restrict__ tags, double* __restrict__ wtab,
                         double* __restrict__ ftab, float* __restrict__ wtab_f,
                         float* __restrict__ ftab_f) {
  pdl_enter();
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  const Geom& g = G[g_geo[p]];
  const int d = g.dim;
  uint32_t m = g_meta[p];
  double psi = g_psi[p];
  double n[3] = {g_n[p], g_n[ng + p], g_n[2 * (size_t)ng + p]};
  double X2[3] = {1, 1, 1}, Xs[3] = {0, 0, 0}, r2[3] = {1, 1, 1};
  int ijk[3];
  cell_ijk3(g, g_cell[p], ijk);
  // fixed-trip axis loops predicated on the dimension: static indices keep
  // the small arrays in registers.  x_2 - x_1 = r e h on a uniform grid; on
  // a stretched one the centre of the cell r_i e_i cells away minus the
  // ghost's (the index clamped into the grid: a stencil that leaves it is
  // reported by k_deps, and its weights are never used)
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < d) {
      const int step = meta_r(m, a) * meta_e(m, a);
      if (g.stretched) {
        const int far = min(max(ijk[a] + step, 0), g.n[a] - 1);
        X2[a] = g.cen[a][far] - g.cen[a][ijk[a]];
      } else {
        X2[a] = step * g.h[a];
      }
      Xs[a] = psi * n[a];
      r2[a] = 1.0 / X2[a];
    }
  }
  double wd[8], wn[8];
  dirichlet_w(d, X2, Xs, wd);
  neumann_w(d, X2, Xs, n, wn);
  // the tables and their float copies (what the kernels of FP32 fields read:
  // the same rounding as converting on use, without the conversions); only
  // the entries a stencil of this dimension has (slots 0 .. K-1 and the
  // boundary slot 7) are written, since no kernel reads the others
  const int Kd = stencil_k(d);
  for (int q = 0; q < 8; ++q) {
    if (q >= Kd && q != 7) continue;
    wtab[(size_t)q * ng + p] = wd[q];
    wtab[(size_t)(8 + q) * ng + p] = wn[q];
    wtab_f[(size_t)q * ng + p] = (float)wd[q];
    wtab_f[(size_t)(8 + q) * ng + p] = (float)wn[q];
  }
  // surface weight: faces shared with tag-0 cells, |n_face . n| times face
  // area (the ghost cell's own widths)
  const int8_t* tg = tags + g.cell_off;
  double wG = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= d) continue;
    double area = 1.0;
#pragma unroll
    for (int b = 0; b < 3; ++b)
      if (b < d && b != a) area *= width_of(g, b, ijk[b]);
#pragma unroll
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      int nb[3] = {ijk[0], ijk[1], ijk[2]};
      nb[a] += sgn;
      if (nb[a] < 0 || nb[a] >= g.n[a]) continue;
      if (tg[cell_lin(g, nb)] == 0) wG += area * fabs(n[a]);
    }
  }
  double f[33];
  for (int q = 0; q < 33; ++q) f[q] = 0.0;
  f[0] = wG;
  // phi_s = (phi_G - sum_k wd_k phi_k) / wd_s
  double rws = 1.0 / wd[7];
  f[1] = rws;
  const int K = stencil_k(d);
#pragma unroll
  for (int k = 0; k < 7; ++k)
    if (k < K) f[2 + k] = -wd[k] * rws;
  // gradient at S, local coordinates (x_1 = 0): fx0 = (x_2 - x_s)/(x_2 - x_1),
  // fx1 = (x_s - x_1)/(x_2 - x_1), divided differences over h = x_2 - x_1
  double fx0 = (X2[0] - Xs[0]) * r2[0], fx1 = Xs[0] * r2[0];
  double fy0 = (X2[1] - Xs[1]) * r2[1], fy1 = Xs[1] * r2[1];
  double* bx = f + 9;
  double* by = f + 17;
  double* bz = f + 25;
  if (d == 2) {
    double ix = r2[0], iy = r2[1];
    bx[0] = -fy0 * ix; bx[1] = fy0 * ix; bx[2] = -fy1 * ix; bx[3] = fy1 * ix;
    by[0] = -fx0 * iy; by[1] = -fx1 * iy; by[2] = fx0 * iy; by[3] = fx1 * iy;
  } else {
    double fz0 = (X2[2] - Xs[2]) * r2[2], fz1 = Xs[2] * r2[2];
    double ix = r2[0], iy = r2[1], iz = r2[2];
    // slots: 0 G, 1 P1, 2 P2, 3 P3, 4 P4, 5 P5, 6 P6, 7 P7
    bx[0] = -fy0 * fz0 * ix; bx[1] = fy0 * fz0 * ix; bx[2] = -fy1 * fz0 * ix; bx[4] = fy1 * fz0 * ix;
    bx[3] = -fy0 * fz1 * ix; bx[6] = fy0 * fz1 * ix; bx[5] = -fy1 * fz1 * ix; bx[7] = fy1 * fz1 * ix;
    by[0] = -fx0 * fz0 * iy; by[2] = fx0 * fz0 * iy; by[1] = -fx1 * fz0 * iy; by[4] = fx1 * fz0 * iy;
    by[3] = -fx0 * fz1 * iy; by[5] = fx0 * fz1 * iy; by[6] = -fx1 * fz1 * iy; by[7] = fx1 * fz1 * iy;
    bz[0] = -fx0 * fy0 * iz; bz[3] = fx0 * fy0 * iz; bz[1] = -fx1 * fy0 * iz; bz[6] = fx1 * fy0 * iz;
    bz[2] = -fx0 * fy1 * iz; bz[5] = fx0 * fy1 * iz; bz[4] = -fx1 * fy1 * iz; bz[7] = fx1 * fy1 * iz;
  }
  // ftab entries read for this dimension: w_G, the phi_s weights of the
  // ghost and its K members, the gradient weights of each axis
  for (int q = 0; q < 33; ++q) {
    const int a = q < 9 ? -1 : (q - 9) / 8, sl = q < 9 ? q - 1 : (q - 9) % 8;
    if (q > 0 && (sl > Kd || a >= d)) continue;
    ftab[(size_t)q * ng + p] = f[q];
    ftab_f[(size_t)q * ng + p] = (float)f[q];
  }
}

void launch_tables(const Geom* G, int ng, const int* g_cell, const int* g_geo, const double* g_psi,
                   const double* g_n, const uint32_t* g_meta, const int8_t* tags, double* wtab,
                   double* ftab, float* wtab_f, float* ftab_f, cudaStream_t s, int T) {
  if (ng <= 0) return;
  launch(k_tables, (ng + T - 1) / T, T, 0, s, G, ng, g_cell, g_geo, g_psi, g_n, g_meta, tags, wtab, ftab, wtab_f,
         ftab_f);
}

// ---------------------------------------------------------------------------
// Ghost targets' source lists (the adjoint reads the dependency relation of
// Sec. 3.2 backwards): ghost p's list is p itself (slot 0) followed by every
// (q, k + 1) whose stencil member k is p -- active or not, since the Sec. 6
// boundary-gradient stencils use every member -- in ascending (q, slot)
// order.  Built by transposition, without probing neighbourhoods:
//   k_gsrc_count    per ghost q: the ghost position of each member (mem[k][q],
//                   -1 when the member is not a ghost of this plan) and one
//                   more source for each such member (cnt starts at 1, set by
//                   k_poscell)
//   k_gsrc_self     offsets known: p's own entry first, the cursor after it
//   k_gsrc_place    the same in one launch with the offsets (single-pass scan
//                   of cnt; a re-run, checked against the planned total)
//   k_gsrc_scatter  each (q, k) takes the next entry of its target's list
//   k_gsrc_sort     each list after the own entry sorted (a list holds a few
//                   entries), so the order does not depend on the scatter
// ---------------------------------------------------------------------------
// An active member is a ghost exactly when it is a dependency (k_deps), whose
// position g_dep holds already; only inactive members (n_a = 0 along an
// offset axis) are looked up through the tags.
__global__ void k_gsrc_count(const Geom* __restrict__ G, int ng, const int* __restrict__ g_cell,
                             const int* __restrict__ g_geo, const uint32_t* __restrict__ g_meta,
                             const int* __restrict__ g_dep, const int8_t* __restrict__ tags,
                             const int* __restrict__ pos_of_cell, int kmax, int* __restrict__ mem,
                             int* __restrict__ cnt) {
  pdl_enter();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ng) return;
  const uint32_t m = g_meta[q];
  const uint32_t act = meta_active(m), dm = meta_depmask(m);
  const Geom* gp = nullptr;
  int ijk[3] = {0, 0, 0};
  for (int k = 0; k < kmax; ++k) {
    int p = -1;
    if (dm >> k & 1u) {
      p = g_dep[(size_t)k * ng + q];
    } else if (!(act >> k & 1u)) {
      if (!gp) {
        gp = &G[g_geo[q]];
        cell_ijk3(*gp, g_cell[q], ijk);
      }
      const Geom& g = *gp;
      int mijk[3];
      if (k < stencil_k(g.dim)) {
        member_ijk(g, ijk, m, k, mijk);
        if (in_grid(g, mijk)) {
          const int mc = cell_lin(g, mijk);
          const int8_t t = tags[g.cell_off + mc];
          if (t == 2 || t == -2) p = ghost_slot_of(g, mc, pos_of_cell + g.cell_off, g_cell);
        }
      }
    }
    if (p >= ng) p = -1;
    mem[(size_t)k * ng + q] = p;
    if (p >= 0) atomicAdd(&cnt[p], 1);
  }
}

__global__ void k_gsrc_self(int ng, const int* __restrict__ ptr, int* __restrict__ src, int* __restrict__ cursor) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  const int o = ptr[p];
  src[o] = p << 3;
  cursor[p] = o + 1;
}

__global__ void k_gsrc_place(int ng, int* __restrict__ cnt_cursor, int* __restrict__ ptr, int* __restrict__ src,
                             int cap, const Lookback L, int* status) {
  pdl_enter();
  __shared__ int sh[32];
  const LbBlock blk = lb_begin(L);
  const int p = blk.tile * blockDim.x + threadIdx.x;
  const bool on = p < ng;
  const int cnt = on ? cnt_cursor[p] : 0;
  int agg;
  const int ex = block_excl_scan(cnt, sh, agg);
  const long long base = lb_prefix(L, blk, (unsigned)agg, status);
  if (base < 0 && on) cnt_cursor[p] = cap;   // gave up: the scatter writes nothing for p
  if (base >= 0) {
    if (on) {
      const int o = (int)(base + ex);
      ptr[p] = o;
      if (o + cnt > cap) {
        set_status(status, S_ESHAPE);
        cnt_cursor[p] = cap;            // the scatter then writes nothing for p
      } else {
        src[o] = p << 3;
        cnt_cursor[p] = o + 1;
      }
    }
    if (p == ng - 1) {
      const long long total = base + ex + cnt;
      ptr[ng] = (int)min(total, (long long)cap);
      if (total != cap) set_status(status, S_ESHAPE);
    }
  }
  lb_end(L);
}

// entries outside [0, cap) are never written (a count that differs from the
// plan has set EBR_ESHAPE already)
__global__ void k_gsrc_scatter(int ng, int kmax, const int* __restrict__ mem, const int* __restrict__ ptr,
                               int* __restrict__ cursor, int* __restrict__ src, int cap, int* status) {
  pdl_enter();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ng) return;
  for (int k = 0; k < kmax; ++k) {
    const int p = mem[(size_t)k * ng + q];
    if (p < 0 || p >= ng) continue;
    const int o = atomicAdd(&cursor[p], 1);
    if (o >= 0 && o < ptr[p + 1] && o < cap) src[o] = (q << 3) | (k + 1);
    else set_status(status, S_ESHAPE);
  }
}

__global__ void k_gsrc_sort(int ng, const int* __restrict__ ptr, int* __restrict__ src, int cap) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  const int a = max(ptr[p] + 1, 0), b = min(ptr[p + 1], cap);
  for (int x = a + 1; x < b; ++x) {
    const int key = src[x];
    int y = x - 1;
    while (y >= a && src[y] > key) {
      src[y + 1] = src[y];
      --y;
    }
    src[y + 1] = key;
  }
}

void launch_gsrc_count(const Geom* G, int ng, const int* g_cell, const int* g_geo, const uint32_t* g_meta,
                       const int* g_dep, const int8_t* tags, const int* pos_of_cell, int kmax, int* mem, int* cnt,
                       cudaStream_t s, int T) {
  if (ng <= 0) return;
  launch(k_gsrc_count, (ng + T - 1) / T, T, 0, s, G, ng, g_cell, g_geo, g_meta, g_dep, tags, pos_of_cell, kmax,
         mem, cnt);
}

void launch_gsrc_lists(int ng, int kmax, const int* mem, const int* ptr, int* cursor, int* src, int cap,
                       int* status, bool self, cudaStream_t s, int T) {
  if (ng <= 0) return;
  if (self) launch(k_gsrc_self, (ng + T - 1) / T, T, 0, s, ng, ptr, src, cursor);
  launch(k_gsrc_scatter, (ng + T - 1) / T, T, 0, s, ng, kmax, mem, ptr, cursor, src, cap, status);
  launch(k_gsrc_sort, (ng + T - 1) / T, T, 0, s, ng, ptr, src, cap);
}

void launch_gsrc_place(int ng, int* cnt_cursor, int* ptr, int* src, int cap, const Lookback& L, int* status,
                       cudaStream_t s) {
  if (ng <= 0) return;
  launch(k_gsrc_place, (ng + LB_T - 1) / LB_T, LB_T, 0, s, ng, cnt_cursor, ptr, src, cap, L, status);
}

}  // namespace ebr
