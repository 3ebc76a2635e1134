// Many-field reconstruction in the field-minor ("packed") layout: one array
// [cells][F] whose F values of a cell are contiguous, so that the stencil
// gather of one ghost reads F consecutive values per member (a 128-byte line
// per 32 FP32 fields) instead of one 4-byte value per field array.
//
// Schedule (Sec. 3.2 level order; the closed forms of Secs. 4-5 through the
// weight table).  Levels 1..L0, which hold most ghosts, run as grid-wide
// launches; the thin tail of long dependency chains (levels > L0, planned so
// that no geometry has more than a few dozen ghosts in any of them) runs in
// one CTA per geometry with block barriers between levels.
//
// Every item (ghost or fluid target) has a fixed-size record, built once per
// plan and field type: global cells of its rows, the weights of both
// boundary-condition kinds in the field type, and up to CI inline source
// entries (longer source lists continue in a CSR array).  A warp handles one
// item: its lanes load the record in one coalesced step, then the warp issues
// all row loads of the item at once with a lane per field.  Two dependent
// memory steps per item, and many items in flight per SM.
//
//   forward: every ghost's boundary term + fluid members ("partial", final for
//            level 1); levels 2..L0 add their ghost members; the tail CTAs
//            add them for the remaining levels.
//   adjoint (vector-Jacobian product of the in-place fill): on entry cot holds
//            dJ/d(field after the fill); on exit dJ/d(field before the fill):
//            ghost entries 0 (the fill overwrites them), fluid entries
//            incremented by the transposed weights; grad_bc = dJ/d(boundary
//            data).  lambda_G = cot_G + sum over consumers (H, k) of
//            w_(H,k) lambda_H in reverse level order (tail CTAs, then levels
//            L0..1 grid-wide); then every fluid target T adds
//            sum over its sources (H, k) of w_(H,k) lambda_H (fixed order:
//            the first active incidence of a target owns it), each target
//            written once, without atomics.
#include "ebr_kernels.cuh"
#include "ebr_probe.cuh"

namespace ebr {

constexpr int PK_T = 256;        // grid-wide kernels: 8 warps per CTA
#ifndef EBR_PK_CT
#define EBR_PK_CT 256
#endif
constexpr int PK_CT = EBR_PK_CT;  // shared-memory tail kernels: 8 warps per CTA
constexpr int PK_CA = 512;       // adjoint tail: 16 warps per CTA, two CTAs per SM
#ifndef EBR_PK_G
#define EBR_PK_G 6
#endif
// 32-field chunks per warp pass: 192 fields, whose row loads the warp issues
// together (measured, 192 fields: 0.247 -> 0.242 ms per overlapped step;
// 8 chunks: 0.359 ms)
constexpr int PK_G = EBR_PK_G;
constexpr int CI = 4;            // inline source entries per record

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

// ---------------------------------------------------------------------------
// records: 32-bit words; a value of type T takes WPV<T> words
//   forward  [0] cell, [1..K] member cells, [K+1] masks (non-dependency
//            active | dependency active << 8), [K+2..2K+1] ghost position of
//            each dependency member (-1 otherwise), then w0[0..K], w1[0..K]
//            (index K = boundary datum)
//   adjoint  [0] cell, [1] n consumers, [2] CSR offset of the consumers,
//            [3..] wb0, wb1 (boundary weights), then CI x (q, w0, w1)
//   fluid    [0] cell, [1] n sources, [2] CSR offset, then CI x (q, w0, w1)
// ---------------------------------------------------------------------------
template <typename T> struct WPV { static constexpr int v = sizeof(T) / 4; };

__host__ __device__ constexpr int rec_round(int w) { return w <= 16 ? 16 : (w <= 32 ? 32 : 64); }
template <int K> __host__ __device__ constexpr int fw_w() { return 2 * K + 2; }   // first weight word
template <typename T, int K> __host__ __device__ constexpr int rec_fwd_words() {
  return rec_round(fw_w<K>() + 2 * (K + 1) * WPV<T>::v);
}
template <typename T> __host__ __device__ constexpr int rec_src_words() {
  return rec_round(3 + 2 * WPV<T>::v + CI * (1 + 2 * WPV<T>::v));
}

__device__ __forceinline__ void put_val(uint32_t* r, int w, float v) { r[w] = __float_as_uint(v); }
__device__ __forceinline__ void put_val(uint32_t* r, int w, double v) {
  r[w] = (uint32_t)__double2loint(v);
  r[w + 1] = (uint32_t)__double2hiint(v);
}

// the record of the lane's item lives in registers a (words 0..31) and b
// (words 32..63); word(x) broadcasts word x to the warp.  It is a whole-warp
// shuffle: every lane of the warp must call it (never inside a lane branch).
struct Rec {
  uint32_t a, b;
  __device__ __forceinline__ uint32_t word(int x) const {
    return __shfl_sync(0xffffffffu, x < 32 ? a : b, x & 31);
  }
  __device__ __forceinline__ int iword(int x) const { return (int)word(x); }
  __device__ __forceinline__ void val(int x, float& v) const { v = __uint_as_float(word(x)); }
  __device__ __forceinline__ void val(int x, double& v) const {
    v = __hiloint2double((int)word(x + 1), (int)word(x));
  }
};

__device__ __forceinline__ Rec load_rec(const uint32_t* __restrict__ rec, long long item, int stride) {
  const int lane = threadIdx.x & 31;
  const uint32_t* r = rec + item * stride;
  Rec R;
  R.a = lane < stride ? r[lane] : 0u;
  R.b = 32 + lane < stride ? r[32 + lane] : 0u;
  return R;
}

template <typename T, int K>
__global__ void k_rec_fwd(int ng, const Geom* __restrict__ G, const int* __restrict__ g_geo,
                          const int* __restrict__ g_cell, const uint32_t* __restrict__ g_meta,
                          const int* __restrict__ g_dep, const double* __restrict__ wtab,
                          uint32_t* __restrict__ out) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  constexpr int S = rec_fwd_words<T, K>(), V = WPV<T>::v;
  uint32_t* r = out + (long long)p * S;
  const Geom& g = G[g_geo[p]];
  const int lc = g_cell[p];
  const uint32_t m = g_meta[p];
  const uint32_t act = meta_active(m), dm = meta_depmask(m) & act;
  r[0] = (uint32_t)(g.cell_off + lc);
  for (int k = 0; k < K; ++k)
    r[1 + k] = (act >> k & 1u) ? (uint32_t)(g.cell_off + member_lin(g, lc, m, k)) : 0xffffffffu;
  r[K + 1] = (act & ~dm) | (dm << 8);
  for (int k = 0; k < K; ++k) r[K + 2 + k] = (dm >> k & 1u) ? (uint32_t)g_dep[(size_t)k * ng + p] : 0xffffffffu;
  constexpr int W = fw_w<K>();
  for (int k = 0; k <= K; ++k) {
    const int slot = k < K ? k : 7;
    put_val(r, W + k * V, (T)wtab[(size_t)slot * ng + p]);
    put_val(r, W + (K + 1 + k) * V, (T)wtab[(size_t)(8 + slot) * ng + p]);
  }
  for (int w = W + 2 * (K + 1) * V; w < S; ++w) r[w] = 0u;
}

// source records: n entries (q << 3 | slot) of src[a, a + n), inline up to CI
template <typename T>
__device__ inline void put_sources(uint32_t* r, int base, const int* __restrict__ src, int a, int n,
                                   const double* __restrict__ wtab, int ng) {
  constexpr int V = WPV<T>::v;
  for (int x = 0; x < CI; ++x) {
    uint32_t* e = r + base + x * (1 + 2 * V);
    if (x < n) {
      const int s = src[a + x];
      const int q = s >> 3, sl = s & 7;
      e[0] = (uint32_t)q;
      put_val(e, 1, (T)wtab[(size_t)(sl - 1) * ng + q]);
      put_val(e, 1 + V, (T)wtab[(size_t)(8 + sl - 1) * ng + q]);
    } else {
      for (int w = 0; w < 1 + 2 * V; ++w) e[w] = 0u;
    }
  }
}

template <typename T>
__global__ void k_rec_adj(int ng, const Geom* __restrict__ G, const int* __restrict__ g_geo,
                          const int* __restrict__ g_cell, const int* __restrict__ cons_ptr,
                          const int* __restrict__ cons, const double* __restrict__ wtab,
                          uint32_t* __restrict__ out) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  constexpr int S = rec_src_words<T>(), V = WPV<T>::v;
  uint32_t* r = out + (long long)p * S;
  const int a = cons_ptr[p], n = cons_ptr[p + 1] - a;
  r[0] = (uint32_t)(G[g_geo[p]].cell_off + g_cell[p]);
  r[1] = (uint32_t)n;
  r[2] = (uint32_t)a;
  put_val(r, 3, (T)wtab[(size_t)7 * ng + p]);
  put_val(r, 3 + V, (T)wtab[(size_t)15 * ng + p]);
  put_sources<T>(r, 3 + 2 * V, cons, a, n, wtab, ng);
  for (int w = 3 + 2 * V + CI * (1 + 2 * V); w < S; ++w) r[w] = 0u;
}

template <typename T>
__global__ void k_rec_fluid(int n_ft, const int* __restrict__ ft_cell, const int* __restrict__ ft_ptr,
                            const int* __restrict__ ft_src, const double* __restrict__ wtab, int ng,
                            uint32_t* __restrict__ out) {
  pdl_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_ft) return;
  constexpr int S = rec_src_words<T>(), V = WPV<T>::v;
  uint32_t* r = out + (long long)t * S;
  const int a = ft_ptr[t], n = ft_ptr[t + 1] - a;
  r[0] = (uint32_t)ft_cell[t];
  r[1] = (uint32_t)n;
  r[2] = (uint32_t)a;
  for (int w = 3; w < 3 + 2 * V; ++w) r[w] = 0u;
  put_sources<T>(r, 3 + 2 * V, ft_src, a, n, wtab, ng);
  for (int w = 3 + 2 * V + CI * (1 + 2 * V); w < S; ++w) r[w] = 0u;
}

// ---------------------------------------------------------------------------
// forward item: one ghost, all fields
// ---------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void pf_item(const Rec& R, T* __restrict__ fld, const T* __restrict__ bc, int F,
                                        const KindBits& kb, long long p, bool partial, int f_lo,
                                        int f_hi, bool& bad) {
  constexpr int V = WPV<T>::v;
  const int lane = threadIdx.x & 31;
  const long long cell = (long long)R.word(0);
  const uint32_t masks = R.word(K + 1);
  const uint32_t use = partial ? (masks & 0xffu) : (masks >> 8);
  long long mc[K];
  T w0[K + 1], w1[K + 1];
#pragma unroll
  for (int k = 0; k < K; ++k) mc[k] = (long long)R.word(1 + k);
#pragma unroll
  for (int k = 0; k <= K; ++k) {
    R.val(fw_w<K>() + k * V, w0[k]);
    R.val(fw_w<K>() + (K + 1 + k) * V, w1[k]);
  }
  for (int f0 = f_lo; f0 < f_hi; f0 += 32 * PK_G) {
    T v[PK_G];
#pragma unroll
    for (int c = 0; c < PK_G; ++c) {
      const int f = f0 + c * 32 + lane;
      v[c] = T(0);
      if (f < f_hi) {
        const bool nk = kind_of(kb, f);
        T a = partial ? (nk ? w1[K] : w0[K]) * bc[p * F + f] : fld[cell * F + f];
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (use >> k & 1u) a += (nk ? w1[k] : w0[k]) * fld[mc[k] * F + f];
        v[c] = a;
      }
    }
#pragma unroll
    for (int c = 0; c < PK_G; ++c) {
      const int f = f0 + c * 32 + lane;
      if (f < f_hi) {
        fld[cell * F + f] = v[c];
        if (!isfinite((double)v[c])) bad = true;
      }
    }
  }
}

// grid-wide forward: warp per ghost of `list` (all ghosts when list == null)
template <typename T, int K>
__global__ void __launch_bounds__(PK_T) k_pf_grid(T* __restrict__ fld, const T* __restrict__ bc, int F,
                                                  const __grid_constant__ KindBits kb,
                                                  const uint32_t* __restrict__ rec,
                                                  const int* __restrict__ list, int n, int partial,
                                                  int* status) {
  pdl_enter();
  const int i = (blockIdx.x * PK_T + threadIdx.x) >> 5;
  if (i >= n) return;
  const long long p = list ? list[i] : i;
  const Rec R = load_rec(rec, p, rec_fwd_words<T, K>());
  bool bad = false;
  pf_item<T, K>(R, fld, bc, F, kb, p, partial != 0, 0, F, bad);
  if (bad) set_status(status, S_ENONFINITE);
}

// tail chain, forward: levels > L0 of one geometry per CTA, warp per
// (ghost, 32 fields)
template <typename T, int K>
__global__ void __launch_bounds__(PK_CT) k_pf_tail(T* __restrict__ fld, int F,
                                                   const __grid_constant__ KindBits kb,
                                                   const Geom* __restrict__ G,
                                                   const int* __restrict__ geo_list,
                                                   const uint32_t* __restrict__ rec,
                                                   const int* __restrict__ lev_ptr, int L0,
                                                   int* status) {
  pdl_enter();
  const Geom& g = G[geo_list[blockIdx.x]];
  const int* lp = lev_ptr + g.lev_off;
  const int n_levels = g.n_levels;     // in a register: the kernel stores to global memory
  const int warp = threadIdx.x >> 5, nw = PK_CT / 32;
  const int nch = (F + 31) / 32;
  bool bad = false;
  for (int lv = L0 + 1; lv <= n_levels; ++lv) {
    const int a = lp[lv - 1], b = lp[lv];
    for (int t = warp; t < (b - a) * nch; t += nw) {
      const int p = a + t / nch, c = t % nch;
      const Rec R = load_rec(rec, p, rec_fwd_words<T, K>());
      pf_item<T, K>(R, fld, nullptr, F, kb, p, false, c * 32, min(F, c * 32 + 32), bad);
    }
    __syncthreads();
  }
  if (bad) set_status(status, S_ENONFINITE);
}

// tail chain in shared memory, forward: CTA per (tail geometry, 32 fields).
// Phase A gathers, for every tail ghost, its partial plus the terms of its
// dependency members outside the tail (final already) and records the
// members inside the tail; phase B walks the tail levels on shared memory.
template <typename T, int K>
struct TailF {
  static size_t bytes(int nt) {
    return (size_t)nt * (32 * sizeof(T) + sizeof(int) + K * (sizeof(int) + 2 * sizeof(T))) + 64;
  }
};

template <typename T, int K>
__global__ void __launch_bounds__(PK_CT, 2) k_pf_tail_s(T* __restrict__ fld, int F,
                                                     const __grid_constant__ KindBits kb,
                                                     const Geom* __restrict__ G,
                                                     const int* __restrict__ geo_list,
                                                     const uint32_t* __restrict__ rec,
                                                     const int* __restrict__ lev_ptr, int L0,
                                                     int cap, int ng, int* status) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int V = WPV<T>::v;
  const Geom& g = G[geo_list[blockIdx.y]];   // chunks of one geometry launch together
  const int* lp = lev_ptr + g.lev_off;
  const int n_levels = g.n_levels;     // in a register: the kernel stores to global memory
  const int t0 = lp[L0], nt = lp[n_levels] - t0;
  // the plan sized the shared memory for `cap` tail ghosts
  if (nt < 0 || nt > cap || t0 < 0 || t0 + nt > ng) {
    if (threadIdx.x == 0) set_status(status, S_ESHAPE);
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = PK_CT / 32;
  const int f = blockIdx.x * 32 + lane;
  const bool on = f < F;
  const int fo = on ? f : 0;
  const bool nk = on && kind_of(kb, f);
  T* vals = reinterpret_cast<T*>(smem);                          // [nt][32]
  T* dw = vals + (size_t)nt * 32;                                // [nt][K][2]
  int* dl = reinterpret_cast<int*>(dw + (size_t)nt * K * 2);     // [nt][K]
  int* cellS = dl + (size_t)nt * K;                              // [nt]
  // phase A: four ghosts per warp at a time, so that their record and row
  // loads are in flight together
  constexpr int NB = 4;
  for (int s0 = warp; s0 < nt; s0 += nw * NB) {
    Rec R[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int s = s0 + u * nw;
      R[u] = s < nt ? load_rec(rec, t0 + s, rec_fwd_words<T, K>()) : Rec{0u, 0u};
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int s = s0 + u * nw;
      if (s >= nt) continue;                       // warp-uniform
      const long long cell = (long long)R[u].word(0);
      const uint32_t dm = R[u].word(K + 1) >> 8;
      T v = fld[cell * F + fo];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        int loc = -1;
        T w0 = T(0), w1 = T(0);
        if (dm >> k & 1u) {                       // warp-uniform
          const int q = R[u].iword(K + 2 + k);
          const long long mcell = (long long)R[u].word(1 + k);
          R[u].val(fw_w<K>() + k * V, w0);
          R[u].val(fw_w<K>() + (K + 1 + k) * V, w1);
          // dependencies sit at lower levels of the same geometry: inside the
          // tail (shared memory) or before it (final in global memory)
          if (q >= t0 && q < t0 + nt) loc = q - t0;
          else v += (nk ? w1 : w0) * fld[mcell * F + fo];
        }
        if (lane == 0) {
          dl[s * K + k] = loc;
          dw[(s * K + k) * 2] = w0;
          dw[(s * K + k) * 2 + 1] = w1;
        }
      }
      vals[s * 32 + lane] = v;
      if (lane == 0) cellS[s] = (int)cell;
    }
  }
  __syncthreads();
  bool bad = false;
  for (int lv = L0 + 1; lv <= n_levels; ++lv) {
    const int a = max(lp[lv - 1] - t0, 0), b = min(lp[lv] - t0, nt);
    for (int s = a + warp; s < b; s += nw) {
      T v = vals[s * 32 + lane];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int d = dl[s * K + k];
        if (d >= 0) v += dw[(s * K + k) * 2 + (nk ? 1 : 0)] * vals[d * 32 + lane];
      }
      vals[s * 32 + lane] = v;
      if (on) {
        fld[(long long)cellS[s] * F + f] = v;
        if (!isfinite((double)v)) bad = true;
      }
    }
    __syncthreads();
  }
  if (bad) set_status(status, S_ENONFINITE);
}

// tail chain in shared memory, adjoint: every consumer of a tail ghost is a
// tail ghost (its level is higher), so lambda stays in shared memory.
// Record words are broadcast by whole-warp shuffles: every lane reads them,
// lane 0 alone stores them.
template <typename T>
struct TailA {
  static size_t bytes(int nt) {
    return (size_t)nt * (32 * sizeof(T) + 3 * sizeof(int) + 2 * sizeof(T) +
                         CI * (sizeof(int) + 2 * sizeof(T))) + 64;
  }
};

template <typename T>
__global__ void __launch_bounds__(PK_CT, 2) k_pa_tail_s(T* __restrict__ cot, T* __restrict__ lamP,
                                                     T* __restrict__ gbc, int F,
                                                     const __grid_constant__ KindBits kb,
                                                     const Geom* __restrict__ G,
                                                     const int* __restrict__ geo_list,
                                                     const uint32_t* __restrict__ rec,
                                                     const int* __restrict__ lev_ptr, int L0,
                                                     const int* __restrict__ cons,
                                                     const double* __restrict__ wtab, int ng,
                                                     int cap, int* status) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int V = WPV<T>::v;
  const Geom& g = G[geo_list[blockIdx.y]];   // chunks of one geometry launch together
  const int* lp = lev_ptr + g.lev_off;
  const int n_levels = g.n_levels;     // in a register: the kernel stores to global memory
  const int t0 = lp[L0], nt = lp[n_levels] - t0;
  // the plan sized the shared memory for `cap` tail ghosts
  if (nt < 0 || nt > cap || t0 < 0 || t0 + nt > ng) {
    if (threadIdx.x == 0) set_status(status, S_ESHAPE);
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = PK_CT / 32;
  const int f = blockIdx.x * 32 + lane;
  const bool on = f < F;
  const int fo = on ? f : 0;
  const bool nk = on && kind_of(kb, f);
  T* lam = reinterpret_cast<T*>(smem);                           // [nt][32]
  T* bw = lam + (size_t)nt * 32;                                 // [nt][2]
  T* cw = bw + (size_t)nt * 2;                                   // [nt][CI][2]
  int* cl = reinterpret_cast<int*>(cw + (size_t)nt * CI * 2);    // [nt][CI]
  int* cellS = cl + (size_t)nt * CI;                             // [nt]
  int* nS = cellS + nt;                                          // [nt]
  int* aS = nS + nt;                                             // [nt]
  // phase A: four ghosts per warp at a time (record and row loads in flight
  // together); every lane reads the record words, lane 0 stores them
  constexpr int NB = 4;
  for (int s0 = warp; s0 < nt; s0 += nw * NB) {
    Rec R[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int s = s0 + u * nw;
      R[u] = s < nt ? load_rec(rec, t0 + s, rec_src_words<T>()) : Rec{0u, 0u};
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int s = s0 + u * nw;
      if (s >= nt) continue;                       // warp-uniform
      const long long cell = (long long)R[u].word(0);
      int n = R[u].iword(1);
      const int a0 = R[u].iword(2);
      if (n < 0 || n > PACKED_MAX_SOURCES) {
        if (lane == 0) set_status(status, S_EINVAL);
        n = 0;
      }
      lam[s * 32 + lane] = cot[cell * F + fo];
      T b0, b1;
      R[u].val(3, b0);
      R[u].val(3 + V, b1);
#pragma unroll
      for (int x = 0; x < CI; ++x) {
        const int e = 3 + 2 * V + x * (1 + 2 * V);
        const int q = R[u].iword(e);
        T w0, w1;
        R[u].val(e + 1, w0);
        R[u].val(e + 1 + V, w1);
        if (lane == 0) {
          // consumers sit at higher levels of the same geometry: in the tail
          cl[s * CI + x] = (x < n && q >= t0 && q < t0 + nt) ? q - t0 : -1;
          cw[(s * CI + x) * 2] = w0;
          cw[(s * CI + x) * 2 + 1] = w1;
        }
      }
      if (lane == 0) {
        cellS[s] = (int)cell;
        nS[s] = n;
        aS[s] = a0;
        bw[s * 2] = b0;
        bw[s * 2 + 1] = b1;
      }
    }
  }
  __syncthreads();
  for (int lv = n_levels; lv > L0; --lv) {
    const int a = max(lp[lv - 1] - t0, 0), b = min(lp[lv] - t0, nt);
    for (int s = a + warp; s < b; s += nw) {
      T v = lam[s * 32 + lane];
      const int n = nS[s];
#pragma unroll
      for (int x = 0; x < CI; ++x) {
        const int d = cl[s * CI + x];
        if (d >= 0) v += cw[(s * CI + x) * 2 + (nk ? 1 : 0)] * lam[d * 32 + lane];
      }
      for (int x = CI; x < n; ++x) {               // rare: long consumer lists
        const int e = cons[aS[s] + x];
        const int q = e >> 3, sl = e & 7;
        if (q >= t0 && q < t0 + nt)
          v += (T)wtab[(size_t)((nk ? 8 : 0) + sl - 1) * ng + q] * lam[(q - t0) * 32 + lane];
      }
      lam[s * 32 + lane] = v;
      if (on) {
        const long long p = t0 + s;
        lamP[p * F + f] = v;
        gbc[p * F + f] = bw[s * 2 + (nk ? 1 : 0)] * v;
        cot[(long long)cellS[s] * F + f] = T(0);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// adjoint items: sum over the sources of an item, lane field f
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void src_sum(const Rec& R, int base, T* acc, int f0, int f_hi, const KindBits& kb,
                                        int F, const T* __restrict__ lamP, const int* __restrict__ csr,
                                        const double* __restrict__ wtab, int ng) {
  constexpr int V = WPV<T>::v;
  const int lane = threadIdx.x & 31;
  const int a = R.iword(2);
  const int n = min(max(R.iword(1), 0), PACKED_MAX_SOURCES);
#pragma unroll
  for (int x = 0; x < CI; ++x) {
    if (x >= n) break;
    const int e = base + x * (1 + 2 * V);
    const long long q = R.iword(e);
    T w0, w1;
    R.val(e + 1, w0);
    R.val(e + 1 + V, w1);
#pragma unroll
    for (int c = 0; c < PK_G; ++c) {
      const int f = f0 + c * 32 + lane;
      if (f < f_hi) acc[c] += (kind_of(kb, f) ? w1 : w0) * lamP[q * F + f];
    }
  }
  for (int x = CI; x < n; ++x) {                 // rare: long source lists
    const int s = csr[a + x];
    const long long q = s >> 3;
    const int sl = s & 7;
    const T w0 = (T)wtab[(size_t)(sl - 1) * ng + q], w1 = (T)wtab[(size_t)(8 + sl - 1) * ng + q];
#pragma unroll
    for (int c = 0; c < PK_G; ++c) {
      const int f = f0 + c * 32 + lane;
      if (f < f_hi) acc[c] += (kind_of(kb, f) ? w1 : w0) * lamP[q * F + f];
    }
  }
}

// adjoint ghost item: lambda = cot_G + consumers; writes lambda, dJ/db, 0
template <typename T>
__device__ __forceinline__ void pa_item(const Rec& R, T* __restrict__ cot, T* __restrict__ lamP,
                                        T* __restrict__ gbc, int F, const KindBits& kb, long long p,
                                        int f_lo, int f_hi, const int* __restrict__ cons,
                                        const double* __restrict__ wtab, int ng) {
  constexpr int V = WPV<T>::v;
  const int lane = threadIdx.x & 31;
  const long long cell = (long long)R.word(0);
  T b0, b1;
  R.val(3, b0);
  R.val(3 + V, b1);
  for (int f0 = f_lo; f0 < f_hi; f0 += 32 * PK_G) {
    T acc[PK_G];
#pragma unroll
    for (int c = 0; c < PK_G; ++c) {
      const int f = f0 + c * 32 + lane;
      acc[c] = f < f_hi ? cot[cell * F + f] : T(0);
    }
    src_sum<T>(R, 3 + 2 * V, acc, f0, f_hi, kb, F, lamP, cons, wtab, ng);
#pragma unroll
    for (int c = 0; c < PK_G; ++c) {
      const int f = f0 + c * 32 + lane;
      if (f < f_hi) {
        lamP[p * F + f] = acc[c];
        gbc[p * F + f] = (kind_of(kb, f) ? b1 : b0) * acc[c];
        cot[cell * F + f] = T(0);
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(PK_T) k_pa_grid(T* __restrict__ cot, T* __restrict__ lamP,
                                                  T* __restrict__ gbc, int F,
                                                  const __grid_constant__ KindBits kb,
                                                  const uint32_t* __restrict__ rec,
                                                  const int* __restrict__ cons,
                                                  const double* __restrict__ wtab, int ng,
                                                  const int* __restrict__ list, int n) {
  pdl_enter();
  const int i = (blockIdx.x * PK_T + threadIdx.x) >> 5;
  if (i >= n) return;
  const long long p = list[i];
  const Rec R = load_rec(rec, p, rec_src_words<T>());
  pa_item<T>(R, cot, lamP, gbc, F, kb, p, 0, F, cons, wtab, ng);
}

// tail chain, adjoint: levels n..L0+1 of one geometry per CTA (at most
// PACKED_TAIL_MAX_ADJ ghosts per level: at most one per warp, all fields);
// each warp loads the record of its ghost of the next level before the
// level barrier, so only the lambda rows wait on memory inside a level
template <typename T>
__global__ void __launch_bounds__(PK_CA, 2) k_pa_tail(T* __restrict__ cot, T* __restrict__ lamP,
                                                   T* __restrict__ gbc, int F,
                                                   const __grid_constant__ KindBits kb,
                                                   const Geom* __restrict__ G,
                                                   const int* __restrict__ geo_list,
                                                   const uint32_t* __restrict__ rec,
                                                   const int* __restrict__ lev_ptr, int L0,
                                                   const int* __restrict__ cons,
                                                   const double* __restrict__ wtab, int ng) {
  pdl_enter();
  const Geom& g = G[geo_list[blockIdx.x]];
  const int warp = threadIdx.x >> 5, nw = PK_CA / 32;
  const int* lp = lev_ptr + g.lev_off;
  const int n_levels = g.n_levels;     // in a register: the kernel stores to global memory
  // bring every tail record and ghost-cotangent row into L2 up front (the
  // rows of one ghost are F consecutive values, 128-byte lines)
  {
    const int t0 = lp[L0], t1 = lp[n_levels];
    const int lines = (int)((F * sizeof(T) + 127) / 128);
    for (int i = threadIdx.x; i < (t1 - t0) * (lines + 1); i += PK_CA) {
      const int p = t0 + i / (lines + 1), l = i % (lines + 1);
      const void* a;
      if (l == 0) {
        a = rec + (long long)p * rec_src_words<T>();
      } else {
        const long long cell = (long long)rec[(long long)p * rec_src_words<T>()];
        a = reinterpret_cast<const char*>(cot + cell * F) + (l - 1) * 128;
      }
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
  }
  Rec nxt{0u, 0u};
  if (n_levels > L0 && lp[n_levels - 1] + warp < lp[n_levels])
    nxt = load_rec(rec, lp[n_levels - 1] + warp, rec_src_words<T>());
  for (int lv = n_levels; lv > L0; --lv) {
    const int a = lp[lv - 1], b = lp[lv];
    for (int p = a + warp; p < b; p += nw) {
      const Rec R = p == a + warp ? nxt : load_rec(rec, p, rec_src_words<T>());
      pa_item<T>(R, cot, lamP, gbc, F, kb, p, 0, F, cons, wtab, ng);
    }
    if (lv - 1 > L0 && lp[lv - 2] + warp < lp[lv - 1])
      nxt = load_rec(rec, lp[lv - 2] + warp, rec_src_words<T>());
    __syncthreads();
  }
}

// fluid targets: warp per target
template <typename T>
__global__ void __launch_bounds__(PK_T) k_pa_fluid(T* __restrict__ cot, const T* __restrict__ lamP,
                                                   int F, const __grid_constant__ KindBits kb,
                                                   const uint32_t* __restrict__ rec,
                                                   const int* __restrict__ ft_src,
                                                   const double* __restrict__ wtab, int ng, int n) {
  pdl_enter();
  constexpr int V = WPV<T>::v;
  const int i = (blockIdx.x * PK_T + threadIdx.x) >> 5;
  if (i >= n) return;
  const int lane = threadIdx.x & 31;
  const Rec R = load_rec(rec, i, rec_src_words<T>());
  const long long cell = (long long)R.word(0);
  for (int f0 = 0; f0 < F; f0 += 32 * PK_G) {
    T acc[PK_G];
#pragma unroll
    for (int c = 0; c < PK_G; ++c) {
      const int f = f0 + c * 32 + lane;
      acc[c] = f < F ? cot[cell * F + f] : T(0);
    }
    src_sum<T>(R, 3 + 2 * V, acc, f0, F, kb, F, lamP, ft_src, wtab, ng);
#pragma unroll
    for (int c = 0; c < PK_G; ++c) {
      const int f = f0 + c * 32 + lane;
      if (f < F) cot[cell * F + f] = acc[c];
    }
  }
}

// plan: consumer lists (active incidences of each ghost as a member of
// another ghost) and fluid-target source lists (fixed probe order; the first
// active incidence of a target owns it)
// ---------------------------------------------------------------------------
__global__ void k_cons(int ng, const int* __restrict__ gsrc_ptr, const int* __restrict__ gsrc,
                       const uint32_t* __restrict__ g_meta, const int* __restrict__ ptr,
                       int* __restrict__ out) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  int c = 0, o = ptr ? ptr[p] : 0;
  for (int j = gsrc_ptr[p]; j < gsrc_ptr[p + 1]; ++j) {
    const int e = gsrc[j];
    const int q = e >> 3, sl = e & 7;
    if (sl == 0 || !(meta_active(g_meta[q]) >> (sl - 1) & 1u)) continue;
    if (ptr) out[o++] = e; else ++c;
  }
  if (!ptr) out[p] = c;
}

__global__ void k_ftgt(int ng, int kmax, const Geom* __restrict__ G, const int* __restrict__ g_geo,
                       const int* __restrict__ g_cell, const uint32_t* __restrict__ g_meta,
                       const int8_t* __restrict__ tags, const int* __restrict__ pos_of_cell, int R,
                       int* __restrict__ flag, int* __restrict__ cnt, const int* __restrict__ tpos,
                       const int* __restrict__ epos, int* __restrict__ ft_cell,
                       int* __restrict__ ft_ptr, int* __restrict__ ft_src) {
  pdl_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)ng * kmax) return;
  const int p = (int)(i / kmax), k = (int)(i - (long long)p * kmax);
  const bool write = tpos != nullptr;
  if (!write) { flag[i] = 0; cnt[i] = 0; }
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
  bool first = true, owner = false;
  int n = 0, o = write ? epos[i] : 0;
  probe_sources(g, tijk, tg, pc, g_cell, g_meta, R, [&](int q, int slot) {
    if (!(meta_active(g_meta[q]) >> (slot - 1) & 1u)) return true;
    if (first) {
      first = false;
      owner = (q == p && slot == k + 1);
      if (!owner) return false;
    }
    if (write) ft_src[o++] = (q << 3) | slot; else ++n;
    return true;
  });
  if (!owner) return;
  if (write) {
    const int t = tpos[i];
    ft_cell[t] = (int)(g.cell_off + cell_lin(g, tijk));
    ft_ptr[t] = epos[i];
  } else {
    flag[i] = 1;
    cnt[i] = n;
  }
}

void launch_packed_plan_cons(int ng, const int* gsrc_ptr, const int* gsrc, const uint32_t* g_meta,
                             const int* ptr, int* out, cudaStream_t s) {
  if (ng <= 0) return;
  launch(k_cons, (ng + 127) / 128, 128, 0, s, ng, gsrc_ptr, gsrc, g_meta, ptr, out);
}

void launch_packed_plan_ftgt(int ng, int kmax, const Geom* G, const int* g_geo, const int* g_cell,
                             const uint32_t* g_meta, const int8_t* tags, const int* pos_of_cell,
                             int R, int* flag, int* cnt, const int* tpos, const int* epos,
                             int* ft_cell, int* ft_ptr, int* ft_src, cudaStream_t s) {
  long long n = (long long)ng * kmax;
  if (n <= 0) return;
  launch(k_ftgt, (unsigned)((n + 127) / 128), 128, 0, s, ng, kmax, G, g_geo, g_cell, g_meta, tags,
                                                     pos_of_cell, R, flag, cnt, tpos, epos, ft_cell,
                                                     ft_ptr, ft_src);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static unsigned warp_blocks(long long n) { return (unsigned)((n * 32 + PK_T - 1) / PK_T); }

size_t packed_rec_words(int dtype, int dim, int which) {
  if (which == 0) {
    if (dtype == 0) return dim == 2 ? rec_fwd_words<float, 3>() : rec_fwd_words<float, 7>();
    return dim == 2 ? rec_fwd_words<double, 3>() : rec_fwd_words<double, 7>();
  }
  return dtype == 0 ? rec_src_words<float>() : rec_src_words<double>();
}

template <typename T>
static void recs_t(int dim, const Geom* G, int ng, const int* g_geo, const int* g_cell,
                   const uint32_t* g_meta, const int* g_dep, const double* wtab, const PackedPlan& pp,
                   uint32_t* fwd, uint32_t* adj, uint32_t* fl, cudaStream_t s) {
  if (ng > 0) {
    if (dim == 2) launch(k_rec_fwd<T, 3>, (ng + 127) / 128, 128, 0, s, ng, G, g_geo, g_cell, g_meta, g_dep, wtab, fwd);
    else launch(k_rec_fwd<T, 7>, (ng + 127) / 128, 128, 0, s, ng, G, g_geo, g_cell, g_meta, g_dep, wtab, fwd);
    launch(k_rec_adj<T>, (ng + 127) / 128, 128, 0, s, ng, G, g_geo, g_cell, pp.cons_ptr, pp.cons, wtab, adj);
  }
  if (pp.n_ft > 0)
    launch(k_rec_fluid<T>, (pp.n_ft + 127) / 128, 128, 0, s, pp.n_ft, pp.ft_cell, pp.ft_ptr, pp.ft_src, wtab,
                                                         ng, fl);
}

void launch_packed_records(int dtype, int dim, const Geom* G, int ng, const int* g_geo,
                           const int* g_cell, const uint32_t* g_meta, const int* g_dep,
                           const double* wtab, const PackedPlan& pp, uint32_t* fwd, uint32_t* adj,
                           uint32_t* fl, cudaStream_t s) {
  if (dtype == 0) recs_t<float>(dim, G, ng, g_geo, g_cell, g_meta, g_dep, wtab, pp, fwd, adj, fl, s);
  else recs_t<double>(dim, G, ng, g_geo, g_cell, g_meta, g_dep, wtab, pp, fwd, adj, fl, s);
}

// shared memory of the tail kernels for the largest tail (0 = does not fit)
size_t packed_tail_smem(int dtype, int dim, int which, int max_nt, int limit) {
  size_t b;
  if (which == 0) {
    if (dtype == 0) b = dim == 2 ? TailF<float, 3>::bytes(max_nt) : TailF<float, 7>::bytes(max_nt);
    else b = dim == 2 ? TailF<double, 3>::bytes(max_nt) : TailF<double, 7>::bytes(max_nt);
  } else {
    b = dtype == 0 ? TailA<float>::bytes(max_nt) : TailA<double>::bytes(max_nt);
  }
  return b <= (size_t)limit ? b : 0;
}

template <typename T, int K>
static void pfill_t(int F, void* fld, const void* bc, const KindBits& kb, const Geom* G,
                    const int* lev_ptr, int ng, const PackedPlan& pp, const uint32_t* rec,
                    int* status, cudaStream_t s, int phase) {
  auto grid = [&](int n, const int* list, int partial) {
    if (n <= 0) return;
    launch(k_pf_grid<T, K>, warp_blocks(n), PK_T, 0, s, (T*)fld, (const T*)bc, F, kb, rec, list, n,
                                                    partial, status);
  };
  if (phase == 0) grid(ng, nullptr, 1);
  if (phase == 1)
    for (int lv = 2; lv <= pp.L0; ++lv)
      grid(pp.h_lvl_off[lv] - pp.h_lvl_off[lv - 1], pp.d_lvl + pp.h_lvl_off[lv - 1], 0);
  if (phase == 2 && pp.n_tail > 0) {
    const size_t sm = pp.tail_smem[0][sizeof(T) == 4 ? 0 : 1];
    if (sm > 0) {
      smem_raise<k_pf_tail_s<T, K>>(sm);
      launch(k_pf_tail_s<T, K>, dim3((F + 31) / 32, pp.n_tail), PK_CT, sm, s, (T*)fld, F, kb, G, pp.d_tail, rec,
                                                                         lev_ptr, pp.L0, pp.tail_max, ng,
                                                                         status);
    } else {
      launch(k_pf_tail<T, K>, pp.n_tail, PK_CT, 0, s, (T*)fld, F, kb, G, pp.d_tail, rec, lev_ptr, pp.L0, status);
    }
  }
}

void launch_pfill(int dtype, int dim, int F, void* fld, const void* bc, const KindBits& kb,
                  const Geom* G, const int* lev_ptr, int ng, const PackedPlan& pp,
                  const uint32_t* rec, int* status, cudaStream_t s, int phase) {
  if (F <= 0 || ng <= 0) return;
  if (dtype == 0 && dim == 2) pfill_t<float, 3>(F, fld, bc, kb, G, lev_ptr, ng, pp, rec, status, s, phase);
  else if (dtype == 0) pfill_t<float, 7>(F, fld, bc, kb, G, lev_ptr, ng, pp, rec, status, s, phase);
  else if (dim == 2) pfill_t<double, 3>(F, fld, bc, kb, G, lev_ptr, ng, pp, rec, status, s, phase);
  else pfill_t<double, 7>(F, fld, bc, kb, G, lev_ptr, ng, pp, rec, status, s, phase);
}

int pfill_launches(const PackedPlan& pp, int ng) {
  if (ng <= 0) return 0;
  int n = 1;
  for (int lv = 2; lv <= pp.L0; ++lv) n += pp.h_lvl_off[lv] > pp.h_lvl_off[lv - 1];
  return n + (pp.n_tail > 0);
}

template <typename T>
static void padj_t(int F, void* cot, void* lamP, void* gbc, const KindBits& kb, const Geom* G, int ng,
                   const int* lev_ptr, const double* wtab, const PackedPlan& pp,
                   const uint32_t* rec_adj, const uint32_t* rec_fl, int* status, cudaStream_t s,
                   int phase) {
  if (phase == 0 && pp.n_tail_a > 0) {
    const size_t sm = pp.tail_smem[1][sizeof(T) == 4 ? 0 : 1];
    if (sm > 0) {
      smem_raise<k_pa_tail_s<T>>(sm);
      launch(k_pa_tail_s<T>, dim3((F + 31) / 32, pp.n_tail_a), PK_CT, sm, s, (T*)cot, (T*)lamP, (T*)gbc, F, kb,
                                                                        G, pp.d_tail_a, rec_adj, lev_ptr,
                                                                        pp.L0a, pp.cons, wtab, ng,
                                                                        pp.tail_max_a, status);
    } else {
      launch(k_pa_tail<T>, pp.n_tail_a, PK_CA, 0, s, (T*)cot, (T*)lamP, (T*)gbc, F, kb, G, pp.d_tail_a,
                                                 rec_adj, lev_ptr, pp.L0a, pp.cons, wtab, ng);
    }
  }
  if (phase == 1)
    for (int lv = pp.L0a; lv >= 1; --lv) {
      const int n = pp.h_lvl_off[lv] - pp.h_lvl_off[lv - 1];
      if (n <= 0) continue;
      launch(k_pa_grid<T>, warp_blocks(n), PK_T, 0, s, (T*)cot, (T*)lamP, (T*)gbc, F, kb, rec_adj, pp.cons,
                                                   wtab, ng, pp.d_lvl + pp.h_lvl_off[lv - 1], n);
    }
  if (phase == 2 && pp.n_ft > 0)
    launch(k_pa_fluid<T>, warp_blocks(pp.n_ft), PK_T, 0, s, (T*)cot, (const T*)lamP, F, kb, rec_fl, pp.ft_src,
                                                        wtab, ng, pp.n_ft);
}

void launch_padj(int dtype, int F, void* cot, void* lamP, void* gbc, const KindBits& kb,
                 const Geom* G, int ng, const int* lev_ptr, const double* wtab,
                 const PackedPlan& pp, const uint32_t* rec_adj, const uint32_t* rec_fl,
                 int* status, cudaStream_t s, int phase) {
  if (F <= 0 || ng <= 0) return;
  if (dtype == 0) padj_t<float>(F, cot, lamP, gbc, kb, G, ng, lev_ptr, wtab, pp, rec_adj, rec_fl, status, s, phase);
  else padj_t<double>(F, cot, lamP, gbc, kb, G, ng, lev_ptr, wtab, pp, rec_adj, rec_fl, status, s, phase);
}

int padj_launches(const PackedPlan& pp, int ng) {
  if (ng <= 0) return 0;
  int n = (pp.n_tail_a > 0) + (pp.n_ft > 0);
  for (int lv = 1; lv <= pp.L0a; ++lv) n += pp.h_lvl_off[lv] > pp.h_lvl_off[lv - 1];
  return n;
}

}  // namespace ebr
