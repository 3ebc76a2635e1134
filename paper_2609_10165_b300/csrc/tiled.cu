// Tiled level-by-level fill with per-level exchange (Sec. 3.2, the
// distributed-memory paragraph), on one GPU.
//
// The grid is cut into rectangular tiles; a ghost belongs to the tile of its
// cell.  Tiles are the subdomains: one persistent CTA owns one or more tiles
// (tile i goes to CTA i mod gridDim).  For each level L_k every CTA fills the
// ghosts of its tiles in L_k, reading fluid values and ghosts of its own tiles
// from the field arrays and ghosts of other tiles only from the exchange
// buffer; a ghost that some other tile's stencil reads (a "sent" ghost, with
// its slot in the exchange buffer) is also written there.  Then all CTAs meet
// at a device-wide barrier before L_{k+1}: exactly the level-wise exchange of
// the paper, with the exchange buffer standing for the messages.
//
// The barrier is a counter in global memory (arrivals since the launch) and an
// abort word.  Every wait is bounded: a CTA that has polled `spin_limit` times
// without seeing all arrivals records EBR_ETIMEOUT, raises the abort word and
// returns, and a CTA that sees the abort word returns too, so the launch always
// ends.  The launch is cooperative (all CTAs resident), so in a correct run
// the wait ends by itself.
//
// Each ghost is combined exactly as in the level-launch fill (boundary term
// first, then the active members in member order), so the two give the same
// bits.
#include "ebr_kernels.cuh"

namespace ebr {

constexpr int TL_T = 256;

struct TiledFields {
  void* f[8];
  const void* bc[8];
  int kind[8];
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Device-wide barrier of the persistent tiled kernel: returns false when the
// wait gave up (here or in another CTA), in which case the caller returns.
__device__ bool tiled_barrier(unsigned* bar, unsigned target, int spin_limit, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&bar[0], 1u);
    int ok = 1;
    for (int it = 0;; ++it) {
      if (ld_acquire(&bar[0]) >= target) break;
      if (ld_acquire(&bar[1]) != 0u) { ok = 0; break; }
      if (it >= spin_limit) {
        set_status(status, S_ETIMEOUT);
        atomicExch(&bar[1], 1u);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T, int D>
__global__ void __launch_bounds__(TL_T) k_tiled_fill(TiledFields P, int F, const Geom* __restrict__ G,
                                                     TiledPlanDev A, const int* __restrict__ g_geo,
                                                     const int* __restrict__ g_cell,
                                                     const uint32_t* __restrict__ g_meta,
                                                     const int* __restrict__ g_dep,
                                                     const T* __restrict__ wtab, int ng,
                                                     T* __restrict__ xbuf, unsigned* bar,
                                                     int extra_arrivals, int* status) {
  constexpr int K = D == 2 ? 3 : 7;
  const int W = A.Lmax + 1;
  for (int L = 1; L <= A.Lmax; ++L) {
    for (int i = blockIdx.x; i < A.n_tiles; i += gridDim.x) {
      const int a = A.t_ptr[(size_t)i * W + L - 1], b = A.t_ptr[(size_t)i * W + L];
      for (int e = a + threadIdx.x; e < b; e += TL_T) {
        const int p = A.t_list[e];
        const Geom& g = G[g_geo[p]];
        const int nx = g.n[0], ny = g.n[1];
        const long long cell_off = g.cell_off;
        const int cell = g_cell[p];
        const uint32_t m = g_meta[p];
        const uint32_t act = meta_active(m), dm = meta_depmask(m);
        const int tp = A.tile_of[p];
        const int slot = A.slot_of[p];
        // where each member's value comes from: the field (fluid cells and
        // this tile's ghosts, written at lower levels) or the exchange
        // buffer (another tile's ghosts)
        int mc[K], xs[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          int o[3];
          stencil_off(D, k, o);
          int off = o[0] * meta_r(m, 0) * meta_e(m, 0) + nx * (o[1] * meta_r(m, 1) * meta_e(m, 1));
          if (D == 3) off += nx * ny * (o[2] * meta_r(m, 2) * meta_e(m, 2));
          mc[k] = cell + off;
          xs[k] = -1;
          if (dm >> k & 1u) {
            const int d = g_dep[(size_t)k * ng + p];
            if (A.tile_of[d] != tp) xs[k] = A.slot_of[d];
          }
        }
        T w0[K + 1], w1[K + 1];
        w0[K] = (T)wtab[(size_t)7 * ng + p];
        w1[K] = (T)wtab[(size_t)15 * ng + p];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          w0[k] = (T)wtab[(size_t)k * ng + p];
          w1[k] = (T)wtab[(size_t)(8 + k) * ng + p];
        }
        // every load of the ghost before its stores (its members are never
        // in its own level); values written during this launch are read
        // through L2
        T val[8][K + 1];
#pragma unroll
        for (int f = 0; f < 8; ++f) {
          if (f >= F) break;
          const T* fld = static_cast<const T*>(P.f[f]) + cell_off;
          val[f][K] = static_cast<const T*>(P.bc[f])[p];
#pragma unroll
          for (int k = 0; k < K; ++k) {
            T v = T(0);
            if (act >> k & 1u) {
              if (xs[k] >= 0) v = __ldcg(xbuf + (size_t)f * A.n_slots + xs[k]);
              else if (dm >> k & 1u) v = __ldcg(fld + mc[k]);
              else v = fld[mc[k]];
            }
            val[f][k] = v;
          }
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
          if (slot >= 0) xbuf[(size_t)f * A.n_slots + slot] = acc;
          if (!isfinite((double)acc)) set_status(status, S_ENONFINITE);
        }
      }
    }
    if (L < A.Lmax) {
      const unsigned target = (unsigned)gridDim.x * (unsigned)L + (unsigned)extra_arrivals;
      if (!tiled_barrier(bar, target, A.spin_limit, status)) return;
    }
  }
}

int tiled_grid(int dtype, int n_tiles) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the 3D instances use the most registers: their residency bounds both
  if (dtype == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tiled_fill<float, 3>, TL_T, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tiled_fill<double, 3>, TL_T, 0);
  const long long cap = (long long)std::max(per, 1) * std::max(sms, 1);
  return (int)std::max<long long>(1, std::min<long long>(n_tiles, cap));
}

cudaError_t launch_tiled_fill(int dtype, int dim, int F, void* const* fields, const int* bc_kind, const void* const* bc,
                              const Geom* G, const TiledPlanDev& A, int grid, const int* g_geo,
                              const int* g_cell, const uint32_t* g_meta, const int* g_dep, const void* wtab,
                              int ng, void* xbuf, unsigned* bar, int extra_arrivals, int* status,
                              cudaStream_t s) {
  TiledFields P;
  for (int f = 0; f < 8; ++f) {
    P.f[f] = f < F ? fields[f] : nullptr;
    P.bc[f] = f < F ? bc[f] : nullptr;
    P.kind[f] = f < F ? bc_kind[f] : 0;
  }
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(TL_T);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (dtype == 0 && dim == 2)
    return cudaLaunchKernelEx(&cfg, k_tiled_fill<float, 2>, P, F, G, A, g_geo, g_cell, g_meta, g_dep, (const float*)wtab, ng,
                              static_cast<float*>(xbuf), bar, extra_arrivals, status);
  if (dtype == 0)
    return cudaLaunchKernelEx(&cfg, k_tiled_fill<float, 3>, P, F, G, A, g_geo, g_cell, g_meta, g_dep, (const float*)wtab, ng,
                              static_cast<float*>(xbuf), bar, extra_arrivals, status);
  if (dim == 2)
    return cudaLaunchKernelEx(&cfg, k_tiled_fill<double, 2>, P, F, G, A, g_geo, g_cell, g_meta, g_dep, (const double*)wtab, ng,
                              static_cast<double*>(xbuf), bar, extra_arrivals, status);
  return cudaLaunchKernelEx(&cfg, k_tiled_fill<double, 3>, P, F, G, A, g_geo, g_cell, g_meta, g_dep, (const double*)wtab, ng,
                            static_cast<double*>(xbuf), bar, extra_arrivals, status);
}

}  // namespace ebr
