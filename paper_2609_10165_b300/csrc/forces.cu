// Boundary quantities and forces (Sec. 6).
//
// Per ghost the traction of traction.cuh (p_s, grad u at S, f = -p_s n +
// mu (grad u + grad u^T) n, weighted by w_G).  Ghosts are cut into chunks of at most
// 256 that never straddle geometries; each CTA reduces its chunk with a fixed
// tree, and the last chunk of a geometry to finish adds the chunk partials of
// the geometry in chunk order, so the sums are bitwise reproducible.
#include "ebr_kernels.cuh"
#include "traction.cuh"

namespace ebr {

constexpr int FC_T = 256;

// D (2 or 3) fixed at compile time keeps the per-ghost arrays in registers
template <typename T, int D>
__global__ void __launch_bounds__(FC_T) k_forces_chunk(VelSet V, double mu, const Geom* __restrict__ G,
                                                       const int4* __restrict__ chunks,
                                                       const int* __restrict__ g_cell,
                                                       const int* __restrict__ g_geo,
                                                       const double* __restrict__ g_n,
                                                       const uint32_t* __restrict__ g_meta,
                                                       const T* __restrict__ ftab, int ng,
                                                       double* __restrict__ partial,
                                                       const int* __restrict__ chunk_ptr,
                                                       int* __restrict__ done, int B,
                                                       double* __restrict__ out) {
  pdl_enter();
  // [quantity][thread]: a warp's 32 doubles of one quantity are contiguous
  // (no bank conflicts in the tree below)
  __shared__ double red[8][FC_T];
  int4 ch = chunks[blockIdx.x];        // (geometry, p0, p1, -)
  const Geom& g = G[ch.x];
  int p = ch.y + threadIdx.x;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (p < ch.z) ghost_traction<T, D>(V, mu, g, p, g_cell, g_n, g_meta, ftab, ng, acc);
  // fixed tree: at level w, element i < w becomes element i + element i + w
  // (w = 128, 64 in shared memory; 32 by warp 0 from shared memory; 16 .. 1
  // by shuffles, which add the same pairs in the same order)
#pragma unroll
  for (int q = 0; q < 8; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
#pragma unroll
  for (int w = FC_T / 2; w > 32; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 8; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = red[q][threadIdx.x] + red[q][threadIdx.x + 32];
#pragma unroll
    for (int w = 16; w > 0; w >>= 1)
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], w);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) partial[(size_t)blockIdx.x * 8 + q] = v[q];
      // the last chunk of the geometry to finish adds the chunk partials in
      // chunk order (the same sums whatever the order the chunks ran in) and
      // resets the geometry's counter for the next launch
      const int b = ch.x;
      const int c0 = chunk_ptr[b], nch = chunk_ptr[b + 1] - c0;
      __threadfence();
      if (atomicAdd(&done[b], 1) == nch - 1) {
        __threadfence();
        constexpr int W = 2 * D + 2;
        double sum[W];
#pragma unroll
        for (int q = 0; q < W; ++q) sum[q] = 0.0;
        for (int c = c0; c < c0 + nch; ++c)
#pragma unroll
          for (int q = 0; q < W; ++q) sum[q] += __ldcg(&partial[(size_t)c * 8 + q]);
#pragma unroll
        for (int q = 0; q < W; ++q) out[(size_t)b * W + q] = sum[q];
        atomicExch(&done[b], 0);
      }
    }
  }
  // geometries without ghosts have no chunk: zeros
  if (blockIdx.x == 0) {
    constexpr int W = 2 * D + 2;
    for (int b = threadIdx.x; b < B; b += FC_T)
      if (chunk_ptr[b + 1] == chunk_ptr[b])
#pragma unroll
        for (int q = 0; q < W; ++q) out[(size_t)b * W + q] = 0.0;
  }
}

// no ghost in the whole set: every output zero
__global__ void k_forces_zero(int n, double* __restrict__ out) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = 0.0;
}

void launch_forces(int dtype, int dim, const void* const* vel, const void* p, double mu,
                   const double* dirs, const Geom* G, int n_chunks, const int4* chunks,
                   const int* g_cell, const int* g_geo, const double* g_n, const uint32_t* g_meta,
                   const void* ftab, int ng_total, double* partial, int* done, int B, double* out,
                   const int* chunk_ptr, cudaStream_t s) {
  VelSet V;
  for (int i = 0; i < 3; ++i) V.u[i] = i < dim ? vel[i] : nullptr;
  V.p = p;
  for (int q = 0; q < 6; ++q) V.dirs[q] = q < 2 * dim ? dirs[q] : 0.0;
  if (n_chunks <= 0) {
    const int n = B * (2 * dim + 2);
    if (n > 0) launch(k_forces_zero, (n + 127) / 128, 128, 0, s, n, out);
    return;
  }
  if (dtype == 0 && dim == 2)
    launch(k_forces_chunk<float, 2>, n_chunks, FC_T, 0, s, V, mu, G, chunks, g_cell, g_geo, g_n, g_meta, (const float*)ftab,
           ng_total, partial, chunk_ptr, done, B, out);
  else if (dtype == 0)
    launch(k_forces_chunk<float, 3>, n_chunks, FC_T, 0, s, V, mu, G, chunks, g_cell, g_geo, g_n, g_meta, (const float*)ftab,
           ng_total, partial, chunk_ptr, done, B, out);
  else if (dim == 2)
    launch(k_forces_chunk<double, 2>, n_chunks, FC_T, 0, s, V, mu, G, chunks, g_cell, g_geo, g_n, g_meta, (const double*)ftab,
           ng_total, partial, chunk_ptr, done, B, out);
  else
    launch(k_forces_chunk<double, 3>, n_chunks, FC_T, 0, s, V, mu, G, chunks, g_cell, g_geo, g_n, g_meta, (const double*)ftab,
           ng_total, partial, chunk_ptr, done, B, out);
}

}  // namespace ebr
