// Boundary quantities and forces (Sec. 6).
//
// Per ghost the traction of traction.cuh (p_s, grad u at S, f = -p_s n +
// mu (grad u + grad u^T) n, weighted by w_G).  Ghosts are cut into chunks of at most
// 256 that never straddle geometries; each CTA reduces its chunk with a fixed
// tree, and a second kernel adds the chunk partials of each geometry in order,
// so the sums are bitwise reproducible.
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
                                                       const double* __restrict__ ftab, int ng,
                                                       double* __restrict__ partial) {
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
    if (threadIdx.x == 0)
#pragma unroll
      for (int q = 0; q < 8; ++q) partial[(size_t)blockIdx.x * 8 + q] = v[q];
  }
}

__global__ void k_forces_final(int B, const Geom* __restrict__ G, const int* __restrict__ chunk_ptr,
                               const double* __restrict__ partial, double* __restrict__ out) {
  pdl_enter();
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  int d = G[b].dim, W = 2 * d + 2;
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int c = chunk_ptr[b]; c < chunk_ptr[b + 1]; ++c)
    for (int q = 0; q < W; ++q) s[q] += partial[(size_t)c * 8 + q];
  for (int q = 0; q < W; ++q) out[(size_t)b * W + q] = s[q];
}

void launch_forces(int dtype, int dim, const void* const* vel, const void* p, double mu,
                   const double* dirs, const Geom* G, int n_chunks, const int4* chunks,
                   const int* g_cell, const int* g_geo, const double* g_n, const uint32_t* g_meta,
                   const double* ftab, int ng_total, double* partial, int B, double* out,
                   const int* chunk_ptr, cudaStream_t s) {
  VelSet V;
  for (int i = 0; i < 3; ++i) V.u[i] = i < dim ? vel[i] : nullptr;
  V.p = p;
  for (int q = 0; q < 6; ++q) V.dirs[q] = q < 2 * dim ? dirs[q] : 0.0;
  if (n_chunks > 0) {
    if (dtype == 0 && dim == 2)
      launch(k_forces_chunk<float, 2>, n_chunks, FC_T, 0, s, V, mu, G, chunks, g_cell, g_geo, g_n, g_meta, ftab, ng_total, partial);
    else if (dtype == 0)
      launch(k_forces_chunk<float, 3>, n_chunks, FC_T, 0, s, V, mu, G, chunks, g_cell, g_geo, g_n, g_meta, ftab, ng_total, partial);
    else if (dim == 2)
      launch(k_forces_chunk<double, 2>, n_chunks, FC_T, 0, s, V, mu, G, chunks, g_cell, g_geo, g_n, g_meta, ftab, ng_total, partial);
    else
      launch(k_forces_chunk<double, 3>, n_chunks, FC_T, 0, s, V, mu, G, chunks, g_cell, g_geo, g_n, g_meta, ftab, ng_total, partial);
  }
  launch(k_forces_final, (B + 127) / 128, 128, 0, s, B, G, chunk_ptr, partial, out);
}

}  // namespace ebr
