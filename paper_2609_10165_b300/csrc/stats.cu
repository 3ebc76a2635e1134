// Stability diagnostics of a ghost set (Sec. 7, Eq. stability_alpha_max):
// per ghost and axis the normalized ghost-to-boundary distance
//   alpha_i = (x_s,i - x_1,i) / (x_2,i - x_1,i),
// x_1 the ghost centre, x_s its boundary point, x_2 the diagonally opposite
// stencil point (r_i e_i cells away); alpha_i < 0 for a ghost whose centre
// lies in the fluid.  Per geometry the largest and smallest alpha_i, over all
// ghosts a histogram of alpha_i and one of the multipliers r_i.  Integer
// counts and order-free extrema: the results do not depend on the schedule.
#include "ebr_kernels.cuh"
#include "ebr_probe.cuh"

namespace ebr {

// doubles ordered as unsigned integers (atomicMax / atomicMin on the bits)
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | (1ull << 63));
}

__global__ void k_stats(const Geom* __restrict__ G, int ng, const int* __restrict__ g_geo,
                        const int* __restrict__ g_cell, const double* __restrict__ g_psi,
                        const double* __restrict__ g_n, const uint32_t* __restrict__ g_meta, int n_bins,
                        unsigned long long* __restrict__ ext, unsigned long long* __restrict__ ahist,
                        unsigned long long* __restrict__ rhist) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ng) return;
  const int b = g_geo[p];
  const Geom& g = G[b];
  const uint32_t m = g_meta[p];
  const double psi = g_psi[p];
  int ijk[3];
  cell_ijk3(g, g_cell[p], ijk);
  for (int a = 0; a < g.dim; ++a) {
    const int r = meta_r(m, a), step = r * meta_e(m, a);
    double X2;
    if (g.stretched) {
      const int far = min(max(ijk[a] + step, 0), g.n[a] - 1);
      X2 = g.cen[a][far] - g.cen[a][ijk[a]];
    } else {
      X2 = step * g.h[a];
    }
    const double alpha = psi * g_n[(size_t)a * ng + p] / X2;
    atomicMax(&ext[(size_t)b * 6 + a], ordered_bits(alpha));
    atomicMax(&ext[(size_t)b * 6 + 3 + a], ordered_bits(-alpha));   // largest -alpha: smallest alpha
    int bin = (int)floor((alpha + 0.5) / 1.5 * n_bins);
    bin = min(max(bin, 0), n_bins - 1);
    atomicAdd(&ahist[(size_t)a * n_bins + bin], 1ull);
    atomicAdd(&rhist[(size_t)a * 16 + min(r, 15)], 1ull);
  }
}

void launch_stats(const Geom* G, int ng, const int* g_geo, const int* g_cell, const double* g_psi,
                  const double* g_n, const uint32_t* g_meta, int n_bins, unsigned long long* ext,
                  unsigned long long* ahist, unsigned long long* rhist, cudaStream_t s) {
  if (ng <= 0) return;
  k_stats<<<(ng + 127) / 128, 128, 0, s>>>(G, ng, g_geo, g_cell, g_psi, g_n, g_meta, n_bins, ext, ahist, rhist);
}

}  // namespace ebr
