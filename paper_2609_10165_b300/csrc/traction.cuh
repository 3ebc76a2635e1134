// Boundary traction of one ghost (Sec. 6), shared by the force kernels.
//
// p_s from the Dirichlet relation solved for phi_s, grad u at S from Eq.
// derivative_bilinear / Eqs. derivative_trilinear_x/y/z (both through the ftab
// coefficients: ftab[0] the surface element w_G, ftab[1 + s] the p_s weights,
// ftab[9 + 8 a + s] the d/dx_a weights of stencil value s, s = 0 the ghost),
// traction f = -p_s n + mu (grad u + grad u^T) n, weighted by w_G; the sums
// over ghosts in double.
#pragma once

#include "ebr_device.cuh"

namespace ebr {

struct VelSet {
  const void* u[3];      // velocity components (null: not present)
  const void* p;         // pressure
  double dirs[6];        // drag direction [D], lift direction [D]
};

// Adds ghost p's pressure force [0, D), viscous force [D, 2D), drag (2D) and
// lift (2D + 1) to acc.  The stencil values are read from the field arrays.
// The ghost's terms are computed in the field type from the coefficient
// table in that type (FP32 fields: the float copy of the double table, as the
// fill does with its weights; FP64 fields: all in double) and added to acc in
// double.
template <typename T, int D>
__device__ inline void ghost_traction(const VelSet& V, double mu, const Geom& g, int p,
                                      const int* __restrict__ g_cell, const double* __restrict__ g_n,
                                      const uint32_t* __restrict__ g_meta, const T* __restrict__ ftab,
                                      int ng, double acc[8]) {
  constexpr int K = D == 2 ? 3 : 7;
  const int nx = g.n[0], ny = g.n[1];
  const int cell = g_cell[p];
  const uint32_t m = g_meta[p];
  int slots[K + 1];
  slots[0] = cell;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int o[3];
    stencil_off(D, k, o);
    int off = o[0] * meta_r(m, 0) * meta_e(m, 0) + nx * (o[1] * meta_r(m, 1) * meta_e(m, 1));
    if (D == 3) off += nx * ny * (o[2] * meta_r(m, 2) * meta_e(m, 2));
    slots[k + 1] = cell + off;
  }
  T n[D];
#pragma unroll
  for (int a = 0; a < D; ++a) n[a] = (T)g_n[(size_t)a * ng + p];
  const T wG = (T)ftab[p];
  const T* pp = static_cast<const T*>(V.p) + g.cell_off;
  T ps = T(0);
#pragma unroll
  for (int s = 0; s <= K; ++s) ps += (T)ftab[(size_t)(1 + s) * ng + p] * pp[slots[s]];
  T Gm[D][D];                                             // Gm[i][a] = d u_i / d x_a
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int a = 0; a < D; ++a) Gm[i][a] = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    if (!V.u[i]) continue;
    const T* ui = static_cast<const T*>(V.u[i]) + g.cell_off;
#pragma unroll
    for (int s = 0; s <= K; ++s) {
      const T v = ui[slots[s]];
#pragma unroll
      for (int a = 0; a < D; ++a) Gm[i][a] += (T)ftab[(size_t)(9 + 8 * a + s) * ng + p] * v;
    }
  }
  const T muT = (T)mu;
  T dr = T(0), li = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const T fp = -ps * n[i] * wG;
    T t = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) t += (Gm[i][a] + Gm[a][i]) * n[a];
    const T fv = muT * t * wG;
    acc[i] += (double)fp;
    acc[D + i] += (double)fv;
    dr += (fp + fv) * (T)V.dirs[i];
    li += (fp + fv) * (T)V.dirs[D + i];
  }
  acc[2 * D] += (double)dr;
  acc[2 * D + 1] += (double)li;
}

}  // namespace ebr
