// Device-side data structures and geometry for the ghost-cell library.
//
// Geometry (Sec. 3.1): cell centres x_a = lo_a + (i_a + 1/2) h_a; a cell is
// solid when its centre lies in the closed body (psi >= 0, Eq.
// signed_distance).  psi, the boundary point S and the unit normal n (into the
// fluid) are evaluated in double only on cells next to the boundary.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ebr {

enum BodyKind { CIRCLE = 0, SPHERE = 1, ELLIPSE = 2, AIRFOIL4 = 3 };
enum Placement { HGC = 0, CGC = 1, CGC_ES = 2 };

// status codes (same values as ebr_status)
enum Status {
  S_OK = 0, S_EINVAL = -1, S_ENOMEM = -2, S_ECUDA = -3, S_ECYCLE = -4,
  S_ESTENCIL_OOB = -5, S_ESTENCIL_SOLID = -6, S_ETIMEOUT = -7, S_ENONFINITE = -8,
  S_ESHAPE = -9
};

constexpr int MAXK = 7;      // stencil members in 3D (P1..P7)

// One geometry (grid + body) as the kernels see it.
struct Geom {
  int dim;
  int n[3];
  double lo[3];
  double h[3];
  int kind;
  int placement;
  double centre[3];
  double radii[3];
  double rot[9];        // body -> world, row-major
  double t, c;          // airfoil thickness and chord
  long long cell_off;   // first flat cell
  int row_off;          // first flat row (rows run along x)
  int n_rows;           // n[1] * n[2]
  // planned sizes / offsets (filled after the planning pass)
  int iface_off, n_iface;
  int ghost_off, n_ghost;
  int lev_off, n_levels;     // level pointers at lev_ptr[lev_off .. lev_off + n_levels]
  // float copies for the float pre-decisions (no double work or conversions
  // per cell); hgc_mrg = safety margin of the float HGC decision
  float flo[3], fh[3], fcentre[3], fradii[3], frot[9], ft, fc, hgc_mrg;
  float fext;                // max(1, largest |grid corner - centre| over the axes)
  // second ghost layer (Sec. 7): layers = 2 adds the solid cells with
  // psi <= 1.5 dn; reach = box (cells per axis) holding a fluid cell for each
  int layers;
  int reach[3];
  // stretched grids (Sec. 7, local mesh spacing): per axis the cell centres,
  // widths and float centres (device arrays of n_a entries, owned by the
  // context); lo then holds the first face and h the smallest width per axis.
  // stretched == 0: uniform, centres lo + (i + 1/2) h.
  int stretched;
  double hmax;               // largest cell width over the axes
  double span[3];            // last face minus first face per axis (stretched grids)
  const double* cen[3];
  const double* wid[3];
  const float* fcen[3];
};

// ---------------------------------------------------------------------------
// ghost meta word
//   bits 0..2   e_a < 0 (sign of the normal component; n_a = 0 -> e_a = +1)
//   bits 3..14  r_x, r_y, r_z (4 bits each)
//   bits 15..21 active mask of P_1..P_K (structurally non-zero weight)
//   bit  22     centre in the fluid (tag -2)
//   bits 23..29 member k is itself a ghost (dependency)
// ---------------------------------------------------------------------------
__host__ __device__ inline int meta_e(uint32_t m, int a) { return (m >> a) & 1u ? -1 : 1; }
__host__ __device__ inline int meta_r(uint32_t m, int a) { return (m >> (3 + 4 * a)) & 15u; }
__host__ __device__ inline uint32_t meta_active(uint32_t m) { return (m >> 15) & 127u; }
__host__ __device__ inline bool meta_fluid(uint32_t m) { return (m >> 22) & 1u; }
__host__ __device__ inline uint32_t meta_depmask(uint32_t m) { return (m >> 23) & 127u; }

// Offsets of P_1..P_K in units of r_a e_a h_a (Secs. 4 and 5, Appendix A).
__host__ __device__ inline int stencil_k(int dim) { return dim == 2 ? 3 : 7; }
__host__ __device__ inline void stencil_off(int dim, int k, int o[3]) {
  // 3 bits (x, y, z) per member: 2D P1..P3 = (1,0), (0,1), (1,1);
  // 3D P1..P7 = (1,0,0), (0,1,0), (0,0,1), (1,1,0), (0,1,1), (1,0,1), (1,1,1)
  const unsigned code = dim == 2 ? (1u | 2u << 3 | 3u << 6)
                                 : (1u | 2u << 3 | 4u << 6 | 3u << 9 | 6u << 12 | 5u << 15 | 7u << 18);
  unsigned v = code >> (3 * k);
  o[0] = v & 1u;
  o[1] = (v >> 1) & 1u;
  o[2] = (v >> 2) & 1u;
}

// Structurally active members (meta bits 15..21 before the grid and tag
// checks): P_k drops out when its offset runs along an axis on which the
// normal has no component (zero: bit a set when n_a == 0).
__host__ __device__ inline uint32_t active_of_zero(int dim, uint32_t zero) {
  uint32_t act = 0;
  for (int k = 0; k < stencil_k(dim); ++k) {
    int o[3];
    stencil_off(dim, k, o);
    bool on = true;
    for (int a = 0; a < dim; ++a)
      if (o[a] && (zero >> a & 1u)) on = false;
    if (on) act |= 1u << k;
  }
  return act;
}

// Cell centre along axis a, evaluated without contraction (uniform grids).
__device__ __forceinline__ double centre_of(const Geom& g, int a, int i) {
  if (g.stretched) return g.cen[a][i];
  return __dadd_rn(g.lo[a], __dmul_rn((double)i + 0.5, g.h[a]));
}

// Width of cell i along axis a.
__device__ __forceinline__ double width_of(const Geom& g, int a, int i) {
  return g.stretched ? g.wid[a][i] : g.h[a];
}

// Float centre along axis a (the float pre-tests; their margins cover the
// rounding of either form by a wide factor).
__device__ __forceinline__ float fcentre_of(const Geom& g, int a, int i) {
  return g.stretched ? g.fcen[a][i] : g.flo[a] + ((float)i + 0.5f) * g.fh[a];
}

// ---------------------------------------------------------------------------
// inside predicate (solid <=> psi >= 0), double, no contraction
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sq(double v) { return __dmul_rn(v, v); }

__device__ inline double airfoil_yt(double t, double c, double x) {
  // y_t(x) = 5 t c [a0 sqrt(xi) + a1 xi + a2 xi^2 + a3 xi^3 + a4 xi^4], xi = x / c
  double xi = __ddiv_rn(x, c);
  double poly = __dadd_rn(-0.1260, __dmul_rn(xi, __dadd_rn(-0.3516, __dmul_rn(xi, __dadd_rn(0.2843, __dmul_rn(xi, -0.1015))))));
  double s = __dadd_rn(__dmul_rn(0.2969, __dsqrt_rn(xi)), __dmul_rn(xi, poly));
  return __dmul_rn(__dmul_rn(__dmul_rn(5.0, t), c), s);
}

__device__ inline void to_body2(const Geom& g, double x, double y, double& px, double& py) {
  double dx = __dadd_rn(x, -g.centre[0]);
  double dy = __dadd_rn(y, -g.centre[1]);
  px = __dadd_rn(__dmul_rn(g.rot[0], dx), __dmul_rn(g.rot[3], dy));
  py = __dadd_rn(__dmul_rn(g.rot[1], dx), __dmul_rn(g.rot[4], dy));
}

__device__ inline bool solid_at(const Geom& g, double x, double y, double z) {
  switch (g.kind) {
    case CIRCLE: {
      double q = __dadd_rn(sq(__dadd_rn(x, -g.centre[0])), sq(__dadd_rn(y, -g.centre[1])));
      return __dsqrt_rn(q) <= g.radii[0];
    }
    case SPHERE: {
      double q = __dadd_rn(__dadd_rn(sq(__dadd_rn(x, -g.centre[0])), sq(__dadd_rn(y, -g.centre[1]))),
                           sq(__dadd_rn(z, -g.centre[2])));
      return __dsqrt_rn(q) <= g.radii[0];
    }
    case ELLIPSE: {
      double px, py;
      to_body2(g, x, y, px, py);
      double qx = __ddiv_rn(px, g.radii[0]);
      double qy = __ddiv_rn(py, g.radii[1]);
      return __dadd_rn(sq(qx), sq(qy)) <= 1.0;
    }
    default: {  // AIRFOIL4
      double px, py;
      to_body2(g, x, y, px, py);
      if (!(px >= 0.0 && px <= g.c)) return false;
      return fabs(py) <= airfoil_yt(g.t, g.c, px);
    }
  }
}

__device__ inline bool solid_cell(const Geom& g, int i, int j, int k) {
  double x = centre_of(g, 0, i), y = centre_of(g, 1, j);
  double z = g.dim == 3 ? centre_of(g, 2, k) : 0.0;
  return solid_at(g, x, y, z);
}

// ---------------------------------------------------------------------------
// closest point: unsigned distance and unit normal (world frame, into fluid)
// ---------------------------------------------------------------------------

// Ellipse x^2/a^2 + y^2/b^2 = 1, body-frame point (p, q).  Closest point
// X = a^2 p / (a^2 + t), Y = b^2 q / (b^2 + t) where t solves
// F(t) = (a p / (a^2 + t))^2 + (b q / (b^2 + t))^2 - 1 = 0.  F is decreasing and
// convex on t > -min(a^2, b^2), so safeguarded Newton from t = 0 converges.
// The iteration runs in float first; a few double steps then polish t to
// the rounding level (the FP64 pipe is the scarce resource).
__device__ inline void ellipse_closest(double a, double b, double p, double q,
                                       double& dist, double& nx, double& ny) {
  double a2 = a * a, b2 = b * b;
  double tmin = -fmin(a2, b2);
  float af = (float)a, bf = (float)b, pf = (float)p, qf = (float)q;
  float a2f = af * af, b2f = bf * bf, tminf = (float)tmin;
  float tf = 0.0f;
  for (int it = 0; it < 16; ++it) {
    float rua = 1.0f / (a2f + tf), rub = 1.0f / (b2f + tf);
    float fx = af * pf * rua, fy = bf * qf * rub;
    float F = fx * fx + fy * fy - 1.0f;
    float dF = -2.0f * (fx * fx * rua + fy * fy * rub);
    if (F == 0.0f || dF == 0.0f) break;
    float tn = tf - F / dF;
    if (!(tn > tminf)) tn = 0.5f * (tf + tminf);
    float dt = fabsf(tn - tf);
    tf = tn;
    if (dt <= 1e-5f * fabsf(tf)) break;
  }
  double t = (double)tf;
  if (!(t > tmin)) t = 0.0;
  // Halley steps in double (cubic convergence; the increment in float): from
  // the float solution one step leaves an error of about the float rounding of
  // the increment (~1e-14 relative), so a step of <= 1e-6 relative is final;
  // the reciprocals at the new t follow from the last ones to second order,
  // 1/(u + d) = (1/u)(1 - e + e^2), e = d/u, error O(e^3)
  double rua = 0.0, rub = 0.0;
  bool have = false;
  for (int it = 0; it < 12; ++it) {
    // one double reciprocal per iteration: 1/(a^2+t) and 1/(b^2+t) from
    // 1/((a^2+t)(b^2+t))
    const double ua = a2 + t, ub = b2 + t;
    const double r = 1.0 / (ua * ub);
    rua = ub * r;
    rub = ua * r;
    const double fx = a * p * rua, fy = b * q * rub;
    const double fx2 = fx * fx, fy2 = fy * fy;
    const double F = fx2 + fy2 - 1.0;
    const double dF = -2.0 * (fx2 * rua + fy2 * rub);
    if (F == 0.0 || dF == 0.0) { have = true; break; }
    const double d2F = 6.0 * (fx2 * rua * rua + fy2 * rub * rub);
    const float Ff = (float)F, dFf = (float)dF, d2Ff = (float)d2F;
    const float den = 2.0f * dFf * dFf - Ff * d2Ff;
    const float step = den > 0.0f ? 2.0f * Ff * dFf / den : Ff / dFf;
    double tn = t - (double)step;
    if (!(tn > tmin)) tn = 0.5 * (t + tmin);
    const double d = tn - t;
    t = tn;
    if (fabs(d) <= 1e-6 * fabs(t)) {
      const double ea = d * rua, eb = d * rub;
      rua = rua * (1.0 - ea + ea * ea);
      rub = rub * (1.0 - eb + eb * eb);
      have = true;
      break;
    }
  }
  if (!have) {
    const double ua = a2 + t, ub = b2 + t;
    const double r = 1.0 / (ua * ub);
    rua = ub * r;
    rub = ua * r;
  }
  // G - S = (p t / ua, q t / ub): no cancellation; the outward normal at S is
  // along (X / a^2, Y / b^2) = (p / ua, q / ub)
  const double ex = p * t * rua, ey = q * t * rub;
  dist = sqrt(ex * ex + ey * ey);
  const double mx = p * rua, my = q * rub;
  const double inv = rsqrt(mx * mx + my * my);
  nx = mx * inv;
  ny = my * inv;
}

// Upper airfoil surface as polynomials in u = sqrt(x / c).
// Nested (Horner) form in u^2: y/k = a0 u + u^2 (a1 + u^2 (a2 + u^2 (a3 + u^2 a4))),
// its derivatives likewise -- about a third of the double operations of the
// power sums (the double pipe is the bound of the closest-point kernel).
__device__ inline void airfoil_u(double t, double c, double u, double& x, double& y,
                                 double& dx, double& dy, double& ddx, double& ddy) {
  const double a0 = 0.2969, a1 = -0.1260, a2 = -0.3516, a3 = 0.2843, a4 = -0.1015;
  const double k = 5.0 * t * c;
  const double u2 = u * u;
  x = c * u2;
  y = k * fma(a0, u, u2 * fma(u2, fma(u2, fma(u2, a4, a3), a2), a1));
  dx = 2.0 * c * u;
  dy = k * fma(u, fma(u2, fma(u2, fma(u2, 8.0 * a4, 6.0 * a3), 4.0 * a2), 2.0 * a1), a0);
  ddx = 2.0 * c;
  ddy = k * fma(u2, fma(u2, fma(u2, 56.0 * a4, 30.0 * a3), 12.0 * a2), 2.0 * a1);
}

// d^3 y / du^3 of the upper surface (x is quadratic in u: its third derivative is 0)
__device__ inline double airfoil_dddy(double t, double c, double u) {
  const double a2 = -0.3516, a3 = 0.2843, a4 = -0.1015;
  const double u2 = u * u;
  return 5.0 * t * c * u * fma(u2, fma(u2, 336.0 * a4, 120.0 * a3), 24.0 * a2);
}

__device__ inline void airfoil_u32(float t, float c, float u, float& x, float& y, float& dx,
                                   float& dy, float& ddx, float& ddy) {
  const float a0 = 0.2969f, a1 = -0.1260f, a2 = -0.3516f, a3 = 0.2843f, a4 = -0.1015f;
  float k = 5.0f * t * c;
  float u2 = u * u, u3 = u2 * u, u4 = u2 * u2, u5 = u4 * u, u6 = u4 * u2, u7 = u6 * u, u8 = u4 * u4;
  x = c * u2;
  y = k * (a0 * u + a1 * u2 + a2 * u4 + a3 * u6 + a4 * u8);
  dx = 2.0f * c * u;
  dy = k * (a0 + 2.0f * a1 * u + 4.0f * a2 * u3 + 6.0f * a3 * u5 + 8.0f * a4 * u7);
  ddx = 2.0f * c;
  ddy = k * (2.0f * a1 + 12.0f * a2 * u2 + 30.0f * a3 * u4 + 56.0f * a4 * u6);
}

// Closest point on the airfoil to the body-frame point (px, py): the upper
// surface by coarse float sampling in u, float Newton on
// g(u) = (P(u) - q) . P'(u) inside the bracket, and a double polish of u; the
// base x = c; the lower surface by symmetry (|py|, exact ties -> upper
// surface).  At the trailing-edge corner a fluid point's normal is
// (G - S) / |G - S|.
__device__ inline void airfoil_closest(double t, double c, double px, double py, bool inside,
                                       double& dist, double& nx, double& ny) {
  double qx = px, qy = fabs(py);
  const int NS = 64;
  float fqx = (float)qx, fqy = (float)qy, fc = (float)c, ft = (float)t;
  int best = 0;
  float bd = 3.4e38f;
  for (int s = 0; s <= NS; ++s) {
    float u = (float)s / NS;
    float u2 = u * u;
    float x = fc * u2;
    float y = 5.0f * ft * fc * (0.2969f * u + u2 * (-0.1260f + u2 * (-0.3516f + u2 * (0.2843f + u2 * -0.1015f))));
    float d = (x - fqx) * (x - fqx) + (y - fqy) * (y - fqy);
    if (d < bd) { bd = d; best = s; }
  }
  double lo = fmax(0.0, (double)(best - 1) * (1.0 / NS)), hi = fmin(1.0, (double)(best + 1) * (1.0 / NS));
  // surface point, first and second derivatives at the last evaluated u
  double x = 0.0, y = 0.0, dx = 0.0, dy = 0.0, ddx = 0.0, ddy = 0.0;
  auto g = [&](double u, double& gv, double& dg) {
    airfoil_u(t, c, u, x, y, dx, dy, ddx, ddy);
    gv = (x - qx) * dx + (y - qy) * dy;
    dg = dx * dx + dy * dy + (x - qx) * ddx + (y - qy) * ddy;
  };
  // sign of g at a bracket end: in float where it is clearly away from zero
  // (the margin bounds the float rounding of both products by a wide
  // factor), in double otherwise
  auto end_sign = [&](double ue) -> int {
    float xf, yf, dxf, dyf, ddxf, ddyf;
    airfoil_u32(ft, fc, (float)ue, xf, yf, dxf, dyf, ddxf, ddyf);
    const float gf = (xf - fqx) * dxf + (yf - fqy) * dyf;
    const float m = 1e-5f * (1.0f + fabsf(xf) + fabsf(fqx) + fabsf(yf) + fabsf(fqy)) * (fabsf(dxf) + fabsf(dyf));
    if (gf > m) return 1;
    if (gf < -m) return -1;
    double gv, dg;
    g(ue, gv, dg);
    return gv > 0.0 ? 1 : (gv < 0.0 ? -1 : 0);
  };
  double u;
  bool have = false;           // x .. ddy hold the values at u
  if (end_sign(lo) >= 0) {
    u = lo;                    // distance increases from lo on (lo == 0 here)
  } else if (end_sign(hi) <= 0) {
    u = hi;                    // distance decreases up to hi (hi == 1 here)
  } else {
    // float Newton inside the bracket
    float flo = (float)lo, fhi = (float)hi, uf = 0.5f * (flo + fhi);
    for (int it = 0; it < 16; ++it) {
      float x, y, dx, dy, ddx, ddy;
      airfoil_u32(ft, fc, uf, x, y, dx, dy, ddx, ddy);
      float gv = (x - fqx) * dx + (y - fqy) * dy;
      float dg = dx * dx + dy * dy + (x - fqx) * ddx + (y - fqy) * ddy;
      if (gv == 0.0f) break;
      // converged: accept the (tiny) Newton step before any safeguard
      if (dg > 0.0f && fabsf(gv / dg) <= 1e-5f * fmaxf(uf, 1e-3f)) {
        uf = fminf(fmaxf(uf - gv / dg, flo), fhi);
        break;
      }
      if (gv < 0.0f) flo = uf; else fhi = uf;
      float un = uf - gv / dg;
      if (!(un > flo && un < fhi) || dg <= 0.0f) un = 0.5f * (flo + fhi);
      uf = un;
    }
    u = fmin(fmax((double)uf, lo), hi);
    // double polish: safeguarded Halley steps inside [lo, hi] (cubic
    // convergence; the increment in float).  From the float solution one step
    // leaves an error of about the float rounding of the increment (~1e-14
    // relative), so a step of <= 1e-6 relative is final: the point and its
    // tangent at the new u follow from the last evaluation by Taylor
    // expansion -- x exactly (it is quadratic in u), y and y' to third order
    // (the neglected terms are ~step^4 and ~step^3).
    for (int it = 0; it < 40; ++it) {
      double gv, dg;
      g(u, gv, dg);
      if (gv == 0.0) { have = true; break; }
      const double dddy = airfoil_dddy(t, c, u);
      const double d2g = 3.0 * (dx * ddx + dy * ddy) + (y - qy) * dddy;
      double st = 0.0;
      if (dg > 0.0) {
        const float gf = (float)gv, dgf = (float)dg, d2f = (float)d2g;
        const float den = 2.0f * dgf * dgf - gf * d2f;
        st = den > 0.0f ? (double)(2.0f * gf * dgf / den) : (double)(gf / dgf);
      }
      if (dg > 0.0 && fabs(st) <= 1e-6 * fmax(u, 1e-3)) {
        const double un = fmin(fmax(u - st, lo), hi), du = un - u;
        const double h2 = 0.5 * du * du;
        x += dx * du + ddx * h2;
        y += dy * du + ddy * h2 + dddy * h2 * du * (1.0 / 3.0);
        dx += ddx * du;
        dy += ddy * du + dddy * h2;
        u = un;
        have = true;
        break;
      }
      if (gv < 0.0) lo = u; else hi = u;
      double un = u - st;
      if (!(un > lo && un < hi) || dg <= 0.0) un = 0.5 * (lo + hi);
      u = un;
    }
  }
  if (!have) airfoil_u(t, c, u, x, y, dx, dy, ddx, ddy);
  double d2u = (x - qx) * (x - qx) + (y - qy) * (y - qy);
  // half thickness at the trailing edge: the polynomial at u = 1
  const double yte = 5.0 * t * c * (0.2969 + -0.1260 + -0.3516 + 0.2843 + -0.1015);
  double by = fmin(qy, yte);
  double d2b = (qx - c) * (qx - c) + (qy - by) * (qy - by);
  double sx, sy;
  bool base = d2b < d2u;
  if (base) {
    sx = c; sy = by; nx = 1.0; ny = 0.0;
  } else {
    sx = x; sy = y;
    const double inv = rsqrt(dx * dx + dy * dy);
    nx = -dy * inv;
    ny = dx * inv;
  }
  bool corner = !inside && ((base && qy > yte) || (!base && u == 1.0));
  if (corner) {
    sx = c; sy = yte;
    const double vx = qx - c, vy = qy - yte, inv = rsqrt(vx * vx + vy * vy);
    nx = vx * inv;
    ny = vy * inv;
  }
  dist = sqrt((qx - sx) * (qx - sx) + (qy - sy) * (qy - sy));
  if (py < 0.0) ny = -ny;
}

// ---------------------------------------------------------------------------
// float closest point, used to decide HGC candidacy away from the
// thresholds (a cell whose float decision is within a safety margin of a
// threshold is decided with the double closest point instead) and the sign
// and zero pattern of the normal.  *unsure (when given) is set where the
// normal's signs and zeros may differ from the double closest point's: a
// component within 1e-3 of zero, a foot point whose position is
// ill-conditioned (the point within a quarter of the radius of curvature of
// the evolute, where a perturbation of the input moves the normal by several
// times itself), a near tie between two branches of the airfoil's closest
// point (surface or base, upper or lower surface).
// ---------------------------------------------------------------------------
__device__ inline float closest_point_f32(const Geom& g, float x, float y, float z, bool solid,
                                          float n[3], bool* unsure = nullptr) {
  n[0] = n[1] = n[2] = 0.0f;
  float dist = 0.0f;
  bool ill = false;
  switch (g.kind) {
    case CIRCLE:
    case SPHERE: {
      float dx = x - g.fcentre[0], dy = y - g.fcentre[1];
      float dz = g.kind == SPHERE ? z - g.fcentre[2] : 0.0f;
      float rho = sqrtf(dx * dx + dy * dy + dz * dz);
      float r = 1.0f / fmaxf(rho, 1e-30f);
      dist = fabsf(g.fradii[0] - rho);
      n[0] = dx * r; n[1] = dy * r; n[2] = dz * r;
      ill = rho < 0.25f * g.fradii[0];
      break;
    }
    case ELLIPSE: {
      const float wx = x - g.fcentre[0], wy = y - g.fcentre[1];
      const float p = g.frot[0] * wx + g.frot[3] * wy, q = g.frot[1] * wx + g.frot[4] * wy;
      const float a = g.fradii[0], b = g.fradii[1];
      float a2 = a * a, b2 = b * b, tmin = -fminf(a2, b2), t = 0.0f;
      bool conv = false;
      for (int it = 0; it < 16; ++it) {
        float rua = 1.0f / (a2 + t), rub = 1.0f / (b2 + t);
        float fx = a * p * rua, fy = b * q * rub;
        float F = fx * fx + fy * fy - 1.0f;
        float dF = -2.0f * (fx * fx * rua + fy * fy * rub);
        if (F == 0.0f || dF == 0.0f) { conv = true; break; }
        float tn = t - F / dF;
        if (!(tn > tmin)) tn = 0.5f * (t + tmin);
        float dt = fabsf(tn - t);
        t = tn;
        // converged: a step small against t, or against a^2 + t and b^2 + t
        // (which set the normal; near the boundary t itself is near 0 and the
        // float rounding of F keeps the steps above 1e-5 |t|)
        if (dt <= 1e-5f * fabsf(t) || dt <= 1e-6f * fminf(a2 + t, b2 + t)) { conv = true; break; }
      }
      float rua = 1.0f / (a2 + t), rub = 1.0f / (b2 + t);
      float ex = p * t * rua, ey = q * t * rub;
      dist = sqrtf(ex * ex + ey * ey);
      float mx = p * rua, my = q * rub;           // (X / a^2, Y / b^2)
      float mn = 1.0f / sqrtf(mx * mx + my * my);
      float bx = mx * mn, by = my * mn;
      n[0] = g.frot[0] * bx + g.frot[1] * by;
      n[1] = g.frot[3] * bx + g.frot[4] * by;
      // inside (t < 0) near the evolute a^2 + t or b^2 + t approaches 0
      ill = !conv || a2 + t < 0.25f * a2 || b2 + t < 0.25f * b2;
      break;
    }
    default: {  // AIRFOIL4
      const float wx = x - g.fcentre[0], wy = y - g.fcentre[1];
      const float qd = g.frot[1] * wx + g.frot[4] * wy;
      const float c = g.fc, t = g.ft, qx = g.frot[0] * wx + g.frot[3] * wy, qy = fabsf(qd);
      const int NS = 64;
      int best = 0;
      float bd = 3.4e38f;
      for (int s = 0; s <= NS; ++s) {
        float u = (float)s / NS, u2 = u * u, xx = c * u2;
        float yy = 5.0f * t * c * (0.2969f * u + u2 * (-0.1260f + u2 * (-0.3516f + u2 * (0.2843f + u2 * -0.1015f))));
        float d = (xx - qx) * (xx - qx) + (yy - qy) * (yy - qy);
        if (d < bd) { bd = d; best = s; }
      }
      float lo = fmaxf(0.0f, (float)(best - 1) / NS), hi = fminf(1.0f, (float)(best + 1) / NS);
      float xx, yy, dx, dy, ddx, ddy;
      airfoil_u32(t, c, lo, xx, yy, dx, dy, ddx, ddy);
      float glo = (xx - qx) * dx + (yy - qy) * dy;
      airfoil_u32(t, c, hi, xx, yy, dx, dy, ddx, ddy);
      float ghi = (xx - qx) * dx + (yy - qy) * dy;
      float u;
      bool conv = true;
      if (glo >= 0.0f) u = lo;
      else if (ghi <= 0.0f) u = hi;
      else {
        u = 0.5f * (lo + hi);
        conv = false;
        for (int it = 0; it < 16; ++it) {
          airfoil_u32(t, c, u, xx, yy, dx, dy, ddx, ddy);
          float gv = (xx - qx) * dx + (yy - qy) * dy;
          float dg = dx * dx + dy * dy + (xx - qx) * ddx + (yy - qy) * ddy;
          if (gv == 0.0f) { conv = true; break; }
          // converged: a step below 1e-5 u, or below 1e-6 (near the leading
          // edge the float rounding of g keeps the steps above 1e-5 u; the
          // distance is stationary in u at the foot point, the normal moves
          // by about |P''| / |P'| times the step)
          if (dg > 0.0f && fabsf(gv / dg) <= fmaxf(1e-5f * fmaxf(u, 1e-3f), 1e-6f)) {
            u = fminf(fmaxf(u - gv / dg, lo), hi);
            conv = true;
            break;
          }
          if (gv < 0.0f) lo = u; else hi = u;
          float un = u - gv / dg;
          if (!(un > lo && un < hi) || dg <= 0.0f) un = 0.5f * (lo + hi);
          u = un;
        }
      }
      airfoil_u32(t, c, u, xx, yy, dx, dy, ddx, ddy);
      float d2u = (xx - qx) * (xx - qx) + (yy - qy) * (yy - qy);
      float yte, t1, t2, t3, t4, t5;
      airfoil_u32(t, c, 1.0f, t1, yte, t2, t3, t4, t5);
      float byy = fminf(qy, yte);
      float d2b = (qx - c) * (qx - c) + (qy - byy) * (qy - byy);
      // second derivative of the squared distance along the surface, |P'|^2
      // (1 - d kappa) at the foot point: small near the evolute
      const float tt = dx * dx + dy * dy;
      const float dg = tt + (xx - qx) * ddx + (yy - qy) * ddy;
      ill = !conv || fabsf(qd) <= 1e-4f * c || fabsf(d2b - d2u) <= 1e-2f * (d2b + d2u) ||
            (!(d2b < d2u) && dg < 0.25f * tt);
      float bx, by;
      if (d2b < d2u) {
        dist = sqrtf(d2b);
        bx = 1.0f; by = 0.0f;
        if (!solid && qy > yte) {
          float vx = qx - c, vy = qy - yte, vn = 1.0f / fmaxf(sqrtf(vx * vx + vy * vy), 1e-30f);
          bx = vx * vn; by = vy * vn;
        }
      } else {
        dist = sqrtf(d2u);
        float fn = 1.0f / sqrtf(dx * dx + dy * dy);
        bx = -dy * fn; by = dx * fn;
      }
      if (qd < 0.0f) by = -by;
      n[0] = g.frot[0] * bx + g.frot[1] * by;
      n[1] = g.frot[3] * bx + g.frot[4] * by;
      break;
    }
  }
  if (unsure) {
    for (int a = 0; a < g.dim; ++a) ill = ill || fabsf(n[a]) < 1e-3f;
    *unsure = ill;
  }
  return solid ? dist : -dist;
}

// psi (signed by the solid flag) and world-frame unit normal for a cell centre.
// Returns false when the normal is undefined (centre at a circle's centre).
__device__ inline bool closest_point(const Geom& g, double x, double y, double z, bool solid,
                                     double& psi, double n[3]) {
  n[0] = n[1] = n[2] = 0.0;
  double dist;
  switch (g.kind) {
    case CIRCLE:
    case SPHERE: {
      double dx = x - g.centre[0], dy = y - g.centre[1];
      double dz = g.kind == SPHERE ? z - g.centre[2] : 0.0;
      double rho = __dsqrt_rn(__dadd_rn(__dadd_rn(sq(dx), sq(dy)), sq(dz)));
      if (rho == 0.0) return false;
      dist = fabs(g.radii[0] - rho);
      const double ir = 1.0 / rho;
      n[0] = dx * ir; n[1] = dy * ir; n[2] = dz * ir;
      break;
    }
    case ELLIPSE:
    case AIRFOIL4: {
      double px, py, bx, by;
      to_body2(g, x, y, px, py);
      if (g.kind == ELLIPSE) ellipse_closest(g.radii[0], g.radii[1], px, py, dist, bx, by);
      else airfoil_closest(g.t, g.c, px, py, solid, dist, bx, by);
      n[0] = g.rot[0] * bx + g.rot[1] * by;
      n[1] = g.rot[3] * bx + g.rot[4] * by;
      break;
    }
  }
  psi = solid ? dist : -dist;
  return true;
}

// Eq. delta_n with the widths of the cell (i, j, k).
__device__ inline double delta_n(const Geom& g, const double n[3], int i, int j, int k) {
  const int ijk[3] = {i, j, k};
  double s = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.dim) continue;
    double q = n[a] / width_of(g, a, ijk[a]);
    s += q * q;
  }
  return 1.0 / sqrt(s);
}

// status word: keep the first error
__device__ inline void set_status(int* status, int code) {
  atomicCAS(status, 0, code);
}

}  // namespace ebr
