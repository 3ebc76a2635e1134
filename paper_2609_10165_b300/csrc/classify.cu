// Cell classification and ghost placement (Sec. 3.1, Sec. 7).
//
// Every body is convex, so the solid cells of one grid row (cells along x
// with fixed j, k) form one run [s, t].  A warp owns 32 consecutive rows: each
// lane estimates the run of its row in closed form (circle, sphere, ellipse)
// or by float bracketing (airfoil), confirms both ends with the exact double
// predicate on a 4-cell window, and then the whole warp streams the row's
// tags (0 / 1) with 16-byte stores.  Cells whose tag can become +-2 are exactly
// the cells with a face neighbour on the other side of the boundary
// ("interface" cells); they follow from the runs of a row and its y / z
// neighbour rows, so they are enumerated per row already sorted by linear
// index, without re-reading the tag array.
#include "ebr_kernels.cuh"
#include "lookback.cuh"

namespace ebr {

enum { ROW_EMPTY = 0, ROW_RUN = 1, ROW_TANGENT = 2 };

__device__ inline int iceil_idx(double f) { return (int)ceil(f); }
__device__ inline int ifloor_idx(double f) { return (int)floor(f); }

// fractional cell coordinate of world position x along axis a: cell i has f = i
__device__ inline double frac_cell(const Geom& g, int a, double x) {
  return (x - g.lo[a]) / g.h[a] - 0.5;
}

__device__ inline float airfoil_f32(float t, float c, float r00, float r01, float bx, float by,
                                    float x) {
  // depth y_t(x') - |y'| along a row, x' = r00 x + bx, y' = r01 x + by
  float xp = r00 * x + bx;
  float yp = r01 * x + by;
  float xi = fminf(fmaxf(xp / c, 0.0f), 1.0f);
  float yt = 5.0f * t * c * (0.2969f * sqrtf(xi) + xi * (-0.1260f + xi * (-0.3516f + xi * (0.2843f + xi * -0.1015f))));
  return yt - fabsf(yp);
}

// Per-row constants of the float pre-test of the inside predicate.
struct RowF {
  float ox, hx;        // x - c_x = ox + (i + 1/2) hx (body-relative x of cell i)
  float c0, c1, c2;    // row-constant parts (y / z terms)
  float m;             // safety margin of the float test
  float ia, ib;        // ellipse 1/a, 1/b
  float r00, r01;      // rotation entries multiplying x
};

// Float test of one cell of the row: 1 solid, 0 fluid, -1 too close to call.
// The margins bound the float rounding of every quantity by a wide factor;
// a cell within the margin of the boundary is decided by the double predicate.
__device__ inline int solid_f32(const Geom& g, const RowF& R, int i) {
  float x = g.stretched ? g.fcen[0][i] - g.fcentre[0] : R.ox + ((float)i + 0.5f) * R.hx;
  switch (g.kind) {
    case CIRCLE:
    case SPHERE: {
      float v = x * x + R.c0 - R.c1;             // |d|^2 - r^2
      if (v > R.m) return 0;
      if (v < -R.m) return 1;
      return -1;
    }
    case ELLIPSE: {
      float px = (R.r00 * x + R.c0) * R.ia, py = (R.r01 * x + R.c1) * R.ib;
      float v = px * px + py * py - 1.0f;
      if (v > R.m) return 0;
      if (v < -R.m) return 1;
      return -1;
    }
    default: {  // AIRFOIL4: depth y_t(x') - |y'|, x' in [0, c]
      float px = R.r00 * x + R.c0, py = R.r01 * x + R.c1, c = (float)g.c;
      if (px < -R.m || px > c + R.m) return 0;
      if (px < 1e-3f * c || px > c - R.m) return -1;    // near the nose (sqrt) or the base
      float xi = px / c;
      float yt = 5.0f * (float)g.t * c *
                 (0.2969f * sqrtf(xi) + xi * (-0.1260f + xi * (-0.3516f + xi * (0.2843f + xi * -0.1015f))));
      float v = yt - fabsf(py);
      if (v > R.m) return 1;
      if (v < -R.m) return 0;
      return -1;
    }
  }
}

__device__ inline void row_consts(const Geom& g, int j, int k, RowF& R) {
  double y = centre_of(g, 1, j);
  double z = g.dim == 3 ? centre_of(g, 2, k) : 0.0;
  float ext = 1.0f;
  for (int a = 0; a < g.dim; ++a)
    ext = fmaxf(ext, fmaxf(fabsf((float)(g.lo[a] - g.centre[a])),
                           fabsf((float)(g.lo[a] + g.n[a] * g.h[a] - g.centre[a]))));
  R.ox = (float)(g.lo[0] - g.centre[0]);
  R.hx = (float)g.h[0];
  R.ia = R.ib = 1.0f;
  R.r00 = (float)g.rot[0];
  R.r01 = (float)g.rot[1];
  float dy = (float)(y - g.centre[1]);
  if (g.kind == CIRCLE || g.kind == SPHERE) {
    float dz = g.kind == SPHERE ? (float)(z - g.centre[2]) : 0.0f;
    float r = (float)g.radii[0];
    R.c0 = dy * dy + dz * dz;
    R.c1 = r * r;
    R.m = 1e-5f * (3.0f * ext * ext + r * r);
  } else if (g.kind == ELLIPSE) {
    float a = (float)g.radii[0], b = (float)g.radii[1];
    R.c0 = (float)g.rot[3] * dy;
    R.c1 = (float)g.rot[4] * dy;
    R.ia = 1.0f / a;
    R.ib = 1.0f / b;
    float mn = fminf(a, b);
    R.m = 1e-5f * (1.0f + 2.0f * ext * ext / (mn * mn));
  } else {
    R.c0 = (float)g.rot[3] * dy;
    R.c1 = (float)g.rot[4] * dy;
    R.m = 2e-5f * (1.0f + ext);
  }
}

// Estimate the solid run of row (j, k) in float.  A row is declared empty
// only with a wide margin; near-tangent rows are handed to the exact window.
__device__ void estimate_row(const Geom& g, int j, int k, int& state, int& ia, int& ib, int& iv) {
  const int n = g.n[0];
  float y = (float)(centre_of(g, 1, j) - g.centre[1]);
  float z = g.dim == 3 ? (float)(centre_of(g, 2, k) - g.centre[2]) : 0.0f;
  float lo0 = (float)(g.lo[0] - g.centre[0]), h0 = (float)g.h[0];
  auto frac = [&](float xr) { return (xr - lo0) / h0 - 0.5f; };   // body-relative x -> cell
  state = ROW_EMPTY; ia = 0; ib = -1; iv = 0;
  float cx, xa, xb;
  if (g.kind == CIRCLE || g.kind == SPHERE) {
    float r2 = (float)(g.radii[0] * g.radii[0]);
    float yz = y * y + (g.kind == SPHERE ? z * z : 0.0f);
    float D = r2 - yz;
    cx = 0.0f;
    if (D < -(1e-4f * r2 + 1e-6f * yz)) return;
    if (D <= 0.0f) { state = ROW_TANGENT; iv = (int)lrintf(frac(cx)); return; }
    float sD = sqrtf(D);
    xa = -sD; xb = sD;
  } else if (g.kind == ELLIPSE) {
    float r00 = (float)g.rot[0], r01 = (float)g.rot[1], r10 = (float)g.rot[3], r11 = (float)g.rot[4];
    float ia2 = 1.0f / (float)(g.radii[0] * g.radii[0]), ib2 = 1.0f / (float)(g.radii[1] * g.radii[1]);
    float A = r00 * r00 * ia2 + r01 * r01 * ib2;
    float Bq = 2.0f * y * (r00 * r10 * ia2 + r01 * r11 * ib2);
    float C = y * y * (r10 * r10 * ia2 + r11 * r11 * ib2) - 1.0f;
    float disc = Bq * Bq - 4.0f * A * C;
    cx = -Bq / (2.0f * A);
    float scale = Bq * Bq + 4.0f * A * fabsf(C);
    if (disc < -1e-4f * scale) return;
    if (disc <= 0.0f) { state = ROW_TANGENT; iv = (int)lrintf(frac(cx)); return; }
    float sd = sqrtf(disc) / (2.0f * A);
    xa = cx - sd; xb = cx + sd;
  } else {  // AIRFOIL4: golden-section maximum of the concave depth, bisected roots
    float r00 = (float)g.rot[0], r01 = (float)g.rot[1];
    float bx = (float)g.rot[3] * y, byy = (float)g.rot[4] * y;
    float c = (float)g.c, t = (float)g.t;
    if (!(r00 > 0.0f)) { state = -1; return; }
    float X0 = (0.0f - bx) / r00, X1 = (c - bx) / r00;
    // quick reject: |y'| along the segment exceeds the maximum half thickness
    float ymin = fminf(fabsf(r01 * X0 + byy), fabsf(r01 * X1 + byy));
    if ((r01 * X0 + byy) * (r01 * X1 + byy) < 0.0f) ymin = 0.0f;
    if (ymin > 0.6f * t * c + 1e-4f * c) return;
    const float gr = 0.6180339887f;
    float lo = X0, hi = X1;
    float m1 = hi - gr * (hi - lo), m2 = lo + gr * (hi - lo);
    float f1 = airfoil_f32(t, c, r00, r01, bx, byy, m1), f2 = airfoil_f32(t, c, r00, r01, bx, byy, m2);
    for (int it = 0; it < 40; ++it) {
      if (f1 < f2) { lo = m1; m1 = m2; f1 = f2; m2 = lo + gr * (hi - lo); f2 = airfoil_f32(t, c, r00, r01, bx, byy, m2); }
      else { hi = m2; m2 = m1; f2 = f1; m1 = hi - gr * (hi - lo); f1 = airfoil_f32(t, c, r00, r01, bx, byy, m1); }
    }
    float xm = 0.5f * (lo + hi);
    float fm = airfoil_f32(t, c, r00, r01, bx, byy, xm);
    float tol = 1e-4f * c;
    cx = xm;
    if (fm < -tol) return;
    // a grazing row whose maximum depth rounds to <= 0 holds at most a few
    // cells around the maximum; any positive depth gets bracketed roots
    if (fm <= 0.0f) { state = ROW_TANGENT; iv = (int)lrintf(frac(cx)); return; }
    // roots of the depth on either side of the maximum; where the depth is
    // still >= 0 at the segment end the run ends there (x' = 0 or x' = c)
    float xa_f = X0, xb_f = X1;
    if (airfoil_f32(t, c, r00, r01, bx, byy, X0) < 0.0f) {
      float a = X0, b = xm;
      for (int it = 0; it < 28; ++it) {
        float m = 0.5f * (a + b);
        if (airfoil_f32(t, c, r00, r01, bx, byy, m) < 0.0f) a = m; else b = m;
      }
      xa_f = 0.5f * (a + b);
    }
    if (airfoil_f32(t, c, r00, r01, bx, byy, X1) < 0.0f) {
      float a = xm, b = X1;
      for (int it = 0; it < 28; ++it) {
        float m = 0.5f * (a + b);
        if (airfoil_f32(t, c, r00, r01, bx, byy, m) >= 0.0f) a = m; else b = m;
      }
      xb_f = 0.5f * (a + b);
    }
    xa = xa_f; xb = xb_f;
  }
  float fa = frac(xa), fb = frac(xb);
  if (fb < -2.0f || fa > n + 1.0f) return;
  ia = (int)ceilf(fmaxf(fa, -4.0f));
  ib = (int)floorf(fminf(fb, (float)n + 3.0f));
  if (ia > ib) { state = ROW_TANGENT; iv = (int)lrintf(frac(cx)); return; }
  state = ROW_RUN;
}

__device__ inline bool pred_cell(const Geom& g, const RowF& R, int i, int j, int k) {
  if (i < 0 || i >= g.n[0]) return false;
  int q = solid_f32(g, R, i);
  if (q >= 0) return q == 1;
  return solid_cell(g, i, j, k);
}

// exact run [s, t] of a row (s > t: empty); counts fallbacks in stats[0]
__device__ void exact_run(const Geom& g, int j, int k, int& s, int& t, int* status, int* stats) {
  const int n = g.n[0];
  int state, ia, ib, iv;
  estimate_row(g, j, k, state, ia, ib, iv);
  s = 0; t = -1;
  if (state < 0) { set_status(status, S_EINVAL); return; }
  if (state == ROW_EMPTY) return;
  RowF R;
  row_consts(g, j, k, R);
  bool ok = true;
  if (state == ROW_RUN) {
    unsigned bl = 0, bu = 0;
    for (int m = 0; m < 4; ++m) {
      if (pred_cell(g, R, ia - 2 + m, j, k)) bl |= 1u << m;
      if (pred_cell(g, R, ib - 1 + m, j, k)) bu |= 1u << m;
    }
    if (bl == 0 || bu == 0) ok = false;
    else {
      int m0 = __ffs(bl) - 1, m1 = 31 - __clz(bu);
      s = ia - 2 + m0;
      t = ib - 1 + m1;
      if (m0 == 0 && s > 0) ok = false;
      if (m1 == 3 && t < n - 1) ok = false;
      if (s > t) ok = false;
    }
  } else {  // tangent: a short run (or none) around the vertex
    unsigned bw = 0;
    for (int m = 0; m < 8; ++m)
      if (pred_cell(g, R, iv - 3 + m, j, k)) bw |= 1u << m;
    if (bw == 0) { s = 0; t = -1; return; }
    int m0 = __ffs(bw) - 1, m1 = 31 - __clz(bw);
    s = iv - 3 + m0;
    t = iv - 3 + m1;
    if ((m0 == 0 && s > 0) || (m1 == 7 && t < n - 1)) ok = false;
    unsigned run = bw >> m0;
    if ((run & (run + 1)) != 0) ok = false;     // not contiguous
  }
  if (!ok) {
    atomicAdd(&stats[0], 1);
    // fallback 1: a solid seed inside the estimated run; the run is an
    // interval (convex body), so bisect the exact predicate for both ends
    int seed = state == ROW_RUN ? (ia + ib) / 2 : iv;
    if (seed >= 0 && seed < n && solid_cell(g, seed, j, k)) {
      int lo = -1, hi = seed;            // pred(lo) false (virtual), pred(hi) true
      while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (solid_cell(g, mid, j, k)) hi = mid; else lo = mid;
      }
      s = hi;
      lo = seed; hi = n;                 // pred(lo) true, pred(hi) false (virtual)
      while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (solid_cell(g, mid, j, k)) lo = mid; else hi = mid;
      }
      t = lo;
    } else {
      // fallback 2: sweep the whole row with the exact predicate
      s = 0; t = -1;
      bool any = false;
      for (int i = 0; i < n; ++i) {
        if (solid_cell(g, i, j, k)) {
          if (!any) { s = i; any = true; }
          t = i;
        }
      }
      if (!any) { s = 0; t = -1; }
    }
  }
}

// ---------------------------------------------------------------------------
// rows, RG = 8 lanes per row (4 rows per warp).  The search for the run is
// parallel inside the group: 8 samples per round instead of one lane walking
// dozens of dependent iterations, so that many more rows are in flight.
// Every shuffle and ballot names the group's lanes only, and control flow is
// uniform inside a group (all its lanes hold the same row).
// ---------------------------------------------------------------------------
constexpr int RG = 8;

struct RowGrp {
  unsigned mask;   // the group's lanes
  int sl;          // lane within the group
  int shift;       // first lane of the group
  __device__ __forceinline__ unsigned ballot(bool p) const {
    return (__ballot_sync(mask, p) >> shift) & 0xFFu;
  }
  // group arg-max; ties go to the smaller index (all lanes get the result)
  __device__ __forceinline__ int arg_max(float v) const {
    int a = sl;
    for (int o = 1; o < RG; o <<= 1) {
      const float ov = __shfl_xor_sync(mask, v, o, RG);
      const int oa = __shfl_xor_sync(mask, a, o, RG);
      if (ov > v || (ov == v && oa < a)) { v = ov; a = oa; }
    }
    return a;
  }
  __device__ __forceinline__ int min_i(int v) const {
    for (int o = 1; o < RG; o <<= 1) v = min(v, __shfl_xor_sync(mask, v, o, RG));
    return v;
  }
  __device__ __forceinline__ int max_i(int v) const {
    for (int o = 1; o < RG; o <<= 1) v = max(v, __shfl_xor_sync(mask, v, o, RG));
    return v;
  }
};

// float row constants from the float copies of the geometry (the margins of
// solid_f32 cover the float rounding of the cell centres by a wide factor)
__device__ inline void row_consts_f(const Geom& g, int j, int k, RowF& R) {
  const float dy = fcentre_of(g, 1, j) - g.fcentre[1];
  const float dz = g.dim == 3 ? fcentre_of(g, 2, k) - g.fcentre[2] : 0.0f;
  const float ext = g.fext;
  R.ox = g.flo[0] - g.fcentre[0];
  R.hx = g.fh[0];
  R.ia = R.ib = 1.0f;
  R.r00 = g.frot[0];
  R.r01 = g.frot[1];
  if (g.kind == CIRCLE || g.kind == SPHERE) {
    const float r = g.fradii[0];
    R.c0 = dy * dy + (g.kind == SPHERE ? dz * dz : 0.0f);
    R.c1 = r * r;
    R.m = 1e-5f * (3.0f * ext * ext + r * r);
  } else if (g.kind == ELLIPSE) {
    const float a = g.fradii[0], b = g.fradii[1];
    R.c0 = g.frot[3] * dy;
    R.c1 = g.frot[4] * dy;
    R.ia = 1.0f / a;
    R.ib = 1.0f / b;
    const float mn = fminf(a, b);
    R.m = 1e-5f * (1.0f + 2.0f * ext * ext / (mn * mn));
  } else {
    R.c0 = g.frot[3] * dy;
    R.c1 = g.frot[4] * dy;
    R.m = 2e-5f * (1.0f + ext);
  }
}

// Estimate of the solid run of row (j, k) by the group (same result in every
// lane); same states as estimate_row.
__device__ void estimate_row_grp(const Geom& g, int j, int k, const RowGrp& Gp, int& state, int& ia,
                                 int& ib, int& iv) {
  const int n = g.n[0];
  const float y = fcentre_of(g, 1, j) - g.fcentre[1];
  const float z = g.dim == 3 ? fcentre_of(g, 2, k) - g.fcentre[2] : 0.0f;
  const float lo0 = g.flo[0] - g.fcentre[0], h0 = g.fh[0];
  // body-relative x -> fractional cell index (cell i has its centre at i);
  // on a stretched grid by bisection over the float centres, linear between
  // neighbouring centres (beyond the end centres: half widths of the end cells)
  auto frac = [&](float xr) {
    if (!g.stretched) return (xr - lo0) / h0 - 0.5f;
    const float x = xr + g.fcentre[0];
    const float* c = g.fcen[0];
    if (x <= c[0]) return (x - c[0]) / (float)g.wid[0][0];
    if (x >= c[n - 1]) return (float)(n - 1) + (x - c[n - 1]) / (float)g.wid[0][n - 1];
    int lo = 0, hi = n - 1;            // c[lo] <= x < c[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (c[mid] <= x) lo = mid; else hi = mid;
    }
    return (float)lo + (x - c[lo]) / (c[hi] - c[lo]);
  };
  state = ROW_EMPTY; ia = 0; ib = -1; iv = 0;
  float cx, xa, xb;
  if (g.kind == CIRCLE || g.kind == SPHERE) {
    const float r2 = g.fradii[0] * g.fradii[0];
    const float yz = y * y + (g.kind == SPHERE ? z * z : 0.0f);
    const float D = r2 - yz;
    cx = 0.0f;
    if (D < -(1e-4f * r2 + 1e-6f * yz)) return;
    if (D <= 0.0f) { state = ROW_TANGENT; iv = (int)lrintf(frac(cx)); return; }
    const float sD = sqrtf(D);
    xa = -sD; xb = sD;
  } else if (g.kind == ELLIPSE) {
    const float r00 = g.frot[0], r01 = g.frot[1], r10 = g.frot[3], r11 = g.frot[4];
    const float ia2 = 1.0f / (g.fradii[0] * g.fradii[0]), ib2 = 1.0f / (g.fradii[1] * g.fradii[1]);
    const float A = r00 * r00 * ia2 + r01 * r01 * ib2;
    const float Bq = 2.0f * y * (r00 * r10 * ia2 + r01 * r11 * ib2);
    const float C = y * y * (r10 * r10 * ia2 + r11 * r11 * ib2) - 1.0f;
    const float disc = Bq * Bq - 4.0f * A * C;
    cx = -Bq / (2.0f * A);
    const float scale = Bq * Bq + 4.0f * A * fabsf(C);
    if (disc < -1e-4f * scale) return;
    if (disc <= 0.0f) { state = ROW_TANGENT; iv = (int)lrintf(frac(cx)); return; }
    const float sd = sqrtf(disc) / (2.0f * A);
    xa = cx - sd; xb = cx + sd;
  } else {  // AIRFOIL4: maximum of the concave depth, then the two roots
    const float r00 = g.frot[0], r01 = g.frot[1];
    const float bx = g.frot[3] * y, byy = g.frot[4] * y;
    const float c = g.fc, t = g.ft;
    if (!(r00 > 0.0f)) { state = -1; return; }
    const float X0 = (0.0f - bx) / r00, X1 = (c - bx) / r00;
    // quick reject: |y'| along the segment exceeds the maximum half thickness
    float ymin = fminf(fabsf(r01 * X0 + byy), fabsf(r01 * X1 + byy));
    if ((r01 * X0 + byy) * (r01 * X1 + byy) < 0.0f) ymin = 0.0f;
    if (ymin > 0.6f * t * c + 1e-4f * c) return;
    // maximum: 8 samples per round; for a concave depth the maximum lies
    // within one spacing of the best sample, so the bracket shrinks 4x
    float lo = X0, hi = X1;
    for (int r = 0; r < 8; ++r) {
      const float w = (hi - lo) * (1.0f / RG);
      const int bi = Gp.arg_max(airfoil_f32(t, c, r00, r01, bx, byy, lo + ((float)Gp.sl + 0.5f) * w));
      const float xbest = lo + ((float)bi + 0.5f) * w;
      lo = fmaxf(X0, xbest - w);
      hi = fminf(X1, xbest + w);
    }
    const float xm = 0.5f * (lo + hi);
    const float fm = airfoil_f32(t, c, r00, r01, bx, byy, xm);
    const float tol = 1e-4f * c;
    cx = xm;
    if (fm < -tol) return;
    // a grazing row whose maximum depth rounds to <= 0 holds at most a few
    // cells around the maximum; any positive depth gets bracketed roots
    if (fm <= 0.0f) { state = ROW_TANGENT; iv = (int)lrintf(frac(cx)); return; }
    // roots on either side of the maximum (8-way refinement, depth monotone
    // there); where the depth is still >= 0 at the segment end the run ends
    // there (x' = 0 or x' = c)
    float xa_f = X0, xb_f = X1;
    if (airfoil_f32(t, c, r00, r01, bx, byy, X0) < 0.0f) {
      float a = X0, b = xm;                        // depth(a) < 0 <= depth(b)
      for (int r = 0; r < 6; ++r) {
        const float w = (b - a) * (1.0f / RG);
        const float xs = a + ((float)Gp.sl + 1.0f) * w;
        const unsigned pos = Gp.ballot(Gp.sl == RG - 1 || airfoil_f32(t, c, r00, r01, bx, byy, xs) >= 0.0f);
        const int i0 = __ffs(pos) - 1;
        b = a + (float)(i0 + 1) * w;
        a = a + (float)i0 * w;
      }
      xa_f = 0.5f * (a + b);
    }
    if (airfoil_f32(t, c, r00, r01, bx, byy, X1) < 0.0f) {
      float a = xm, b = X1;                        // depth(a) >= 0 > depth(b)
      for (int r = 0; r < 6; ++r) {
        const float w = (b - a) * (1.0f / RG);
        const float xs = a + ((float)Gp.sl + 1.0f) * w;
        const unsigned neg = Gp.ballot(Gp.sl == RG - 1 || airfoil_f32(t, c, r00, r01, bx, byy, xs) < 0.0f);
        const int i0 = __ffs(neg) - 1;
        b = a + (float)(i0 + 1) * w;
        a = a + (float)i0 * w;
      }
      xb_f = 0.5f * (a + b);
    }
    xa = xa_f; xb = xb_f;
  }
  const float fa = frac(xa), fb = frac(xb);
  if (fb < -2.0f || fa > n + 1.0f) return;
  ia = (int)ceilf(fmaxf(fa, -4.0f));
  ib = (int)floorf(fminf(fb, (float)n + 3.0f));
  if (ia > ib) { state = ROW_TANGENT; iv = (int)lrintf(frac(cx)); return; }
  state = ROW_RUN;
}

// exact run [s, t] of a row by the group: windows of the estimate confirmed
// with the exact predicate (one cell per lane), exact 8-way search or sweep
// as the fallback; counts fallbacks in stats[0]
__device__ void exact_run_grp(const Geom& g, int j, int k, const RowGrp& Gp, int& s, int& t,
                              int* status, int* stats) {
  const int n = g.n[0];
  int state, ia, ib, iv;
  estimate_row_grp(g, j, k, Gp, state, ia, ib, iv);
  s = 0; t = -1;
  if (state < 0) { if (Gp.sl == 0) set_status(status, S_EINVAL); return; }
  if (state == ROW_EMPTY) return;
  RowF R;
  row_consts_f(g, j, k, R);
  bool ok = true;
  if (state == ROW_RUN) {
    const int cell = Gp.sl < 4 ? ia - 2 + Gp.sl : ib - 1 + (Gp.sl - 4);
    const unsigned w = Gp.ballot(pred_cell(g, R, cell, j, k));
    const unsigned bl = w & 0xFu, bu = w >> 4;
    if (bl == 0 || bu == 0) ok = false;
    else {
      const int m0 = __ffs(bl) - 1, m1 = 31 - __clz(bu);
      s = ia - 2 + m0;
      t = ib - 1 + m1;
      if (m0 == 0 && s > 0) ok = false;
      if (m1 == 3 && t < n - 1) ok = false;
      if (s > t) ok = false;
    }
  } else {  // tangent: a short run (or none) around the vertex
    const unsigned bw = Gp.ballot(pred_cell(g, R, iv - 3 + Gp.sl, j, k));
    if (bw == 0) { s = 0; t = -1; return; }
    const int m0 = __ffs(bw) - 1, m1 = 31 - __clz(bw);
    s = iv - 3 + m0;
    t = iv - 3 + m1;
    if ((m0 == 0 && s > 0) || (m1 == 7 && t < n - 1)) ok = false;
    const unsigned run = bw >> m0;
    if ((run & (run + 1)) != 0) ok = false;     // not contiguous
  }
  if (ok) return;
  if (Gp.sl == 0) atomicAdd(&stats[0], 1);
  // fallback 1: a solid seed inside the estimated run; the run is an
  // interval (convex body), so search both ends with the exact predicate
  const int seed = state == ROW_RUN ? (ia + ib) / 2 : iv;
  if (seed >= 0 && seed < n && solid_cell(g, seed, j, k)) {
    int lo = -1, hi = seed;              // pred(lo) false (virtual), pred(hi) true
    while (hi - lo > 1) {
      const int step = (hi - lo + RG - 1) / RG;
      const int x = min(lo + (Gp.sl + 1) * step, hi);
      const unsigned p = Gp.ballot(x >= hi || solid_cell(g, x, j, k));
      const int i0 = __ffs(p) - 1;
      hi = min(lo + (i0 + 1) * step, hi);
      lo = lo + i0 * step;
    }
    s = hi;
    lo = seed; hi = n;                   // pred(lo) true, pred(hi) false (virtual)
    while (hi - lo > 1) {
      const int step = (hi - lo + RG - 1) / RG;
      const int x = min(lo + (Gp.sl + 1) * step, hi);
      const unsigned p = Gp.ballot(x >= hi || !solid_cell(g, x, j, k));
      const int i0 = __ffs(p) - 1;
      hi = min(lo + (i0 + 1) * step, hi);
      lo = lo + i0 * step;
    }
    t = lo;
  } else {
    // fallback 2: sweep the whole row with the exact predicate
    int mn = n, mx = -1;
    for (int i = Gp.sl; i < n; i += RG)
      if (solid_cell(g, i, j, k)) { mn = min(mn, i); mx = max(mx, i); }
    mn = Gp.min_i(mn);
    mx = Gp.max_i(mx);
    if (mx < 0) { s = 0; t = -1; } else { s = mn; t = mx; }
  }
}

__global__ void __launch_bounds__(256, 5) k_rows(const Geom* __restrict__ G, const int* __restrict__ row_off,
                                              int B, int total_rows, int2* __restrict__ runs,
                                              int8_t* __restrict__ tags, int* status, int* stats) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  // rows interleaved across blocks: an airfoil's chord band searches for
  // longer than other rows
  const int row = interleaved_item() / RG;
  if (row >= total_rows) return;                 // the whole group leaves together
  RowGrp Gp;
  Gp.sl = lane & (RG - 1);
  Gp.shift = lane & ~(RG - 1);
  Gp.mask = 0xFFu << Gp.shift;
  const int b = find_seg(row_off, B, row);
  const Geom& g = G[b];
  const int local = row - g.row_off;
  const int j = local % g.n[1];
  const int k = local / g.n[1];
  int s, t;
  exact_run_grp(g, j, k, Gp, s, t, status, stats);
  if (Gp.sl == 0) runs[row] = make_int2(s, t);
  // the group streams the tags of its row
  const int nx = g.n[0];
  const long long rst = g.cell_off + (long long)local * nx, end = rst + nx;
  // 16-byte alignment of the actual addresses (the caller's buffer may be offset)
  const long long mis = (long long)(reinterpret_cast<uintptr_t>(tags) & 15u);
  long long a0 = ((rst + mis + 15) & ~15LL) - mis;
  long long a1 = ((end + mis) & ~15LL) - mis;
  if (a0 > end) a0 = end;
  if (a1 < a0) a1 = a0;
  for (long long q = rst + Gp.sl; q < a0; q += RG) {
    const long long i = q - rst;
    tags[q] = (int8_t)(i >= s && i <= t);
  }
  for (long long q = a1 + Gp.sl; q < end; q += RG) {
    const long long i = q - rst;
    tags[q] = (int8_t)(i >= s && i <= t);
  }
  // aligned middle: 16-byte chunks, chunk c holding cells [ia0 + 16 c,
  // ia0 + 16 c + 15] (offsets from the row start in 32-bit).  Chunks [0, zb)
  // lie before the run, [ib0, ib1) inside it, [za, nch) after it: constant
  // words in tight store loops, lane sl taking the chunks c = sl (mod RG).
  // Only the (at most two) chunks of [zb, ib0) and [ib1, za) hold an end of
  // the run and build their bytes: bytes [lo, hi) lie inside, each 32-bit word
  // a difference of two prefix masks of 0x01 bytes.
  int8_t* const rowp = tags + rst;
  const int ia0 = (int)(a0 - rst), ia1 = (int)(a1 - rst);
  const int nch = (ia1 - ia0) >> 4;
  int zb = nch, ib0 = nch, ib1 = nch, za = nch;
  if (s <= t) {
    zb = min(max((s - ia0) >> 4, 0), nch);
    ib0 = min(max((s - ia0 + 15) >> 4, 0), nch);
    ib1 = max(min(max((t + 1 - ia0) >> 4, 0), nch), ib0);
    za = min(max(((t - ia0) >> 4) + 1, 0), nch);
  }
  const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
  const uint4 one4 = make_uint4(0x01010101u, 0x01010101u, 0x01010101u, 0x01010101u);
  uint4* const chunk = reinterpret_cast<uint4*>(rowp + ia0);
  // first chunk index >= c0 that belongs to this lane
  auto first = [&](int c0) { return c0 + ((Gp.sl - c0) & (RG - 1)); };
  for (int c = first(0); c < zb; c += RG) chunk[c] = zero4;
  for (int c = first(ib0); c < ib1; c += RG) chunk[c] = one4;
  for (int c = first(za); c < nch; c += RG) chunk[c] = zero4;
  auto edge = [&](int c) {
    const int i0 = ia0 + 16 * c;
    const int lo = min(max(s - i0, 0), 16);
    const int hi = min(max(t + 1 - i0, 0), 16);
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int l = min(max(lo - 4 * q, 0), 4), h = min(max(hi - 4 * q, 0), 4);
      const uint32_t ph = h ? (0x01010101u >> (8 * (4 - h))) : 0u;
      const uint32_t pl = l ? (0x01010101u >> (8 * (4 - l))) : 0u;
      w[q] = h > l ? (ph & ~pl) : 0u;
    }
    chunk[c] = make_uint4(w[0], w[1], w[2], w[3]);
  };
  for (int c = first(zb); c < ib0; c += RG) edge(c);
  for (int c = first(ib1); c < za; c += RG) edge(c);
}

void launch_rows(const Geom* G, const int* row_off, int B, int total_rows, int2* runs,
                 int8_t* tags, int* status, int* stats, cudaStream_t s) {
  if (total_rows <= 0) return;
  const long long threads = (long long)total_rows * RG;
  launch(k_rows, (unsigned)((threads + 255) / 256), 256, 0, s, G, row_off, B, total_rows, runs, tags, status, stats);
}

// ---------------------------------------------------------------------------
// interface cells of a row from the runs of the row and its neighbour rows
// ---------------------------------------------------------------------------
struct Iv { int a, b; };

__device__ inline void add_iv(Iv* v, int& m, int a, int b, int n) {
  a = max(a, 0);
  b = min(b, n - 1);
  if (a <= b) { v[m].a = a; v[m].b = b; ++m; }
}

// R \ Q for runs (s > t empty)
__device__ inline void add_diff(Iv* v, int& m, int2 R, int2 Q, int n) {
  if (R.x > R.y) return;
  if (Q.x > Q.y) { add_iv(v, m, R.x, R.y, n); return; }
  add_iv(v, m, R.x, min(R.y, Q.x - 1), n);
  add_iv(v, m, max(R.x, Q.y + 1), R.y, n);
}

// interface intervals of one row (sorted, merged: v[0..w)), its run and the
// band limits of the second layer
struct RowIface {
  Iv v[24];
  int w;
  int2 R;
  int bandA, bandB, bandC, bandD;
  int j, k, ny, nz, n;
  // the usual row (non-empty run, every in-grid face-neighbour run non-empty
  // and overlapping it, one layer): the intervals are the cells around the
  // run's first cell and those around its last cell, two intervals (f0, f1),
  // merged when they touch; v is not used then
  bool fast;
  Iv f0, f1;
};

__device__ inline void row_iface(const Geom& g, int local, const int2* __restrict__ runs, RowIface& I) {
  const int ny = g.n[1], nz = g.dim == 3 ? g.n[2] : 1, n = g.n[0];
  const int j = local % ny, k = local / ny;
  I.j = j; I.k = k; I.ny = ny; I.nz = nz; I.n = n;
  const int2 R = runs[g.row_off + local];
  I.R = R;
  const int dj[4] = {-1, 1, 0, 0}, dk[4] = {0, 0, -1, 1};
  int2 Qn[4];
  bool qin[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int jj = j + dj[q], kk = k + dk[q];
    qin[q] = !(jj < 0 || jj >= ny || kk < 0 || kk >= nz);
    Qn[q] = qin[q] ? runs[g.row_off + jj + ny * kk] : make_int2(1, 0);
  }
  bool fast = g.layers != 2 && R.x <= R.y;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (qin[q] && !(Qn[q].x <= Qn[q].y && Qn[q].x <= R.y && Qn[q].y >= R.x)) fast = false;
  I.fast = fast;
  I.bandA = 1; I.bandB = 0; I.bandC = 1; I.bandD = 0;
  if (fast) {
    // every piece of R \ Q and Q \ R touches R.x - 1 / R.x or R.y / R.y + 1,
    // as do the cells across the run's ends: their unions are one interval
    // each side
    constexpr int INF = 1 << 30;
    int llo = INF, lhi = -INF, rlo = INF, rhi = -INF;
    if (R.x > 0) { llo = R.x - 1; lhi = R.x; }
    if (R.y < n - 1) { rlo = R.y; rhi = R.y + 1; }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!qin[q]) continue;
      const int2 Q = Qn[q];
      if (Q.x < R.x) { llo = min(llo, Q.x); lhi = max(lhi, R.x - 1); }
      else if (Q.x > R.x) { llo = min(llo, R.x); lhi = max(lhi, Q.x - 1); }
      if (Q.y < R.y) { rlo = min(rlo, Q.y + 1); rhi = max(rhi, R.y); }
      else if (Q.y > R.y) { rlo = min(rlo, R.y + 1); rhi = max(rhi, Q.y); }
    }
    llo = max(llo, 0); lhi = min(lhi, n - 1);
    rlo = max(rlo, 0); rhi = min(rhi, n - 1);
    I.f0.a = llo; I.f0.b = lhi;
    I.f1.a = rlo; I.f1.b = rhi;
    if (llo <= lhi && rlo <= rhi && rlo <= lhi + 1) {   // they touch: one interval
      I.f0.b = max(lhi, rhi);
      I.f1.a = 1; I.f1.b = 0;
    } else if (llo > lhi) {                             // only the right one
      I.f0 = I.f1;
      I.f1.a = 1; I.f1.b = 0;
    }
    I.w = 0;
    return;
  }
  Iv* v = I.v;
  int m = 0;
  if (R.x <= R.y) {
    if (R.x > 0) { add_iv(v, m, R.x, R.x, n); add_iv(v, m, R.x - 1, R.x - 1, n); }
    if (R.y < n - 1) { add_iv(v, m, R.y, R.y, n); add_iv(v, m, R.y + 1, R.y + 1, n); }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (!qin[q]) continue;
    add_diff(v, m, R, Qn[q], n);
    add_diff(v, m, Qn[q], R, n);
  }
  // second ghost layer: the solid cells of the row with a fluid cell within
  // the box reach (the run minus its erosion by the box: a cell stays out
  // only when every in-grid row of the box has a run covering it with the
  // reach to spare, a run end at the grid edge counting as covered), listed
  // as band cells (flag 2)
  if (g.layers == 2 && R.x <= R.y) {
    int elo = 0, ehi = n - 1;
    const int ry = g.reach[1], rz = g.dim == 3 ? g.reach[2] : 0, rx = g.reach[0];
    for (int dk2 = -rz; dk2 <= rz && elo <= ehi; ++dk2)
      for (int dj2 = -ry; dj2 <= ry && elo <= ehi; ++dj2) {
        const int jj = j + dj2, kk = k + dk2;
        if (jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
        const int2 Q = (dj2 == 0 && dk2 == 0) ? R : runs[g.row_off + jj + ny * kk];
        if (Q.x > Q.y) { elo = 1; ehi = 0; break; }
        elo = max(elo, Q.x == 0 ? 0 : Q.x + rx);
        ehi = min(ehi, Q.y == n - 1 ? n - 1 : Q.y - rx);
      }
    if (elo > ehi) { I.bandA = R.x; I.bandB = R.y; }
    else {
      I.bandA = R.x; I.bandB = min(R.y, elo - 1);
      I.bandC = max(R.x, ehi + 1); I.bandD = R.y;
    }
    add_iv(v, m, I.bandA, I.bandB, n);
    add_iv(v, m, I.bandC, I.bandD, n);
  }
  // sort by start, merge
  for (int x = 1; x < m; ++x) {
    Iv key = v[x];
    int y = x - 1;
    while (y >= 0 && v[y].a > key.a) { v[y + 1] = v[y]; --y; }
    v[y + 1] = key;
  }
  int w = 0;
  for (int x = 0; x < m; ++x) {
    if (w > 0 && v[x].a <= v[w - 1].b + 1) v[w - 1].b = max(v[w - 1].b, v[x].b);
    else v[w++] = v[x];
  }
  I.w = w;
}

__device__ inline int row_iface_count(const RowIface& I) {
  if (I.fast) return max(I.f0.b - I.f0.a + 1, 0) + max(I.f1.b - I.f1.a + 1, 0);
  int cnt = 0;
  for (int x = 0; x < I.w; ++x) cnt += I.v[x].b - I.v[x].a + 1;
  return cnt;
}

// interface cells of the row from list position o: the run's ends and the
// cells across them, and the cells that differ from a face-neighbour row
// (the same sets as above); the rest of the list (second layer only) are band
// cells.  Returns false (status EBR_ESHAPE) when the list would pass cap.
__device__ inline bool row_iface_write(const Geom& g, int b, const int2* __restrict__ runs, const RowIface& I,
                                       int o, int cap, int* __restrict__ iface_cell, int* __restrict__ iface_geo,
                                       int8_t* __restrict__ iface_solid, int* status) {
  const int dj[4] = {-1, 1, 0, 0}, dk[4] = {0, 0, -1, 1};
  const int2 R = I.R;
  const int n = I.n, j = I.j, k = I.k, ny = I.ny, nz = I.nz;
  const int rowbase = n * (j + ny * k);
  if (I.fast) {
    // one layer: no band cells; the two intervals in order
    for (int x = 0; x < 2; ++x) {
      const Iv iv = x == 0 ? I.f0 : I.f1;
      for (int i = iv.a; i <= iv.b; ++i) {
        if (o >= cap) { set_status(status, S_ESHAPE); return false; }
        iface_cell[o] = rowbase + i;
        iface_geo[o] = b;
        iface_solid[o] = (int8_t)(i >= R.x && i <= R.y);
        ++o;
      }
    }
    return true;
  }
  for (int x = 0; x < I.w; ++x) {
    for (int i = I.v[x].a; i <= I.v[x].b; ++i) {
      if (o >= cap) { set_status(status, S_ESHAPE); return false; }
      const bool sol = i >= R.x && i <= R.y;
      int8_t flag = (int8_t)sol;
      if (g.layers == 2 && sol && ((i >= I.bandA && i <= I.bandB) || (i >= I.bandC && i <= I.bandD))) {
        // a band cell is an interface cell too when a face neighbour is fluid
        bool face = i == R.x && R.x > 0;
        face = face || (i == R.y && R.y < n - 1);
        for (int q = 0; q < 4 && !face; ++q) {
          const int jj = j + dj[q], kk = k + dk[q];
          if (jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
          const int2 Q = runs[g.row_off + jj + ny * kk];
          if (!(i >= Q.x && i <= Q.y)) face = true;
        }
        if (!face) flag = 2;
      }
      iface_cell[o] = rowbase + i;
      iface_geo[o] = b;
      iface_solid[o] = flag;
      ++o;
    }
  }
  return true;
}

__global__ void k_iface(const Geom* __restrict__ G, const int* __restrict__ row_off, int B,
                        int total_rows, const int2* __restrict__ runs, int* __restrict__ row_cnt,
                        const int* __restrict__ row_ptr, int* __restrict__ iface_cell,
                        int* __restrict__ iface_geo, int8_t* __restrict__ iface_solid, int write,
                        int cap, int* status) {
  pdl_enter();
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= total_rows) return;
  int b = find_seg(row_off, B, row);
  const Geom& g = G[b];
  RowIface I;
  row_iface(g, row - g.row_off, runs, I);
  if (!write) {
    row_cnt[row] = row_iface_count(I);
    return;
  }
  row_iface_write(g, b, runs, I, row_ptr[row], cap, iface_cell, iface_geo, iface_solid, status);
}

// One launch instead of count + scan + write: the rows' counts, their
// offsets by a single-pass scan in row order (the same offsets as the scan of
// the counts), then the cells.  row_ptr[total_rows] = total.
__global__ void k_iface_fused(const Geom* __restrict__ G, const int* __restrict__ row_off, int B,
                              int total_rows, const int2* __restrict__ runs, int* __restrict__ row_ptr,
                              int* __restrict__ iface_cell, int* __restrict__ iface_geo,
                              int8_t* __restrict__ iface_solid, int cap, const Lookback L, int* status) {
  pdl_enter();
  __shared__ int sh[32];
  const LbBlock blk = lb_begin(L);
  const int row = blk.tile * blockDim.x + threadIdx.x;
  const bool on = row < total_rows;
  int b = 0, cnt = 0;
  RowIface I;
  if (on) {
    b = find_seg(row_off, B, row);
    row_iface(G[b], row - G[b].row_off, runs, I);
    cnt = row_iface_count(I);
  }
  int agg;
  const int ex = block_excl_scan(cnt, sh, agg);
  const long long base = lb_prefix(L, blk, (unsigned)agg, status);
  if (base >= 0) {
    const int o = (int)(base + ex);
    if (on) {
      row_ptr[row] = o;
      // rows off the two-interval form write their own cells
      if (!I.fast)
        row_iface_write(G[b], b, runs, I, o, cap, iface_cell, iface_geo, iface_solid, status);
    }
    if (row == total_rows - 1) row_ptr[total_rows] = (int)(base + ex + cnt);
    // the warp writes the cells of its two-interval rows together: output
    // position t of the warp's flattened list belongs to the lane r with the
    // largest exclusive prefix <= t (a row of a few hundred cells no longer
    // holds its warp for as many serial stores); every lane takes part in
    // every shuffle
    const int lane = threadIdx.x & 31;
    const int cf = (on && I.fast) ? cnt : 0;
    int incl = cf;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    const int excl = incl - cf;
    const int wtot = __shfl_sync(0xffffffffu, incl, 31);
    const int len0 = (on && I.fast) ? max(I.f0.b - I.f0.a + 1, 0) : 0;
    const int a0 = (on && I.fast) ? I.f0.a : 0, a1 = (on && I.fast) ? I.f1.a : 0;
    const int rx = on ? I.R.x : 0, ry = on ? I.R.y : 0;
    const int rowbase = on ? I.n * (I.j + I.ny * I.k) : 0;
    for (int t0 = 0; t0 < wtot; t0 += 32) {
      const int t = t0 + lane;
      int r = 0;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        const int c = r + d;
        const int v = __shfl_sync(0xffffffffu, excl, c);
        if (v <= t) r = c;
      }
      const int ex_r = __shfl_sync(0xffffffffu, excl, r);
      const int o_r = __shfl_sync(0xffffffffu, o, r);
      const int l0 = __shfl_sync(0xffffffffu, len0, r);
      const int s0 = __shfl_sync(0xffffffffu, a0, r);
      const int s1 = __shfl_sync(0xffffffffu, a1, r);
      const int x0 = __shfl_sync(0xffffffffu, rx, r);
      const int x1 = __shfl_sync(0xffffffffu, ry, r);
      const int rb = __shfl_sync(0xffffffffu, rowbase, r);
      const int br = __shfl_sync(0xffffffffu, b, r);
      if (t < wtot) {
        const int pidx = t - ex_r;
        const int i = pidx < l0 ? s0 + pidx : s1 + (pidx - l0);
        const int q = o_r + pidx;
        if (q >= cap) {
          set_status(status, S_ESHAPE);
        } else {
          iface_cell[q] = rb + i;
          iface_geo[q] = br;
          iface_solid[q] = (int8_t)(i >= x0 && i <= x1);
        }
      }
    }
  }
  lb_end(L);
}

void launch_iface(const Geom* G, const int* row_off, int B, int total_rows, const int2* runs,
                  int* row_cnt, const int* row_ptr, int* iface_cell, int* iface_geo,
                  int8_t* iface_solid, int write, int iface_cap, int* status, cudaStream_t s, int T) {
  if (total_rows <= 0) return;
  launch(k_iface, (total_rows + T - 1) / T, T, 0, s, G, row_off, B, total_rows, runs, row_cnt,
         row_ptr, iface_cell, iface_geo, iface_solid, write, iface_cap, status);
}

void launch_iface_fused(const Geom* G, const int* row_off, int B, int total_rows, const int2* runs,
                        int* row_ptr, int* iface_cell, int* iface_geo, int8_t* iface_solid, int iface_cap,
                        const Lookback& L, int* status, cudaStream_t s) {
  if (total_rows <= 0) return;
  launch(k_iface_fused, (total_rows + LB_T - 1) / LB_T, LB_T, 0, s, G, row_off, B, total_rows, runs, row_ptr,
         iface_cell, iface_geo, iface_solid, iface_cap, L, status);
}

// ---------------------------------------------------------------------------
// placement: psi, n at interface cells; CGC / HGC candidate tags
// ---------------------------------------------------------------------------
__device__ inline void cell_ijk(const Geom& g, int cell, int& i, int& j, int& k) {
  i = cell % g.n[0];
  int r = cell / g.n[0];
  j = r % g.n[1];
  k = r / g.n[1];
}

// iface_meta (HGC only, may be null): for every candidate, the sign bits of
// its normal (bits 0..2, n_a < 0) and its zero components (bits 3..5, n_a ==
// 0), as the double closest point has them: from the float normal where it
// is well conditioned (no component within 1e-3 of zero, no near tie), else
// from the double closest point.
__global__ void __launch_bounds__(256, 5) k_place(const Geom* __restrict__ G, int n_iface, const int* __restrict__ iface_cell,
                        const int* __restrict__ iface_geo, const int8_t* __restrict__ iface_solid,
                        int placement, int8_t* __restrict__ tags, uint8_t* __restrict__ iface_meta,
                        int* status) {
  pdl_enter();
  const int m = interleaved_item();     // airfoil cells cost several times ellipse cells
  if (m >= n_iface) return;
  const Geom& g = G[iface_geo[m]];
  int cell = iface_cell[m];
  bool solid = iface_solid[m] != 0;
  int8_t tag = solid ? 1 : 0;
  if (iface_solid[m] == 2) {
    // a band cell of the second layer (solid, no fluid face neighbour): the
    // first layer leaves it solid; k_layer2 decides it after reclassification
    tags[g.cell_off + cell] = 1;
    return;
  }
  if (placement != HGC) {
    tag = solid ? 2 : 0;   // solid interface cell = solid cell with a fluid face neighbour
  } else {
    int i, j, k;
    cell_ijk(g, cell, i, j, k);
    // Eq. HGC_criterion decided in float where the float psi and dn/2 are
    // clearly apart; the few cells within the safety margin use double
    const float xf = fcentre_of(g, 0, i);
    const float yf = fcentre_of(g, 1, j);
    const float zf = g.dim == 3 ? fcentre_of(g, 2, k) : 0.0f;
    float n32[3];
    bool unsure = false;
    float psi32 = closest_point_f32(g, xf, yf, zf, solid, n32, iface_meta ? &unsure : nullptr);
    float s32 = 0.0f;
    const int ijk[3] = {i, j, k};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= g.dim) continue;
      float q = n32[a] / (g.stretched ? (float)g.wid[a][ijk[a]] : g.fh[a]);
      s32 += q * q;
    }
    float half32 = 0.5f / sqrtf(s32);
    float gap = fabsf(psi32) - half32;
    bool cand, dbl = false;
    double psi, nv[3];
    // the double closest point of the cell centre (false: normal undefined)
    auto exact = [&]() {
      double x = centre_of(g, 0, i), y = centre_of(g, 1, j);
      double z = g.dim == 3 ? centre_of(g, 2, k) : 0.0;
      dbl = closest_point(g, x, y, z, solid, psi, nv);
      return dbl;
    };
    if (fabsf(gap) > g.hgc_mrg) {
      cand = gap <= 0.0f;
    } else {
      if (!exact()) { set_status(status, S_EINVAL); return; }
      double half = 0.5 * delta_n(g, nv, i, j, k);
      cand = solid ? (psi <= half) : (-psi < half);
    }
    if (cand) {
      tag = solid ? 2 : -2;
      if (iface_meta) {
        if (unsure && !dbl && !exact()) { set_status(status, S_EINVAL); return; }
        uint32_t mb = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (a >= g.dim) continue;
          if (dbl ? nv[a] < 0.0 : n32[a] < 0.0f) mb |= 1u << a;
          if (dbl && nv[a] == 0.0) mb |= 8u << a;
        }
        iface_meta[m] = (uint8_t)mb;
      }
    }
  }
  tags[g.cell_off + cell] = tag;
}

void launch_place(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo,
                  const int8_t* iface_solid, int placement, int8_t* tags, uint8_t* iface_meta,
                  int* status, cudaStream_t s, int T) {
  if (n_iface <= 0) return;
  launch(k_place, (n_iface + T - 1) / T, T, 0, s, G, n_iface, iface_cell, iface_geo, iface_solid,
                                                placement, tags, iface_meta, status);
}

// HGC reclassification.  pass 0 (A): -2 without a tag-1 face neighbour -> 0.
// pass 1 (B): +2 without a tag-0 face neighbour -> 1.  In place is safe: pass A
// only turns -2 into 0 and tests for 1; pass B only turns +2 into 1 and tests
// for 0; pass B runs after pass A has completed.
// does cell `cell` of the grid have a face neighbour tagged `look`?
__device__ inline bool has_face_tag(const Geom& g, const int8_t* tg, int cell, int8_t look) {
  int i, j, k;
  cell_ijk(g, cell, i, j, k);
  const int ijk[3] = {i, j, k};
  const int stride[3] = {1, g.n[0], g.n[0] * g.n[1]};
  bool found = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.dim || found) continue;
    if (ijk[a] > 0 && tg[cell - stride[a]] == look) found = true;
    if (ijk[a] < g.n[a] - 1 && tg[cell + stride[a]] == look) found = true;
  }
  return found;
}

__global__ void k_reclassify(const Geom* __restrict__ G, int n_iface, const int* __restrict__ iface_cell,
                             const int* __restrict__ iface_geo, int8_t* __restrict__ tags, int pass) {
  pdl_enter();
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_iface) return;
  const Geom& g = G[iface_geo[m]];
  int cell = iface_cell[m];
  int8_t* tg = tags + g.cell_off;
  int8_t me = tg[cell];
  int8_t want_self = pass == 0 ? -2 : 2;
  if (me != want_self) return;
  if (!has_face_tag(g, tg, cell, pass == 0 ? 1 : 0)) tg[cell] = pass == 0 ? 0 : 1;
}

void launch_reclassify(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo,
                       int8_t* tags, int pass, cudaStream_t s) {
  if (n_iface <= 0) return;
  launch(k_reclassify, (n_iface + 127) / 128, 128, 0, s, G, n_iface, iface_cell, iface_geo, tags, pass);
}

// Second ghost layer (Sec. 7): after the first layer's placement and
// reclassification every listed cell still solid (tag 1) with psi <= 1.5 dn
// (Eq. delta_n with its own normal and widths) becomes a ghost (+2).  Decided
// in float where psi and 1.5 dn are clearly apart (three times the HGC
// margin), in double otherwise.
__global__ void k_layer2(const Geom* __restrict__ G, int n_iface, const int* __restrict__ iface_cell,
                         const int* __restrict__ iface_geo, int8_t* __restrict__ tags, int* status) {
  pdl_enter();
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_iface) return;
  const Geom& g = G[iface_geo[m]];
  if (g.layers != 2) return;
  const int cell = iface_cell[m];
  int8_t* t = tags + g.cell_off + cell;
  if (*t != 1) return;
  int i, j, k;
  cell_ijk(g, cell, i, j, k);
  if (g.kind == CIRCLE || g.kind == SPHERE) {
    // a candidate at the body's centre has depth R and no normal: it stays
    // solid when R > 1.5 max_a h_a (no dn admits it), else the second layer
    // is undefined there
    const double dx = centre_of(g, 0, i) - g.centre[0], dy = centre_of(g, 1, j) - g.centre[1];
    const double dz = g.dim == 3 ? centre_of(g, 2, k) - g.centre[2] : 0.0;
    if (dx == 0.0 && dy == 0.0 && dz == 0.0) {
      if (!(g.radii[0] > 1.5 * g.hmax)) set_status(status, S_EINVAL);
      return;
    }
  }
  const float xf = fcentre_of(g, 0, i);
  const float yf = fcentre_of(g, 1, j);
  const float zf = g.dim == 3 ? fcentre_of(g, 2, k) : 0.0f;
  float n32[3];
  const float psi32 = closest_point_f32(g, xf, yf, zf, true, n32);
  float s32 = 0.0f;
  const int ijk[3] = {i, j, k};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.dim) continue;
    const float q = n32[a] / (g.stretched ? (float)g.wid[a][ijk[a]] : g.fh[a]);
    s32 += q * q;
  }
  const float gap = fabsf(psi32) - 1.5f / sqrtf(s32);
  bool add;
  if (fabsf(gap) > 3.0f * g.hgc_mrg) {
    add = gap <= 0.0f;
  } else {
    const double x = centre_of(g, 0, i), y = centre_of(g, 1, j);
    const double z = g.dim == 3 ? centre_of(g, 2, k) : 0.0;
    double psi, nv[3];
    if (!closest_point(g, x, y, z, true, psi, nv)) { set_status(status, S_EINVAL); return; }
    add = psi <= 1.5 * delta_n(g, nv, i, j, k);
  }
  if (add) *t = 2;
}

void launch_layer2(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo, int8_t* tags,
                   int* status, cudaStream_t s) {
  if (n_iface <= 0) return;
  launch(k_layer2, (n_iface + 127) / 128, 128, 0, s, G, n_iface, iface_cell, iface_geo, tags, status);
}

__global__ void k_ghost_flags(const Geom* __restrict__ G, int n_iface, const int* __restrict__ iface_cell,
                              const int* __restrict__ iface_geo, const int8_t* __restrict__ tags,
                              int* __restrict__ flags) {
  pdl_enter();
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_iface) return;
  const Geom& g = G[iface_geo[m]];
  int8_t t = tags[g.cell_off + iface_cell[m]];
  flags[m] = (t == 2 || t == -2) ? 1 : 0;
}

void launch_ghost_flags(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo,
                        const int8_t* tags, int* flags, cudaStream_t s) {
  if (n_iface <= 0) return;
  launch(k_ghost_flags, (n_iface + 255) / 256, 256, 0, s, G, n_iface, iface_cell, iface_geo, tags, flags);
}

// compaction of the ghosts (index order): cell, geometry, fluid-side flag
__global__ void k_ghost_write(const Geom* __restrict__ G, int n_iface, const int* __restrict__ iface_cell,
                              const int* __restrict__ iface_geo, const int8_t* __restrict__ tags,
                              const int* __restrict__ gpos, int cap, int* __restrict__ gs_cell,
                              int* __restrict__ gs_geo, uint32_t* __restrict__ gs_meta, int* status) {
  pdl_enter();
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_iface) return;
  int b = iface_geo[m];
  const Geom& g = G[b];
  int cell = iface_cell[m];
  int8_t t = tags[g.cell_off + cell];
  if (t != 2 && t != -2) return;
  int s = gpos[m];
  if (s >= cap) { set_status(status, S_ESHAPE); return; }
  gs_cell[s] = cell;
  gs_geo[s] = b;
  gs_meta[s] = t == -2 ? (1u << 22) : 0u;
}

// Ghost compaction in one launch instead of flags + scan + write.  With
// pass_b (HGC, one layer) the cell's reclassification pass B comes first: +2
// without a tag-0 face neighbour becomes 1 (the test reads only 0s, which
// pass B neither makes nor removes, so the cells of the launch may run in any
// order).  Then the ghost flag (tag +-2) of every interface cell, the offsets
// by a single-pass scan in list order (the scan of the flags) and the ghost
// records (cell, geometry, fluid-side flag).  gpos[n_iface] = total.
// With iface_meta (one-layer HGC) the meta word of a ghost is complete here:
// normal signs and structurally active members from the placement's normal
// bytes, r = 1 on every axis; the closest points then only supply psi, S, n.
// After pass A, is a face neighbour of `cell` tagged 0?  From the tags of the
// placement: a neighbour tagged 0, or tagged -2 without a tag-1 face
// neighbour (which pass A turns into 0).
__device__ inline bool zero_after_pass_a(const Geom& g, const int8_t* tg, int cell) {
  int i, j, k;
  cell_ijk(g, cell, i, j, k);
  const int ijk[3] = {i, j, k};
  const int stride[3] = {1, g.n[0], g.n[0] * g.n[1]};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.dim) continue;
#pragma unroll
    for (int sd = -1; sd <= 1; sd += 2) {
      const int ia = ijk[a] + sd;
      if (ia < 0 || ia >= g.n[a]) continue;
      const int nb = cell + sd * stride[a];
      const int8_t v = tg[nb];
      if (v == 0 || (v == -2 && !has_face_tag(g, tg, nb, 1))) return true;
    }
  }
  return false;
}

// pass: 0 none, 1 reclassification pass B of each cell first (in place), 2
// passes A and B both, decided from the placement's tags (nothing written to
// the tag array; the final tag of every interface cell goes to iface_tag,
// for the position kernel to write).
__global__ void k_ghost_compact(const Geom* __restrict__ G, int n_iface, const int* __restrict__ iface_cell,
                                const int* __restrict__ iface_geo, int8_t* __restrict__ tags, int pass,
                                const uint8_t* __restrict__ iface_meta, int8_t* __restrict__ iface_tag,
                                int* __restrict__ gpos, int cap, int* __restrict__ gs_cell,
                                int* __restrict__ gs_geo, uint32_t* __restrict__ gs_meta, const Lookback L,
                                int* status) {
  pdl_enter();
  __shared__ int sh[32];
  const LbBlock blk = lb_begin(L);
  const int m = blk.tile * blockDim.x + threadIdx.x;
  const bool on = m < n_iface;
  int b = 0, cell = 0;
  int8_t t = 0;
  uint32_t mb = 0;
  if (on) {
    b = iface_geo[m];
    const Geom& g = G[b];
    cell = iface_cell[m];
    if (iface_meta) mb = iface_meta[m];     // loaded before the scan's waits
    int8_t* tg = tags + g.cell_off;
    t = tg[cell];
    if (pass == 1 && t == 2 && !has_face_tag(g, tg, cell, 0)) {
      t = 1;
      tg[cell] = 1;
    } else if (pass == 2) {
      if (t == -2 && !has_face_tag(g, tg, cell, 1)) t = 0;
      else if (t == 2 && !zero_after_pass_a(g, tg, cell)) t = 1;
      iface_tag[m] = t;
    }
  }
  const int flag = (t == 2 || t == -2) ? 1 : 0;
  int agg;
  const int ex = block_excl_scan(flag, sh, agg);
  const long long base = lb_prefix(L, blk, (unsigned)agg, status);
  if (base >= 0) {
    if (on) {
      const int q = (int)(base + ex);
      gpos[m] = q;
      if (flag) {
        if (q >= cap) {
          set_status(status, S_ESHAPE);
        } else {
          gs_cell[q] = cell;
          gs_geo[q] = b;
          uint32_t meta = t == -2 ? (1u << 22) : 0u;
          if (iface_meta) {
            const int dim = G[b].dim;
            meta |= (mb & 7u) | (active_of_zero(dim, mb >> 3) << 15);
            for (int a = 0; a < dim; ++a) meta |= 1u << (3 + 4 * a);
          }
          gs_meta[q] = meta;
        }
      }
    }
    if (m == n_iface - 1) gpos[n_iface] = (int)(base + ex + flag);
  }
  lb_end(L);
}

// psi, S and n in double for the compacted ghosts only (Eq. signed_distance),
// one ghost per thread so that no lane idles through the FP64 work; sign
// bits e, stencil multipliers r (Eq. stencil_anisotropic for CGC_ES) and the
// structurally active members.  split: the compaction wrote the meta words
// from the placement's normals (one-layer HGC) and the dependency kernels
// may be reading them already; this kernel then leaves them alone and only
// checks them against the double normal (EBR_EINVAL on a difference).
__global__ void k_ghost_geom(const Geom* __restrict__ G, int ng, int placement,
                             const int* __restrict__ gs_cell, const int* __restrict__ gs_geo,
                             double* __restrict__ gs_psi, double* __restrict__ gs_n,
                             uint32_t* __restrict__ gs_meta, int split, int* rmax, int* status,
                             const PlanCheck chk) {
  pdl_enter();
  plan_check(G, chk, status);
  const int s = interleaved_item();     // airfoil ghosts cost several times ellipse ghosts
  if (s >= ng) return;
  const Geom& g = G[gs_geo[s]];
  int cell = gs_cell[s];
  const uint32_t m0 = gs_meta[s];
  uint32_t meta = m0 & (1u << 22);
  bool solid = meta == 0;
  double psi, nv[3];
  int i, j, k;
  cell_ijk(g, cell, i, j, k);
  double x = centre_of(g, 0, i), y = centre_of(g, 1, j);
  double z = g.dim == 3 ? centre_of(g, 2, k) : 0.0;
  if (!closest_point(g, x, y, z, solid, psi, nv)) { set_status(status, S_EINVAL); return; }
  int rloc = 1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.dim) continue;
    if (nv[a] < 0.0) meta |= 1u << a;
    int r = 1;
    if (placement == CGC_ES || g.layers == 2) {
      // Eq. stencil_anisotropic: r_i = max(1, ceil(2 |n_i psi| / dx_i)),
      // dx_i the ghost cell's width
      const int ijk[3] = {i, j, k};
      double q = 2.0 * fabs(psi * nv[a]) / width_of(g, a, ijk[a]);
      r = max(1, (int)ceil(q));
    }
    if (r > 15) { set_status(status, S_EINVAL); r = 15; }
    rloc = max(rloc, r);
    meta |= (uint32_t)r << (3 + 4 * a);
  }
  uint32_t zero = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < g.dim && nv[a] == 0.0) zero |= 1u << a;
  const uint32_t act = active_of_zero(g.dim, zero);
  meta |= act << 15;
  gs_psi[s] = psi;
  gs_n[s] = nv[0];
  gs_n[ng + s] = nv[1];
  gs_n[2 * (size_t)ng + s] = nv[2];
  if (split) {
    // the dependency kernel keeps bits 0..14 and narrows the active bits to
    // the in-grid members (an out-of-grid member is an error of its own)
    if ((m0 & 0x7fffu) != (meta & 0x7fffu) || ((m0 >> 15) & 127u & ~act) != 0u)
      set_status(status, S_EINVAL);
  } else {
    gs_meta[s] = meta;
  }
  if (rloc > 1) atomicMax(rmax, rloc);
}

void launch_ghost_compact(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo,
                          int8_t* tags, int pass, const uint8_t* iface_meta, int8_t* iface_tag, int* gpos,
                          int ng_cap, int* gs_cell, int* gs_geo, uint32_t* gs_meta, const Lookback& L,
                          int* status, cudaStream_t s) {
  if (n_iface <= 0) return;
  launch(k_ghost_compact, (n_iface + LB_T - 1) / LB_T, LB_T, 0, s, G, n_iface, iface_cell, iface_geo, tags,
         pass, iface_meta, iface_tag, gpos, ng_cap, gs_cell, gs_geo, gs_meta, L, status);
}

// psi, S, n and (split == 0) the meta words of the compacted ghosts
void launch_ghost_geom(const Geom* G, int placement, int ng_cap, int* gs_cell, int* gs_geo, double* gs_psi,
                       double* gs_n, uint32_t* gs_meta, int split, int* rmax, int* status, cudaStream_t s,
                       int T, const PlanCheck& chk) {
  if (ng_cap <= 0) return;
  launch(k_ghost_geom, (ng_cap + T - 1) / T, T, 0, s, G, ng_cap, placement, gs_cell, gs_geo, gs_psi, gs_n,
         gs_meta, split, rmax, status, chk);
}

void launch_ghost_write(const Geom* G, int n_iface, const int* iface_cell, const int* iface_geo,
                        const int8_t* tags, const int* gpos, int placement, int ng_cap, int* gs_cell,
                        int* gs_geo, double* gs_psi, double* gs_n, uint32_t* gs_meta, int* rmax,
                        int* status, cudaStream_t s, int T) {
  if (n_iface <= 0) return;
  launch(k_ghost_write, (n_iface + 255) / 256, 256, 0, s, G, n_iface, iface_cell, iface_geo, tags, gpos,
                                                      ng_cap, gs_cell, gs_geo, gs_meta, status);
  if (ng_cap <= 0) return;
  launch(k_ghost_geom, (ng_cap + T - 1) / T, T, 0, s, G, ng_cap, placement, gs_cell, gs_geo, gs_psi,
         gs_n, gs_meta, 0, rmax, status, PlanCheck{nullptr, nullptr, nullptr, 0, 0, 0, -1});
}

}  // namespace ebr

// ===========================================================================
// Allocation-free classification of one grid (ebr_classify_cells_static).
//
// For callers that cannot let the library allocate device memory.  The
// per-row solid runs this needs between its two kernels live in a fixed
// file-scope device array (EBR_STATIC_MAX_ROWS rows, 2 MiB, resident on every
// device that loads the library until the process exits).  Every call shares
// that array: calls that overlap on the GPU race on it.
// ===========================================================================
#include "../../include/ebr.h"

namespace {

constexpr int kStaticMaxRows = EBR_STATIC_MAX_ROWS;

// [0, 2 * rows): int2 row runs; then the status word and the fallback counter
static __device__ __align__(256) int g_static_scratch[2 * kStaticMaxRows + 64];

__global__ void __launch_bounds__(256) k_rows_static(ebr::Geom g, int2* __restrict__ runs,
                                                     int8_t* __restrict__ tags, int* status,
                                                     int* stats) {
  using namespace ebr;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int total_rows = g.n_rows;
  for (int base = warp * 32; base < total_rows; base += nwarps * 32) {
    int row = base + lane;
    int s = 0, t = -1;
    long long start = 0;
    const int nx = g.n[0];
    if (row < total_rows) {
      int j = row % g.n[1];
      int k = row / g.n[1];
      exact_run(g, j, k, s, t, status, stats);
      runs[row] = make_int2(s, t);
      start = (long long)row * nx;
    }
    int nvalid = min(32, total_rows - base);
    for (int r = 0; r < nvalid; ++r) {
      int rs = __shfl_sync(0xffffffffu, s, r);
      int rt = __shfl_sync(0xffffffffu, t, r);
      long long rst = __shfl_sync(0xffffffffu, start, r);
      long long end = rst + nx;
      long long mis = (long long)(reinterpret_cast<uintptr_t>(tags) & 15u);
      long long a0 = ((rst + mis + 15) & ~15LL) - mis;
      long long a1 = ((end + mis) & ~15LL) - mis;
      if (a0 > end) a0 = end;
      if (a1 < a0) a1 = a0;
      long long nh = a0 - rst, nt = end - a1;
      if (lane < nh) tags[rst + lane] = (int8_t)(lane >= rs && lane <= rt);
      if (lane < nt) {
        long long i = a1 + lane - rst;
        tags[a1 + lane] = (int8_t)(i >= rs && i <= rt);
      }
      for (long long c = a0 + 16LL * lane; c < a1; c += 16LL * 32) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t v = 0;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            long long i = c + 4 * q + m - rst;
            v |= (uint32_t)(i >= rs && i <= rt) << (8 * m);
          }
          w[q] = v;
        }
        *reinterpret_cast<uint4*>(tags + c) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
}

// After the count: a device-side failure recorded by the row kernel (a row
// whose solid run could not be determined leaves that row all fluid) replaces
// the count by the negative status, so the caller sees it.
__global__ void k_static_status(const int* __restrict__ status, long long* __restrict__ count) {
  const int st = *status;
  if (st != 0) *count = st;
}

// interface cells per row from the runs (same interval algebra as k_iface),
// summed into the caller's counter
__global__ void k_iface_count_static(ebr::Geom g, const int2* __restrict__ runs,
                                     unsigned long long* __restrict__ count) {
  using namespace ebr;
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = 0;
  if (row < g.n_rows) {
    int ny = g.n[1], nz = g.dim == 3 ? g.n[2] : 1, n = g.n[0];
    int j = row % ny, k = row / ny;
    int2 R = runs[row];
    Iv v[24];
    int m = 0;
    if (R.x <= R.y) {
      if (R.x > 0) { add_iv(v, m, R.x, R.x, n); add_iv(v, m, R.x - 1, R.x - 1, n); }
      if (R.y < n - 1) { add_iv(v, m, R.y, R.y, n); add_iv(v, m, R.y + 1, R.y + 1, n); }
    }
    const int dj[4] = {-1, 1, 0, 0}, dk[4] = {0, 0, -1, 1};
    for (int q = 0; q < 4; ++q) {
      int jj = j + dj[q], kk = k + dk[q];
      if (jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
      int2 Q = runs[jj + ny * kk];
      add_diff(v, m, R, Q, n);
      add_diff(v, m, Q, R, n);
    }
    for (int x = 1; x < m; ++x) {
      Iv key = v[x];
      int y = x - 1;
      while (y >= 0 && v[y].a > key.a) { v[y + 1] = v[y]; --y; }
      v[y + 1] = key;
    }
    int w = 0;
    for (int x = 0; x < m; ++x) {
      if (w > 0 && v[x].a <= v[w - 1].b + 1) v[w - 1].b = max(v[w - 1].b, v[x].b);
      else v[w++] = v[x];
    }
    for (int x = 0; x < w; ++x) cnt += v[x].b - v[x].a + 1;
  }
  // warp reduction, one atomic per warp (integer: order-independent)
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(count, (unsigned long long)cnt);
}

}  // namespace

extern "C" ebr_status ebr_classify_cells_static(const ebr_grid* h_grid, const ebr_body* h_body,
                                                int8_t* d_tags, int64_t* d_n_interface,
                                                ebr_stream stream) {
  using namespace ebr;
  if (!h_grid || !h_body || !d_tags || !d_n_interface) return EBR_EINVAL;
  const ebr_grid& gr = *h_grid;
  const ebr_body& bd = *h_body;
  if (gr.dim != 2 && gr.dim != 3) return EBR_EINVAL;
  if (bd.kind < 0 || bd.kind > 3) return EBR_EINVAL;
  if ((bd.kind == EBR_SPHERE ? 3 : 2) != gr.dim) return EBR_EINVAL;
  Geom g{};
  g.dim = gr.dim;
  long long n3 = 1;
  for (int a = 0; a < 3; ++a) {
    long long na = a < gr.dim ? gr.n[a] : 1;
    if (a < gr.dim && (na < 2 || !(gr.hi[a] > gr.lo[a]))) return EBR_EINVAL;
    g.n[a] = (int)na;
    g.lo[a] = a < gr.dim ? gr.lo[a] : 0.0;
    g.h[a] = a < gr.dim ? (gr.hi[a] - gr.lo[a]) / (double)na : 1.0;
    n3 *= na;
  }
  if (n3 > (1LL << 31) - 1) return EBR_EINVAL;
  long long rows = (long long)g.n[1] * g.n[2];
  if (rows > kStaticMaxRows) return EBR_EINVAL;     // more rows than the fixed scratch holds
  g.kind = bd.kind;
  for (int a = 0; a < 3; ++a) { g.centre[a] = bd.centre[a]; g.radii[a] = bd.radii[a]; }
  for (int q = 0; q < 9; ++q) g.rot[q] = bd.rot[q];
  g.t = bd.thickness;
  g.c = bd.chord;
  if ((bd.kind == EBR_CIRCLE || bd.kind == EBR_SPHERE) && !(bd.radii[0] > 0)) return EBR_EINVAL;
  if (bd.kind == EBR_ELLIPSE && !(bd.radii[0] > 0 && bd.radii[1] > 0)) return EBR_EINVAL;
  if (bd.kind == EBR_AIRFOIL4 && !(bd.thickness > 0 && bd.chord > 0 && bd.rot[0] > 0)) return EBR_EINVAL;
  g.cell_off = 0;
  g.row_off = 0;
  g.n_rows = (int)rows;

  // Device address of the fixed scratch in the current context (the array's
  // name is only a host-side stand-in).  Looked up on every call: the address
  // belongs to the module as loaded in the current context, so a cached value
  // would dangle after a device reset or name another context's copy.  Once
  // the module is loaded in the context this is a table lookup; the first call
  // in a context may load it, so it should come before any stream capture.
  void* sym = nullptr;
  if (cudaGetSymbolAddress(&sym, g_static_scratch) != cudaSuccess) {
    cudaGetLastError();
    return EBR_ECUDA;
  }
  int* base = static_cast<int*>(sym);
  int2* runs = reinterpret_cast<int2*>(base);
  int* status = base + 2 * kStaticMaxRows;
  int* stats = status + 1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(status, 0, 2 * sizeof(int), s) != cudaSuccess) return EBR_ECUDA;
  if (cudaMemsetAsync(d_n_interface, 0, sizeof(int64_t), s) != cudaSuccess) return EBR_ECUDA;
  int warps = (int)((rows + 31) / 32);
  k_rows_static<<<(warps + 7) / 8, 256, 0, s>>>(g, runs, d_tags, status, stats);
  k_iface_count_static<<<(int)((rows + 127) / 128), 128, 0, s>>>(
      g, runs, reinterpret_cast<unsigned long long*>(d_n_interface));
  k_static_status<<<1, 1, 0, s>>>(status, reinterpret_cast<long long*>(d_n_interface));
  if (cudaGetLastError() != cudaSuccess) return EBR_ECUDA;
  return EBR_OK;
}
