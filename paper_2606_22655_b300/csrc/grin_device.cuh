// grin_device.cuh -- device building blocks of the VRT kernels: index-field
// evaluators (polynomial by nested Horner, tricubic Catmull-Rom gathers),
// enclosing-surface geometry in FP64, and the FP64 vectorial Snell law.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "grin_internal.h"

namespace grin {

// ------------------------------------------------------------- polynomial

// Precision-exact overloads (fmaf / floorf / fmaxf / fminf for float, their
// double versions for double), so that templates never promote to FP64.
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float vfloor(float a) { return floorf(a); }
__device__ __forceinline__ double vfloor(double a) { return ::floor(a); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return ::fmax(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return ::fmin(a, b); }

__host__ __device__ constexpr int tri_count(int m) { return (m + 1) * (m + 2) / 2; }

// Position of c_{ijk} (coefficient of x^i y^j z^k, i + j + k <= D) in the
// Horner layout: blocks by i, inside a block rows by j, inside a row by k.
__host__ __device__ constexpr int hidx(int D, int i, int j, int k) {
  int o = 0;
  for (int ii = 0; ii < i; ++ii) o += tri_count(D - ii);
  for (int jj = 0; jj < j; ++jj) o += D - i - jj + 1;
  return o + k;
}

// p(x, y, z) = sum_i x^i sum_j y^j sum_k c_ijk z^k and its three partials by
// nested Horner with derivative accumulators (one FMA per coefficient for the
// value, one per coefficient and partial for the gradient).  Fully unrolled:
// D is a compile-time constant and every index folds to a constant.
template <int D, typename T>
__device__ __forceinline__ void poly_vg(const T* __restrict__ c, T x, T y, T z, T& p, T& px,
                                        T& py, T& pz) {
  T P = T(0), PX = T(0), PY = T(0), PZ = T(0);
#pragma unroll
  for (int i = D; i >= 0; --i) {
    T A = T(0), AY = T(0), AZ = T(0);
#pragma unroll
    for (int j = D - i; j >= 0; --j) {
      const int top = D - i - j;
      T B = c[hidx(D, i, j, top)];
      T BZ = T(0);
#pragma unroll
      for (int k = top - 1; k >= 0; --k) {
        BZ = (k == top - 1) ? B : fmadd(BZ, z, B);
        B = fmadd(B, z, c[hidx(D, i, j, k)]);
      }
      if (j == D - i) {
        A = B;
        AZ = BZ;
      } else {
        AY = (j == D - i - 1) ? A : fmadd(AY, y, A);
        A = fmadd(A, y, B);
        AZ = fmadd(AZ, y, BZ);
      }
    }
    if (i == D) {
      P = A;
      PY = AY;
      PZ = AZ;
    } else {
      PX = (i == D - 1) ? P : fmadd(PX, x, P);
      P = fmadd(P, x, A);
      PY = fmadd(PY, x, AY);
      PZ = fmadd(PZ, x, AZ);
    }
  }
  p = P;
  px = PX;
  py = PY;
  pz = PZ;
}

// Spherical freeform field of Sec. V and its gradient in the normalised
// coordinates: p = a0 + a1 G1 + a2 G2 + a3 G3 with G1 = 0.3 (r^2 - 1),
// G2 = r cos(5 theta) = z (16 t^2 - 20 t + 5), t = z^2 / r^2 = cos^2(theta)
// (Chebyshev T5), and G3 = r^2 sin^2(theta) cos(2 phi) = x^2 - y^2; at r = 0
// the polar angle is taken as 0 (t = 1).
template <typename T>
__device__ __forceinline__ void sph_vg(const T* a, T x, T y, T z, T& p, T& px, T& py, T& pz) {
  const T r2 = fmadd(x, x, fmadd(y, y, z * z));
  T t = T(1), tx = T(0), ty = T(0), tz = T(0);
  if (r2 > T(0)) {
    const T inv = T(1) / r2;
    t = z * z * inv;
    const T k = T(-2) * t * inv;
    tx = k * x;
    ty = k * y;
    tz = T(2) * z * (T(1) - t) * inv;
  }
  const T q = fmadd(fmadd(T(16), t, T(-20)), t, T(5));  // cos(5 theta) / cos(theta)
  const T zq = z * fmadd(T(32), t, T(-20));             // z dq/dt
  p = fmadd(a[1], T(0.3) * (r2 - T(1)), fmadd(a[2], z * q, fmadd(a[3], fmadd(x, x, -y * y), a[0])));
  px = fmadd(a[1], T(0.6) * x, fmadd(a[2], zq * tx, a[3] * (T(2) * x)));
  py = fmadd(a[1], T(0.6) * y, fmadd(a[2], zq * ty, a[3] * (T(-2) * y)));
  pz = fmadd(a[1], T(0.6) * z, a[2] * fmadd(zq, tz, q));
}

// N2P-GRIN cylinder lens of Sec. VI at (x, y) from its axis:
// n = [1 + u^beta]^gamma, u = (R^2 - (rho/2)^2) / F^2, c = (R, F, beta,
// gamma, shift); returns p = n - shift.  Two powers: w^(gamma - 1) = n / w and
// u^(beta - 1) = u^beta / u in dn/dx = gamma w^(gamma-1) beta u^(beta-1) (-x / (2 F^2)).
template <typename T>
__device__ __forceinline__ void n2p_vg(const T* c, T x, T y, T& p, T& px, T& py, T& pz) {
  const T R = c[0], F = c[1], be = c[2], ga = c[3];
  const T inv_f2 = T(1) / (F * F);
  const T u = fmadd(T(-0.25), fmadd(x, x, y * y), R * R) * inv_f2;
  const T ub = pow(u, be);
  const T w = T(1) + ub;
  const T n = pow(w, ga);
  const T k = ga * (n / w) * be * (ub / u) * (T(-0.5) * inv_f2);
  p = n - c[4];
  px = k * x;
  py = k * y;
  pz = T(0);
}

// The analytic field of class PC: a polynomial, the spherical freeform field
// (PC == kSpherical, coefficients a0..a3) or the N2P lens (PC == kN2P).
template <int PC, typename T>
__device__ __forceinline__ void field_vg(const T* c, T x, T y, T z, T& p, T& px, T& py, T& pz) {
  if constexpr (PC == kSpherical)
    sph_vg<T>(c, x, y, z, p, px, py, pz);
  else if constexpr (PC == kN2P)
    n2p_vg<T>(c, x, y, p, px, py, pz);
  else
    poly_vg<PC, T>(c, x, y, z, p, px, py, pz);
}

// ------------------------------------------------------- tricubic gathers

// Catmull-Rom (Keys cubic convolution, a = -1/2) weights for the taps at -1,
// 0, 1, 2 of the cell containing fraction t, and their t-derivatives, in
// Horner form with the halves folded into the coefficients (18 operations).
template <typename T>
__device__ __forceinline__ void cr_w(T t, T* w, T* dw) {
  const T t2 = t * t;
  const T b = fmadd(T(-1.5), t, T(2));
  w[0] = t * fmadd(fmadd(T(-0.5), t, T(1)), t, T(-0.5));  // (-t^3 + 2t^2 - t) / 2
  w[1] = fmadd(t2, fmadd(T(1.5), t, T(-2.5)), T(1));       // (3t^3 - 5t^2 + 2) / 2
  w[2] = t * fmadd(b, t, T(0.5));                         // (-3t^3 + 4t^2 + t) / 2
  w[3] = t2 * fmadd(T(0.5), t, T(-0.5));                  // (t^3 - t^2) / 2
  dw[0] = fmadd(b, t, T(-0.5));                           // (-3t^2 + 4t - 1) / 2
  dw[1] = t * fmadd(T(4.5), t, T(-5));                    // (9t^2 - 10t) / 2
  dw[2] = fmadd(fmadd(T(-4.5), t, T(4)), t, T(0.5));      // (-9t^2 + 8t + 1) / 2
  dw[3] = t * fmadd(T(1.5), t, T(-1));                    // (3t^2 - 2t) / 2
}

// Interpolated (sample - sub) and its gradient in grid units, from 64 taps
// (edge-clamped).  The x sums of each of the 16 rows are taken first, then y,
// then z: 192 FMAs and 64 cached 4-byte gathers.  Subtracting `sub` (a value
// near the samples) per tap keeps the FP32 result's low bits.
// When the grid's rows start on 16-byte boundaries and no x tap is clamped,
// each row's 4 taps come from the aligned 16-byte block holding the first
// tap and, when the taps straddle it, the next one: 1 or 2 vector loads a row
// instead of 4 scalar ones (half the L1 wavefronts of a scattered warp).  The
// x weights are spread over the 8 loaded positions with zeros around the
// taps, so each row sums the same products in the same order.
template <typename T>
__device__ __forceinline__ void grid_vg(const DevMedium& m, const T* u_in, T sub, T& v, T& gx,
                                        T& gy, T& gz) {
  const int n[3] = {m.nx, m.ny, m.nz};
  T w[3][4], dw[3][4];
  int idx[3][4];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T u = u_in[a];
    u = vmax(u, T(-2));  // a NaN also lands here
    u = vmin(u, T(n[a] + 1));
    T fl = vfloor(u);
    int i0 = (int)fl;
    cr_w(u - fl, w[a], dw[a]);
#pragma unroll
    for (int t = 0; t < 4; ++t) idx[a][t] = min(max(i0 - 1 + t, 0), n[a] - 1);
  }
  const float* __restrict__ g = m.grid;
  T V = T(0), GX = T(0), GY = T(0), GZ = T(0);
  const int x0 = idx[0][0];  // first x tap (unclamped when the window is inside the row)
  const bool vec = m.rows16 && idx[0][0] == idx[0][1] - 1 && idx[0][3] == idx[0][0] + 3;
  if (vec) {
    const int ax = x0 & ~3, o = x0 - ax;  // aligned block start, tap offset in it
    T wx[8], dwx[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const int t = p - o;
      wx[p] = t == 0 ? w[0][0] : t == 1 ? w[0][1] : t == 2 ? w[0][2] : t == 3 ? w[0][3] : T(0);
      dwx[p] = t == 0 ? dw[0][0] : t == 1 ? dw[0][1] : t == 2 ? dw[0][2] : t == 3 ? dw[0][3] : T(0);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      T sv = T(0), sx = T(0), sy = T(0);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int64_t rb = ((int64_t)idx[2][c] * n[1] + idx[1][b]) * n[0] + ax;
        const float4* __restrict__ row4 = reinterpret_cast<const float4*>(
            g + GRIN_IDX(m, rb, m.grid_n - (o ? 7 : 3), kSiteGridFP64));
        const float4 A = __ldg(row4);
        const float4 B = o ? __ldg(row4 + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float q[8] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w};
        T r = T(0), rx = T(0);
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const T s = (T)q[p] - sub;
          r = fmadd(wx[p], s, r);
          rx = fmadd(dwx[p], s, rx);
        }
        sv = fmadd(w[1][b], r, sv);
        sx = fmadd(w[1][b], rx, sx);
        sy = fmadd(dw[1][b], r, sy);
      }
      V = fmadd(w[2][c], sv, V);
      GX = fmadd(w[2][c], sx, GX);
      GY = fmadd(w[2][c], sy, GY);
      GZ = fmadd(dw[2][c], sv, GZ);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      T sv = T(0), sx = T(0), sy = T(0);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int64_t rb = ((int64_t)idx[2][c] * n[1] + idx[1][b]) * n[0];
        T r = T(0), rx = T(0);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          T s = (T)__ldg(g + GRIN_IDX(m, rb + idx[0][a], m.grid_n, kSiteGridFP64)) - sub;
          r = fmadd(w[0][a], s, r);
          rx = fmadd(dw[0][a], s, rx);
        }
        sv = fmadd(w[1][b], r, sv);
        sx = fmadd(w[1][b], rx, sx);
        sy = fmadd(dw[1][b], r, sy);
      }
      V = fmadd(w[2][c], sv, V);
      GX = fmadd(w[2][c], sx, GX);
      GY = fmadd(w[2][c], sy, GY);
      GZ = fmadd(dw[2][c], sv, GZ);
    }
  }
  v = V;
  gx = GX;
  gy = GY;
  gz = GZ;
}

// --------------------------------------------------------- FP64 geometry

struct V3 {
  double x, y, z;
};

__device__ __forceinline__ V3 mk(double x, double y, double z) { return V3{x, y, z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 axpy(double s, V3 a, V3 b) {  // s a + b
  return mk(fma(s, a.x, b.x), fma(s, a.y, b.y), fma(s, a.z, b.z));
}
__device__ __forceinline__ V3 scale(double s, V3 a) { return mk(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ V3 unit(V3 a) {
  double l = sqrt(dot(a, a));
  return mk(a.x / l, a.y / l, a.z / l);
}
__device__ __forceinline__ double comp(V3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }
__device__ __forceinline__ void set_comp(V3& a, int k, double v) {
  if (k == 0) a.x = v;
  else if (k == 1) a.y = v;
  else a.z = v;
}

// Strictly inside the enclosing surface (a point on it is outside).
__device__ __forceinline__ bool inside64(const DevMedium& m, V3 p) {
  const double* b = m.b;
  if (m.bkind == GRIN_BOUNDARY_BOX)
    return p.x > b[0] && p.x < b[3] && p.y > b[1] && p.y < b[4] && p.z > b[2] && p.z < b[5];
  if (m.bkind == GRIN_BOUNDARY_SPHERE) {
    V3 r = mk(p.x - b[0], p.y - b[1], p.z - b[2]);
    return dot(r, r) < b[3] * b[3];
  }
  double x = p.x - b[0], y = p.y - b[1];
  return x * x + y * y < b[2] * b[2] && p.z > b[3] && p.z < b[4];
}

// Roots t1 <= t2 of a t^2 + b t + c = 0 without cancellation; false if none.
__device__ __forceinline__ bool roots2(double a, double b, double c, double& t1, double& t2) {
  double disc = b * b - 4.0 * a * c;
  if (disc < 0.0) return false;
  double sq = sqrt(disc);
  double q = b >= 0.0 ? -0.5 * (b + sq) : 0.5 * (sq - b);
  double r1 = 0.0, r2 = 0.0;
  if (q != 0.0) {
    r1 = q / a;
    r2 = c / q;
  }
  t1 = fmin(r1, r2);
  t2 = fmax(r1, r2);
  return true;
}

// First hit of p0 + t d, t >= 0, from outside; entry point, outward normal
// and face id.  A box entry point is snapped onto its face plane.
__device__ inline bool enter64(const DevMedium& m, V3 p0, V3 d, double& t, V3& pb, V3& nb, int& face) {
  const double* b = m.b;
  if (m.bkind == GRIN_BOUNDARY_BOX) {
    double tn = -INFINITY, tf = INFINITY;
    int axis = -1, hi = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double o = comp(p0, k), dk = comp(d, k);
      if (dk == 0.0) {
        if (!(o > b[k] && o < b[3 + k])) return false;
        continue;
      }
      double t1 = (b[k] - o) / dk, t2 = (b[3 + k] - o) / dk;
      double lo = fmin(t1, t2), up = fmax(t1, t2);
      if (lo > tn) {
        tn = lo;
        axis = k;
        hi = dk < 0.0;
      }
      tf = fmin(tf, up);
    }
    if (axis < 0 || !(tn >= 0.0 && tn < tf)) return false;
    t = tn;
    pb = axpy(tn, d, p0);
    set_comp(pb, axis, hi ? b[3 + axis] : b[axis]);
    nb = mk(0.0, 0.0, 0.0);
    set_comp(nb, axis, hi ? 1.0 : -1.0);
    face = 2 * axis + hi;
    return true;
  }
  if (m.bkind == GRIN_BOUNDARY_SPHERE) {
    V3 r = mk(p0.x - b[0], p0.y - b[1], p0.z - b[2]);
    double t1, t2;
    if (!roots2(dot(d, d), 2.0 * dot(r, d), dot(r, r) - b[3] * b[3], t1, t2)) return false;
    if (!(t1 >= 0.0)) return false;
    t = t1;
    pb = axpy(t1, d, p0);
    nb = unit(mk(pb.x - b[0], pb.y - b[1], pb.z - b[2]));
    face = 0;
    return true;
  }
  double x = p0.x - b[0], y = p0.y - b[1];
  double a2 = d.x * d.x + d.y * d.y;
  double s1 = -INFINITY, s2 = INFINITY;
  if (a2 > 0.0) {
    if (!roots2(a2, 2.0 * (x * d.x + y * d.y), x * x + y * y - b[2] * b[2], s1, s2)) return false;
    if (!(s1 < s2)) return false;
  } else if (!(x * x + y * y < b[2] * b[2])) {
    return false;
  }
  double z1 = -INFINITY, z2 = INFINITY;
  if (d.z != 0.0) {
    double u1 = (b[3] - p0.z) / d.z, u2 = (b[4] - p0.z) / d.z;
    z1 = fmin(u1, u2);
    z2 = fmax(u1, u2);
  } else if (!(p0.z > b[3] && p0.z < b[4])) {
    return false;
  }
  bool side = s1 > z1;
  double tn = side ? s1 : z1, tf = fmin(s2, z2);
  if (!(tn >= 0.0 && tn < tf)) return false;
  t = tn;
  pb = axpy(tn, d, p0);
  if (side) {
    nb = unit(mk(pb.x - b[0], pb.y - b[1], 0.0));
    face = 0;
  } else {
    bool top = d.z < 0.0;
    pb.z = top ? b[4] : b[3];
    nb = mk(0.0, 0.0, top ? 1.0 : -1.0);
    face = top ? 2 : 1;
  }
  return true;
}

// Crossing of the segment p -> q (p inside or on the surface, q outside):
// fraction t in [0, 1], crossing point, outward normal, face id.
__device__ inline void exit64(const DevMedium& m, V3 p, V3 q, double& t, V3& pb, V3& nb, int& face) {
  const double* b = m.b;
  V3 D = mk(q.x - p.x, q.y - p.y, q.z - p.z);
  double best = INFINITY;
  int bf = 0;
  if (m.bkind == GRIN_BOUNDARY_BOX) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double qk = comp(q, k), pk = comp(p, k), dk = comp(D, k);
      if (qk <= b[k]) {
        double tk = (b[k] - pk) / dk;
        if (tk < best) {
          best = tk;
          bf = 2 * k;
        }
      }
      if (qk >= b[3 + k]) {
        double tk = (b[3 + k] - pk) / dk;
        if (tk < best) {
          best = tk;
          bf = 2 * k + 1;
        }
      }
    }
  } else if (m.bkind == GRIN_BOUNDARY_SPHERE) {
    V3 r = mk(p.x - b[0], p.y - b[1], p.z - b[2]);
    double t1 = 0.0, t2 = 0.0;
    roots2(dot(D, D), 2.0 * dot(r, D), dot(r, r) - b[3] * b[3], t1, t2);
    best = t2;
  } else {
    double x = p.x - b[0], y = p.y - b[1];
    double qx = q.x - b[0], qy = q.y - b[1];
    if (qx * qx + qy * qy >= b[2] * b[2]) {
      double t1 = 0.0, t2 = 0.0;
      roots2(D.x * D.x + D.y * D.y, 2.0 * (x * D.x + y * D.y), x * x + y * y - b[2] * b[2], t1, t2);
      best = t2;
    }
    if (q.z <= b[3]) {
      double tk = (b[3] - p.z) / D.z;
      if (tk < best) {
        best = tk;
        bf = 1;
      }
    }
    if (q.z >= b[4]) {
      double tk = (b[4] - p.z) / D.z;
      if (tk < best) {
        best = tk;
        bf = 2;
      }
    }
  }
  if (!(best > 0.0)) best = 0.0;
  if (best > 1.0) best = 1.0;
  t = best;
  face = bf;
  pb = axpy(best, D, p);
  nb = mk(0.0, 0.0, 0.0);
  if (m.bkind == GRIN_BOUNDARY_BOX) {
    int k = bf >> 1;
    set_comp(pb, k, (bf & 1) ? b[3 + k] : b[k]);
    set_comp(nb, k, (bf & 1) ? 1.0 : -1.0);
  } else if (m.bkind == GRIN_BOUNDARY_SPHERE) {
    nb = unit(mk(pb.x - b[0], pb.y - b[1], pb.z - b[2]));
  } else if (bf == 0) {
    nb = unit(mk(pb.x - b[0], pb.y - b[1], 0.0));
  } else {
    pb.z = bf == 2 ? b[4] : b[3];
    nb.z = bf == 2 ? 1.0 : -1.0;
  }
}

// Vectorial Snell law (Eq. 8-9, positive root) or, when
// D = 1 - mu^2 (1 - (N.I)^2) <= 0, the reflection I - 2 (I.N) N of Sec. II
// (v).  d is replaced by the unit result; returns true on reflection.
__device__ __forceinline__ bool refract64(V3& d, V3 N, double mu, double* crit = nullptr) {
  double c = dot(N, d);
  double D = 1.0 - mu * mu * (1.0 - c * c);
  if (crit)  // |N.I| minus its critical value, for mu > 1
    *crit = mu > 1.0 ? fabs(D) / (mu * mu * (fabs(c) + sqrt(1.0 - 1.0 / (mu * mu)))) : INFINITY;
  if (D <= 0.0) {
    d = unit(axpy(-2.0 * c, N, d));
    return true;
  }
  double s = c > 0.0 ? 1.0 : (c < 0.0 ? -1.0 : 0.0);
  double gamma = fma(s, sqrt(D), -mu * c);
  d = unit(axpy(gamma, N, scale(mu, d)));
  return false;
}

// n (after layering) and grad n of the smooth field in FP64 with Horner
// polynomials and fused multiply-adds (the fast FP64 tracer's evaluator, also
// the mixed tracer's at shell crossings).
template <int PC, bool GRID, bool LAYERED>
struct Field64Fast {
  // n (after layering) and grad of the smooth field at p; lvl = level (or 0).
  static __device__ __forceinline__ void eval(const DevMedium& m, V3 p, double& n, V3& g,
                                              int& lvl) {
    double f;
    if (GRID) {
      double u[3] = {(p.x - m.origin[0]) * m.inv_spacing[0], (p.y - m.origin[1]) * m.inv_spacing[1],
                     (p.z - m.origin[2]) * m.inv_spacing[2]};
      double v, gx, gy, gz;
      grid_vg<double>(m, u, 0.0, v, gx, gy, gz);
      f = v;
      g = mk(gx * m.inv_spacing[0], gy * m.inv_spacing[1], gz * m.inv_spacing[2]);
    } else {
      double x = (p.x - m.off[0]) * m.inv_scale[0];
      double y = (p.y - m.off[1]) * m.inv_scale[1];
      double z = (p.z - m.off[2]) * m.inv_scale[2];
      double q, qx, qy, qz;
      field_vg<PC, double>(m.c64, x, y, z, q, qx, qy, qz);
      V3 gq = mk(qx * m.inv_scale[0], qy * m.inv_scale[1], qz * m.inv_scale[2]);
      if (m.form == GRIN_FORM_LINEAR) {
        f = q;
        g = gq;
      } else if (m.form == GRIN_FORM_SQRT) {
        f = sqrt(q);
        g = scale(0.5 / f, gq);
      } else {
        f = m.form_c / q;
        g = scale(-f / q, gq);
      }
    }
    if (LAYERED) {
      double u = (f - m.lvl_lo) * (double)m.n_levels / m.lvl_span;
      double fl = floor(u);
      int k = fl >= 0.0 ? (fl > (double)(m.n_levels - 1) ? m.n_levels - 1 : (int)fl) : 0;
      lvl = k;
      n = m.lvl_lo + ((double)k + 0.5) * m.lvl_span / (double)m.n_levels;
    } else {
      lvl = 0;
      n = f;
    }
  }
};

// ------------------------------------------------------------- ray I/O

__device__ __forceinline__ double ld(const void* p, int64_t i, int dtype) {
  return dtype == GRIN_F64 ? __ldg((const double*)p + i) : (double)__ldg((const float*)p + i);
}

__device__ __forceinline__ void store_ray(const TraceArgs& a, int64_t r, V3 p, V3 d, double opl,
                                          int exit_id, int steps, int tir_i, int tir_b) {
  a.px[r] = p.x;
  a.py[r] = p.y;
  a.pz[r] = p.z;
  a.ux[r] = d.x;
  a.uy[r] = d.y;
  a.uz[r] = d.z;
  a.opl[r] = opl;
  a.exit_id[r] = exit_id;
  a.steps[r] = steps;
  a.tir_i[r] = tir_i;
  a.tir_b[r] = tir_b;
}

__device__ __forceinline__ bool finite3(V3 v) {
  return isfinite(v.x) && isfinite(v.y) && isfinite(v.z);
}

}  // namespace grin
