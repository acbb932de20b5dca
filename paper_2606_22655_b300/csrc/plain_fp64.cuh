// plain_fp64.cuh -- the plain FP64 evaluation of the VRT step's pieces:
// monomial-sum polynomials, the 64-term tricubic sum, the enclosing
// surface and the vectorial Snell law, every expression unfused in a fixed
// left-to-right order.  Included by trace_fp64.cu and adjoint.cu, both
// compiled with --fmad=false, so that the adjoint's forward sweep takes
// exactly the plain tracer's decisions.
#pragma once

#include "grin_device.cuh"

namespace grin {
namespace plain {

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void normalize3(double* a) {
  double l = sqrt(dot3(a, a));
  a[0] = a[0] / l;
  a[1] = a[1] / l;
  a[2] = a[2] / l;
}
__device__ __forceinline__ bool finite3(const double* a) {
  return isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]);
}

// Sum over monomials of total degree <= D (zero-padded beyond the medium's
// degree; a zero term adds exactly nothing), powers by repeated products.
template <int D>
__device__ __forceinline__ void poly(const DevMedium& m, const double* P, double& p, double* gp) {
  double x = (P[0] - m.off[0]) / m.scale[0];
  double y = (P[1] - m.off[1]) / m.scale[1];
  double z = (P[2] - m.off[2]) / m.scale[2];
  double px[D + 1], py[D + 1], pz[D + 1];
  px[0] = py[0] = pz[0] = 1.0;
#pragma unroll
  for (int e = 1; e <= D; ++e) {
    px[e] = px[e - 1] * x;
    py[e] = py[e - 1] * y;
    pz[e] = pz[e - 1] * z;
  }
  double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  int idx = 0;
#pragma unroll
  for (int s = 0; s <= D; ++s) {
#pragma unroll
    for (int i = s; i >= 0; --i) {
#pragma unroll
      for (int j = s - i; j >= 0; --j) {
        const int k = s - i - j;
        const double c = m.cglex[idx++];
        v += c * (px[i] * py[j] * pz[k]);
        if (i > 0) gx += c * ((double)i * px[i - 1] * py[j] * pz[k]);
        if (j > 0) gy += c * ((double)j * px[i] * py[j - 1] * pz[k]);
        if (k > 0) gz += c * ((double)k * px[i] * py[j] * pz[k - 1]);
      }
    }
  }
  p = v;
  gp[0] = gx / m.scale[0];
  gp[1] = gy / m.scale[1];
  gp[2] = gz / m.scale[2];
}

// Keys cubic convolution (a = -1/2) weights and t-derivatives.
__device__ __forceinline__ void keys(double t, double* w, double* dw) {
  double t2 = t * t, t3 = t2 * t;
  w[0] = (-t3 + 2.0 * t2 - t) / 2.0;
  w[1] = (3.0 * t3 - 5.0 * t2 + 2.0) / 2.0;
  w[2] = (-3.0 * t3 + 4.0 * t2 + t) / 2.0;
  w[3] = (t3 - t2) / 2.0;
  dw[0] = (-3.0 * t2 + 4.0 * t - 1.0) / 2.0;
  dw[1] = (9.0 * t2 - 10.0 * t) / 2.0;
  dw[2] = (-9.0 * t2 + 8.0 * t + 1.0) / 2.0;
  dw[3] = (3.0 * t2 - 2.0 * t) / 2.0;
}

__device__ __forceinline__ void tricubic(const DevMedium& m, const double* P, double& f,
                                         double* gf) {
  const int n[3] = {m.nx, m.ny, m.nz};
  int b0[3];
  double w[3][4], dw[3][4];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double u = (P[a] - m.origin[a]) / m.spacing[a];
    if (!(u > -2.0)) u = -2.0;
    if (u > (double)n[a] + 1.0) u = (double)n[a] + 1.0;
    double fl = floor(u);
    b0[a] = (int)fl;
    keys(u - fl, w[a], dw[a]);
  }
  double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  for (int c = 0; c < 4; ++c) {
    int kk = min(max(b0[2] - 1 + c, 0), n[2] - 1);
    for (int b = 0; b < 4; ++b) {
      int jj = min(max(b0[1] - 1 + b, 0), n[1] - 1);
      const int64_t row = ((int64_t)kk * n[1] + jj) * n[0];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        int ii = min(max(b0[0] - 1 + a, 0), n[0] - 1);
        double s = (double)__ldg(m.grid + GRIN_IDX(m, row + ii, m.grid_n, kSiteGridFP64));
        v += w[0][a] * w[1][b] * w[2][c] * s;
        gx += dw[0][a] * w[1][b] * w[2][c] * s;
        gy += w[0][a] * dw[1][b] * w[2][c] * s;
        gz += w[0][a] * w[1][b] * dw[2][c] * s;
      }
    }
  }
  f = v;
  gf[0] = gx / m.spacing[0];
  gf[1] = gy / m.spacing[1];
  gf[2] = gz / m.spacing[2];
}

// Spherical freeform field of Sec. V in the normalised coordinates,
// p = a0 + a1 G1 + a2 G2 + a3 G3 with G1 = 0.3 (r^2 - 1), G2 = r cos(5 theta)
// written as z (16 t^2 - 20 t + 5), t = z^2 / r^2 (cos(theta) = z / r and
// Chebyshev T5), and G3 = r^2 sin^2(theta) cos(2 phi) written as x^2 - y^2;
// the gradient from those forms.  At r = 0 the polar angle is taken as 0.
__device__ __forceinline__ void sph(const DevMedium& m, const double* P, double& p, double* gp) {
  double x = (P[0] - m.off[0]) / m.scale[0];
  double y = (P[1] - m.off[1]) / m.scale[1];
  double z = (P[2] - m.off[2]) / m.scale[2];
  const double* a = m.cglex;
  double r2 = x * x + y * y + z * z;
  double t = 1.0, tx = 0.0, ty = 0.0, tz = 0.0;
  if (r2 > 0.0) {
    t = z * z / r2;
    tx = -2.0 * x * t / r2;
    ty = -2.0 * y * t / r2;
    tz = 2.0 * z * (1.0 - t) / r2;
  }
  double q = 16.0 * t * t - 20.0 * t + 5.0;
  double qt = 32.0 * t - 20.0;
  double g1 = 0.3 * (r2 - 1.0);
  double g2 = z * q;
  double g3 = x * x - y * y;
  p = a[0] + a[1] * g1 + a[2] * g2 + a[3] * g3;
  double gx = a[1] * (0.6 * x) + a[2] * (z * qt * tx) + a[3] * (2.0 * x);
  double gy = a[1] * (0.6 * y) + a[2] * (z * qt * ty) + a[3] * (-2.0 * y);
  double gz = a[1] * (0.6 * z) + a[2] * (q + z * qt * tz);
  gp[0] = gx / m.scale[0];
  gp[1] = gy / m.scale[1];
  gp[2] = gz / m.scale[2];
}

// N2P-GRIN cylinder lens of Sec. VI: n = [1 + u^beta]^gamma with
// u = (R^2 - (rho/2)^2) / F^2, rho measured from the axis through (off[0],
// off[1]); dn/dx = gamma (1 + u^beta)^(gamma - 1) beta u^(beta - 1) (-x / (2 F^2)),
// likewise in y, and dn/dz = 0.
__device__ __forceinline__ void n2p(const DevMedium& m, const double* P, double& p, double* gp) {
  double R = m.cglex[0], F = m.cglex[1], be = m.cglex[2], ga = m.cglex[3];
  double x = P[0] - m.off[0];
  double y = P[1] - m.off[1];
  double u = (R * R - (x * x + y * y) / 4.0) / (F * F);
  double w = 1.0 + pow(u, be);
  p = pow(w, ga);
  double k = ga * pow(w, ga - 1.0) * be * pow(u, be - 1.0) * (-1.0 / (2.0 * F * F));
  gp[0] = k * x;
  gp[1] = k * y;
  gp[2] = 0.0;
}

// n (after layering) and the gradient of the smooth field; lvl = level or -1.
template <int PC, bool GRID, bool LAYERED>
__device__ __forceinline__ void sample(const DevMedium& m, const double* P, double& n, double* g,
                                       int& lvl, double* ucoord = nullptr) {
  double f;
  if (GRID) {
    tricubic(m, P, f, g);
  } else {
    double p, gp[3];
    if constexpr (PC == kSpherical)
      sph(m, P, p, gp);
    else if constexpr (PC == kN2P)
      n2p(m, P, p, gp);
    else
      poly<PC>(m, P, p, gp);
    if (m.form == GRIN_FORM_LINEAR) {
      f = p;
      g[0] = gp[0];
      g[1] = gp[1];
      g[2] = gp[2];
    } else if (m.form == GRIN_FORM_SQRT) {
      double r = sqrt(p);
      f = r;
      g[0] = gp[0] / (2.0 * r);
      g[1] = gp[1] / (2.0 * r);
      g[2] = gp[2] / (2.0 * r);
    } else {
      f = m.form_c / p;
      double q = -m.form_c / (p * p);
      g[0] = q * gp[0];
      g[1] = q * gp[1];
      g[2] = q * gp[2];
    }
  }
  if (LAYERED) {
    double L = (double)m.n_levels;
    double hi = m.lvl_hi;
    double uu = L * (f - m.lvl_lo) / (hi - m.lvl_lo);
    double fl = floor(uu);
    int k;
    if (!(fl >= 0.0)) k = 0;
    else if (fl > L - 1.0) k = m.n_levels - 1;
    else k = (int)fl;
    lvl = k;
    n = m.lvl_lo + ((double)k + 0.5) * (hi - m.lvl_lo) / L;
    if (ucoord) *ucoord = uu;
  } else {
    lvl = -1;
    n = f;
    if (ucoord) *ucoord = 0.5;
  }
}

// Decision margins of a ray (the quantities whose sign decides an integer
// outcome), each the minimum over the trace: [0] distance of |N.I| from its
// critical value at a refraction with mu > 1, [1] |N.I| at gradient steps,
// [2] distance of a step end point to the enclosing surface in steps, [3]
// distance of the level coordinate to the nearest shell boundary.
struct Margins {
  double v[4];
  __device__ __forceinline__ void init() { v[0] = v[1] = v[2] = v[3] = INFINITY; }
  __device__ __forceinline__ void take(int k, double x) { v[k] = x < v[k] ? x : v[k]; }
};

// Distance of the level coordinate u to the nearest shell boundary, the
// integers 1 .. L-1 (u = 0 and u = L decide nothing: the levels clamp).
__device__ __forceinline__ double lmargin(const DevMedium& m, double u) {
  double k = floor(u + 0.5);
  if (k < 1.0) k = 1.0;
  if (k > (double)m.n_levels - 1.0) k = (double)m.n_levels - 1.0;
  return m.n_levels > 1 ? fabs(u - k) : INFINITY;
}

// Distance of a point to the enclosing surface in units of the step h, to
// first order for the curved surfaces.
__device__ __forceinline__ double bmargin(const DevMedium& m, const double* P, double h) {
  const double* b = m.b;
  if (m.bkind == GRIN_BOUNDARY_BOX) {
    double r = INFINITY;
    for (int a = 0; a < 3; ++a) {
      double d1 = fabs(P[a] - b[a]), d2 = fabs(b[3 + a] - P[a]);
      if (d1 < r) r = d1;
      if (d2 < r) r = d2;
    }
    return r / h;
  }
  if (m.bkind == GRIN_BOUNDARY_SPHERE) {
    double r[3] = {P[0] - b[0], P[1] - b[1], P[2] - b[2]};
    return fabs(dot3(r, r) - b[3] * b[3]) / (2.0 * b[3] * h);
  }
  double x = P[0] - b[0], y = P[1] - b[1];
  double r = fabs(x * x + y * y - b[2] * b[2]) / (2.0 * b[2] * h);
  double d1 = fabs(P[2] - b[3]) / h, d2 = fabs(b[4] - P[2]) / h;
  if (d1 < r) r = d1;
  if (d2 < r) r = d2;
  return r;
}

__device__ __forceinline__ bool inside(const DevMedium& m, const double* P) {
  const double* b = m.b;
  if (m.bkind == GRIN_BOUNDARY_BOX)
    return P[0] > b[0] && P[0] < b[3] && P[1] > b[1] && P[1] < b[4] && P[2] > b[2] && P[2] < b[5];
  if (m.bkind == GRIN_BOUNDARY_SPHERE) {
    double r[3] = {P[0] - b[0], P[1] - b[1], P[2] - b[2]};
    return dot3(r, r) < b[3] * b[3];
  }
  double x = P[0] - b[0], y = P[1] - b[1];
  return x * x + y * y < b[2] * b[2] && P[2] > b[3] && P[2] < b[4];
}

__device__ __forceinline__ bool roots(double a, double b, double c, double& t1, double& t2) {
  double disc = b * b - 4.0 * a * c;
  if (disc < 0.0) return false;
  double sq = sqrt(disc);
  double q = b >= 0.0 ? -(b + sq) / 2.0 : (sq - b) / 2.0;
  double r1 = 0.0, r2 = 0.0;
  if (q != 0.0) {
    r1 = q / a;
    r2 = c / q;
  }
  t1 = r1 < r2 ? r1 : r2;
  t2 = r1 < r2 ? r2 : r1;
  return true;
}

__device__ inline bool enter(const DevMedium& m, const double* P0, const double* d, double& t, double* Pb,
                      double* N, int& face) {
  const double* b = m.b;
  if (m.bkind == GRIN_BOUNDARY_BOX) {
    double tn = -INFINITY, tf = INFINITY;
    int axis = -1, hi = 0;
    for (int a = 0; a < 3; ++a) {
      if (d[a] == 0.0) {
        if (!(P0[a] > b[a] && P0[a] < b[3 + a])) return false;
        continue;
      }
      double t1 = (b[a] - P0[a]) / d[a], t2 = (b[3 + a] - P0[a]) / d[a];
      double lo = t1 < t2 ? t1 : t2, up = t1 < t2 ? t2 : t1;
      if (lo > tn) {
        tn = lo;
        axis = a;
        hi = d[a] < 0.0;
      }
      if (up < tf) tf = up;
    }
    if (axis < 0 || !(tn >= 0.0 && tn < tf)) return false;
    t = tn;
    for (int a = 0; a < 3; ++a) Pb[a] = P0[a] + tn * d[a];
    Pb[axis] = hi ? b[3 + axis] : b[axis];
    N[0] = N[1] = N[2] = 0.0;
    N[axis] = hi ? 1.0 : -1.0;
    face = 2 * axis + hi;
    return true;
  }
  if (m.bkind == GRIN_BOUNDARY_SPHERE) {
    double r[3] = {P0[0] - b[0], P0[1] - b[1], P0[2] - b[2]};
    double t1, t2;
    if (!roots(dot3(d, d), 2.0 * dot3(r, d), dot3(r, r) - b[3] * b[3], t1, t2)) return false;
    if (!(t1 >= 0.0)) return false;
    t = t1;
    for (int a = 0; a < 3; ++a) Pb[a] = P0[a] + t1 * d[a];
    N[0] = Pb[0] - b[0];
    N[1] = Pb[1] - b[1];
    N[2] = Pb[2] - b[2];
    normalize3(N);
    face = 0;
    return true;
  }
  double x = P0[0] - b[0], y = P0[1] - b[1];
  double a2 = d[0] * d[0] + d[1] * d[1];
  double s1 = -INFINITY, s2 = INFINITY;
  if (a2 > 0.0) {
    if (!roots(a2, 2.0 * (x * d[0] + y * d[1]), x * x + y * y - b[2] * b[2], s1, s2)) return false;
    if (!(s1 < s2)) return false;
  } else if (!(x * x + y * y < b[2] * b[2])) {
    return false;
  }
  double z1 = -INFINITY, z2 = INFINITY;
  if (d[2] != 0.0) {
    double u1 = (b[3] - P0[2]) / d[2], u2 = (b[4] - P0[2]) / d[2];
    z1 = u1 < u2 ? u1 : u2;
    z2 = u1 < u2 ? u2 : u1;
  } else if (!(P0[2] > b[3] && P0[2] < b[4])) {
    return false;
  }
  bool side = s1 > z1;
  double tn = side ? s1 : z1, tf = s2 < z2 ? s2 : z2;
  if (!(tn >= 0.0 && tn < tf)) return false;
  t = tn;
  for (int a = 0; a < 3; ++a) Pb[a] = P0[a] + tn * d[a];
  if (side) {
    N[0] = Pb[0] - b[0];
    N[1] = Pb[1] - b[1];
    N[2] = 0.0;
    normalize3(N);
    face = 0;
  } else {
    bool top = d[2] < 0.0;
    Pb[2] = top ? b[4] : b[3];
    N[0] = N[1] = 0.0;
    N[2] = top ? 1.0 : -1.0;
    face = top ? 2 : 1;
  }
  return true;
}

__device__ inline void leave(const DevMedium& m, const double* P, const double* Q, double& t, double* Pb,
                      double* N, int& face) {
  const double* b = m.b;
  double D[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
  double best = INFINITY;
  int bf = 0;
  if (m.bkind == GRIN_BOUNDARY_BOX) {
    for (int a = 0; a < 3; ++a) {
      if (Q[a] <= b[a]) {
        double ta = (b[a] - P[a]) / D[a];
        if (ta < best) {
          best = ta;
          bf = 2 * a;
        }
      }
      if (Q[a] >= b[3 + a]) {
        double ta = (b[3 + a] - P[a]) / D[a];
        if (ta < best) {
          best = ta;
          bf = 2 * a + 1;
        }
      }
    }
  } else if (m.bkind == GRIN_BOUNDARY_SPHERE) {
    double r[3] = {P[0] - b[0], P[1] - b[1], P[2] - b[2]};
    double t1 = 0.0, t2 = 0.0;
    roots(dot3(D, D), 2.0 * dot3(r, D), dot3(r, r) - b[3] * b[3], t1, t2);
    best = t2;
  } else {
    double x = P[0] - b[0], y = P[1] - b[1];
    double qx = Q[0] - b[0], qy = Q[1] - b[1];
    if (qx * qx + qy * qy >= b[2] * b[2]) {
      double t1 = 0.0, t2 = 0.0;
      roots(D[0] * D[0] + D[1] * D[1], 2.0 * (x * D[0] + y * D[1]), x * x + y * y - b[2] * b[2], t1,
            t2);
      best = t2;
    }
    if (Q[2] <= b[3]) {
      double ta = (b[3] - P[2]) / D[2];
      if (ta < best) {
        best = ta;
        bf = 1;
      }
    }
    if (Q[2] >= b[4]) {
      double ta = (b[4] - P[2]) / D[2];
      if (ta < best) {
        best = ta;
        bf = 2;
      }
    }
  }
  if (!(best > 0.0)) best = 0.0;
  if (best > 1.0) best = 1.0;
  t = best;
  face = bf;
  for (int a = 0; a < 3; ++a) Pb[a] = P[a] + best * D[a];
  N[0] = N[1] = N[2] = 0.0;
  if (m.bkind == GRIN_BOUNDARY_BOX) {
    int a = bf / 2;
    Pb[a] = (bf & 1) ? b[3 + a] : b[a];
    N[a] = (bf & 1) ? 1.0 : -1.0;
  } else if (m.bkind == GRIN_BOUNDARY_SPHERE) {
    N[0] = Pb[0] - b[0];
    N[1] = Pb[1] - b[1];
    N[2] = Pb[2] - b[2];
    normalize3(N);
  } else if (bf == 0) {
    N[0] = Pb[0] - b[0];
    N[1] = Pb[1] - b[1];
    normalize3(N);
  } else {
    Pb[2] = bf == 2 ? b[4] : b[3];
    N[2] = bf == 2 ? 1.0 : -1.0;
  }
}

// Eq. 8-9 (positive root) or, for D <= 0, the Sec. II (v) reflection;
// d is replaced by the unit result; returns true on reflection.
__device__ __forceinline__ bool snell(double* d, const double* N, double mu,
                                      double* margin = nullptr) {
  double c = dot3(N, d);
  double D = 1.0 - mu * mu * (1.0 - c * c);
  double R[3];
  if (margin) {
    // |N.I| minus its critical value sqrt(1 - 1/mu^2), as D / (mu^2 (|c| + c_crit))
    if (mu > 1.0) {
      double cc = sqrt(1.0 - 1.0 / (mu * mu));
      *margin = fabs(D) / (mu * mu * (fabs(c) + cc));
    } else {
      *margin = INFINITY;
    }
  }
  if (D <= 0.0) {
    for (int a = 0; a < 3; ++a) R[a] = d[a] - 2.0 * c * N[a];
    normalize3(R);
    d[0] = R[0];
    d[1] = R[1];
    d[2] = R[2];
    return true;
  }
  double s = c > 0.0 ? 1.0 : (c < 0.0 ? -1.0 : 0.0);
  double gamma = -mu * c + s * sqrt(D);
  for (int a = 0; a < 3; ++a) R[a] = mu * d[a] + gamma * N[a];
  normalize3(R);
  d[0] = R[0];
  d[1] = R[1];
  d[2] = R[2];
  return false;
}

__device__ __forceinline__ void put(const TraceArgs& a, int64_t r, const double* P, const double* d,
                                    double opl, int exit_id, int steps, int ti, int tb) {
  store_ray(a, r, mk(P[0], P[1], P[2]), mk(d[0], d[1], d[2]), opl, exit_id, steps, ti, tb);
}

}  // namespace plain
}  // namespace grin
