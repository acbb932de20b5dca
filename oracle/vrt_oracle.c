/*
 * vrt_oracle.c -- TEST INFRASTRUCTURE ONLY (see vrt_oracle.h).
 *
 * A plain FP64 transcription of the Vectorial Ray Tracing (VRT) step of
 * Chavez-Islas et al., Sec. II.  Nothing here is blocked, fused or reordered
 * for speed: every step evaluates the medium, picks one of the cases of
 * Sec. II in a fixed order and advances the ray point.  Built with
 * -O2 -ffp-contract=off so that every product and sum is rounded on its own.
 *
 * Readings of the paper taken here (the paper's flowchart figure is missing):
 *   - the ray direction is carried as state; it equals the normalised
 *     difference of successive points (Eq. 6) in exact arithmetic;
 *   - n_prev is the index sampled at the previous point, n_{i-1} = n(P_{i-1})
 *     (Sec. II, after Eq. 3), whatever case that point took; a total internal
 *     reflection steps Delta L_0 / n_{i-1} (Sec. II (v)), every other case
 *     Delta L_0 / n_i, so every full step adds exactly Delta L_0 of optical
 *     path, and a step cut short at the boundary a fraction t adds t Delta L_0;
 *   - case order: boundary crossing, zero or non-finite gradient, tangent
 *     incidence (N.I == 0 exactly), TIR (D <= 0), refraction;
 *   - a boundary crossing ends the step at the exact FP64 intersection with
 *     the enclosing surface (counted as a step); the boundary normal replaces
 *     grad n there (Sec. II (i)) with mu = n_{i-1} / n_ext; on reflection the
 *     boundary point becomes the previous point, with n sampled there;
 *   - the exterior is one straight segment in the homogeneous index n_ext,
 *     not counted as steps; a point exactly on the surface is outside;
 *   - layered shells: n is the centre value of the level of an underlying
 *     smooth field; inside one shell the gradient is taken as zero (case iii),
 *     at a level change the normal is grad of the smooth field;
 *   - every updated direction is renormalised.
 */
#include "vrt_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

enum { EXIT_MISS = -1, EXIT_ENTRY_REFLECT = -2, EXIT_MAXSTEPS = -3, EXIT_INVALID = -4 };

static double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static double norm3(const double* a) { return sqrt(dot3(a, a)); }

static void normalize3(double* a) {
  double l = norm3(a);
  a[0] = a[0] / l;
  a[1] = a[1] / l;
  a[2] = a[2] / l;
}

static int finite3(const double* a) {
  return isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]);
}

static double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r = r * x;
  return r;
}

/* ---------------------------------------------------------------- medium */

/* Polynomial p and its gradient in physical coordinates: a direct sum over
 * the monomials x'^i y'^j z'^k, graded by total degree s = i+j+k, and within
 * one degree ordered by i descending, then j descending. */
static void poly_eval(const orc_medium* m, const double* P, double* p, double* gp) {
  double x = (P[0] - m->off[0]) / m->scale[0];
  double y = (P[1] - m->off[1]) / m->scale[1];
  double z = (P[2] - m->off[2]) / m->scale[2];
  double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  int idx = 0;
  for (int s = 0; s <= m->degree; ++s) {
    for (int i = s; i >= 0; --i) {
      for (int j = s - i; j >= 0; --j) {
        int k = s - i - j;
        double c = m->coeffs[idx++];
        v += c * (ipow(x, i) * ipow(y, j) * ipow(z, k));
        if (i > 0) gx += c * ((double)i * ipow(x, i - 1) * ipow(y, j) * ipow(z, k));
        if (j > 0) gy += c * ((double)j * ipow(x, i) * ipow(y, j - 1) * ipow(z, k));
        if (k > 0) gz += c * ((double)k * ipow(x, i) * ipow(y, j) * ipow(z, k - 1));
      }
    }
  }
  *p = v;
  gp[0] = gx / m->scale[0];
  gp[1] = gy / m->scale[1];
  gp[2] = gz / m->scale[2];
}

/* Spherical freeform field (Sec. V), in the normalised coordinates:
 * p = a0 + a1 G1 + a2 G2 + a3 G3 with G1 = 0.3 (r^2 - 1), G2 = r cos(5 theta)
 * and G3 = r^2 sin^2(theta) cos(2 phi), theta the polar angle from +z' and
 * phi the azimuth.  Written without angles: cos(theta) = z/r and
 * cos(5 theta) = 16 c^5 - 20 c^3 + 5 c (Chebyshev T5) give
 * G2 = z (16 t^2 - 20 t + 5) with t = z^2 / r^2; and
 * r^2 sin^2(theta) cos(2 phi) = (x^2 + y^2)(cos^2 phi - sin^2 phi) = x^2 - y^2.
 * The gradient follows by differentiating these forms (dt/dx = -2 x t / r^2,
 * dt/dy = -2 y t / r^2, dt/dz = 2 z (1 - t) / r^2).  At r = 0 the polar angle
 * is taken as 0 (t = 1, dt = 0). */
static void sph_eval(const orc_medium* m, const double* P, double* p, double* gp) {
  double x = (P[0] - m->off[0]) / m->scale[0];
  double y = (P[1] - m->off[1]) / m->scale[1];
  double z = (P[2] - m->off[2]) / m->scale[2];
  const double* a = m->coeffs;
  double r2 = x * x + y * y + z * z;
  double t = 1.0, tx = 0.0, ty = 0.0, tz = 0.0;
  if (r2 > 0.0) {
    t = z * z / r2;
    tx = -2.0 * x * t / r2;
    ty = -2.0 * y * t / r2;
    tz = 2.0 * z * (1.0 - t) / r2;
  }
  double q = 16.0 * t * t - 20.0 * t + 5.0; /* cos(5 theta) / cos(theta) */
  double qt = 32.0 * t - 20.0;              /* dq/dt */
  double g1 = 0.3 * (r2 - 1.0);
  double g2 = z * q;
  double g3 = x * x - y * y;
  *p = a[0] + a[1] * g1 + a[2] * g2 + a[3] * g3;
  double gx = a[1] * (0.6 * x) + a[2] * (z * qt * tx) + a[3] * (2.0 * x);
  double gy = a[1] * (0.6 * y) + a[2] * (z * qt * ty) + a[3] * (-2.0 * y);
  double gz = a[1] * (0.6 * z) + a[2] * (q + z * qt * tz);
  gp[0] = gx / m->scale[0];
  gp[1] = gy / m->scale[1];
  gp[2] = gz / m->scale[2];
}

/* N2P-GRIN cylindrical lens of Sec. VI: n = [1 + u^beta]^gamma with
 * u = (R^2 - (rho/2)^2) / F^2, rho the distance from the lens axis (the line
 * through off[0], off[1] parallel to z); by the chain rule
 * dn/dx = gamma (1 + u^beta)^(gamma - 1) beta u^(beta - 1) du/dx with
 * du/dx = -x / (2 F^2), likewise in y, and dn/dz = 0. */
static void n2p_eval(const orc_medium* m, const double* P, double* p, double* gp) {
  double R = m->coeffs[0], F = m->coeffs[1], be = m->coeffs[2], ga = m->coeffs[3];
  double x = P[0] - m->off[0];
  double y = P[1] - m->off[1];
  double u = (R * R - (x * x + y * y) / 4.0) / (F * F);
  double w = 1.0 + pow(u, be);
  *p = pow(w, ga);
  double k = ga * pow(w, ga - 1.0) * be * pow(u, be - 1.0) * (-1.0 / (2.0 * F * F));
  gp[0] = k * x;
  gp[1] = k * y;
  gp[2] = 0.0;
}

/* Catmull-Rom cubic convolution weights (Keys 1981, a = -1/2) for the taps at
 * offsets -1, 0, 1, 2 around the cell containing fraction t, and their
 * derivatives with respect to t. */
static void cr_weights(double t, double* w, double* dw) {
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

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Tricubic interpolant of the vertex-centred samples (x fastest) and its
 * analytic gradient; taps beyond the grid repeat the edge sample. */
static void grid_eval(const orc_medium* m, const double* P, double* f, double* gf) {
  int n[3] = {m->nx, m->ny, m->nz};
  int base[3];
  double w[3][4], dw[3][4];
  for (int a = 0; a < 3; ++a) {
    double u = (P[a] - m->origin[a]) / m->spacing[a];
    if (!(u > -2.0)) u = -2.0; /* also catches NaN */
    if (u > (double)n[a] + 1.0) u = (double)n[a] + 1.0;
    double fl = floor(u);
    base[a] = (int)fl;
    cr_weights(u - fl, w[a], dw[a]);
  }
  double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  for (int c = 0; c < 4; ++c) {
    int kk = clampi(base[2] - 1 + c, 0, n[2] - 1);
    for (int b = 0; b < 4; ++b) {
      int jj = clampi(base[1] - 1 + b, 0, n[1] - 1);
      for (int a = 0; a < 4; ++a) {
        int ii = clampi(base[0] - 1 + a, 0, n[0] - 1);
        double s = (double)m->grid[((int64_t)kk * n[1] + jj) * n[0] + ii];
        v += w[0][a] * w[1][b] * w[2][c] * s;
        gx += dw[0][a] * w[1][b] * w[2][c] * s;
        gy += w[0][a] * dw[1][b] * w[2][c] * s;
        gz += w[0][a] * w[1][b] * dw[2][c] * s;
      }
    }
  }
  *f = v;
  gf[0] = gx / m->spacing[0];
  gf[1] = gy / m->spacing[1];
  gf[2] = gz / m->spacing[2];
}

/* The smooth field n(x,y,z) and grad n (before any quantisation). */
static void field_eval(const orc_medium* m, const double* P, double* f, double* g) {
  if (m->kind == 1) {
    grid_eval(m, P, f, g);
    return;
  }
  double p, gp[3];
  if (m->kind == 2)
    sph_eval(m, P, &p, gp);
  else if (m->kind == 3)
    n2p_eval(m, P, &p, gp);
  else
    poly_eval(m, P, &p, gp);
  if (m->form == 0) {
    *f = p;
    g[0] = gp[0];
    g[1] = gp[1];
    g[2] = gp[2];
  } else if (m->form == 1) {
    double n = sqrt(p);
    *f = n;
    g[0] = gp[0] / (2.0 * n);
    g[1] = gp[1] / (2.0 * n);
    g[2] = gp[2] / (2.0 * n);
  } else {
    *f = m->form_c / p;
    double q = -m->form_c / (p * p);
    g[0] = q * gp[0];
    g[1] = q * gp[1];
    g[2] = q * gp[2];
  }
}

/* Layered shells: level k = clamp(floor(L (f - lo) / (hi - lo)), 0, L-1) and
 * index lo + (k + 1/2) (hi - lo) / L.  u returns the unclamped level
 * coordinate for the margin bookkeeping. */
static void level_of(const orc_medium* m, double f, int* k, double* n, double* u) {
  double L = (double)m->n_levels;
  double uu = L * (f - m->level_lo) / (m->level_hi - m->level_lo);
  double fl = floor(uu);
  int kk;
  if (!(fl >= 0.0)) kk = 0;
  else if (fl > L - 1.0) kk = m->n_levels - 1;
  else kk = (int)fl;
  *k = kk;
  *u = uu;
  *n = m->level_lo + ((double)kk + 0.5) * (m->level_hi - m->level_lo) / L;
}

int orc_medium_eval(const orc_medium* m, const double* P, double* n, double* g) {
  double f;
  field_eval(m, P, &f, g);
  if (m->n_levels > 0) {
    int k;
    double u;
    level_of(m, f, &k, n, &u);
  } else {
    *n = f;
  }
  return 0;
}

/* -------------------------------------------------------------- boundary */

static int inside(const orc_medium* m, const double* P) {
  const double* b = m->b;
  if (m->bkind == 0) {
    return P[0] > b[0] && P[0] < b[3] && P[1] > b[1] && P[1] < b[4] && P[2] > b[2] &&
           P[2] < b[5];
  } else if (m->bkind == 1) {
    double r[3] = {P[0] - b[0], P[1] - b[1], P[2] - b[2]};
    return dot3(r, r) < b[3] * b[3];
  } else {
    double x = P[0] - b[0], y = P[1] - b[1];
    return x * x + y * y < b[2] * b[2] && P[2] > b[3] && P[2] < b[4];
  }
}

/* Relative distance of a point to the enclosing surface, in units of the
 * geometric step h. */
static double boundary_margin(const orc_medium* m, const double* P, double h) {
  const double* b = m->b;
  if (m->bkind == 0) {
    double r = INFINITY;
    for (int a = 0; a < 3; ++a) {
      double d1 = fabs(P[a] - b[a]), d2 = fabs(b[3 + a] - P[a]);
      if (d1 < r) r = d1;
      if (d2 < r) r = d2;
    }
    return r / h;
  } else if (m->bkind == 1) {
    double r[3] = {P[0] - b[0], P[1] - b[1], P[2] - b[2]};
    return fabs(dot3(r, r) - b[3] * b[3]) / (2.0 * b[3] * h);
  } else {
    double x = P[0] - b[0], y = P[1] - b[1];
    double r = fabs(x * x + y * y - b[2] * b[2]) / (2.0 * b[2] * h);
    double d1 = fabs(P[2] - b[3]) / h, d2 = fabs(b[4] - P[2]) / h;
    if (d1 < r) r = d1;
    if (d2 < r) r = d2;
    return r;
  }
}

/* Both roots of a t^2 + b t + c = 0 (a > 0) in the cancellation-free form;
 * returns 0 when there is no real root. */
static int quad_roots(double a, double b, double c, double* t1, double* t2) {
  double disc = b * b - 4.0 * a * c;
  if (disc < 0.0) return 0;
  double sq = sqrt(disc);
  double q = b >= 0.0 ? -(b + sq) / 2.0 : (sq - b) / 2.0;
  double r1, r2;
  if (q == 0.0) {
    r1 = 0.0;
    r2 = 0.0;
  } else {
    r1 = q / a;
    r2 = c / q;
  }
  *t1 = r1 < r2 ? r1 : r2;
  *t2 = r1 < r2 ? r2 : r1;
  return 1;
}

/* First intersection of the ray P0 + t d (t >= 0) with the enclosing surface
 * from outside.  Returns 1 on a hit with t, the entry face and the outward
 * unit normal there; the entry point is written to Pb. */
static int enter(const orc_medium* m, const double* P0, const double* d, double* t,
                 double* Pb, double* N, int* face) {
  const double* b = m->b;
  if (m->bkind == 0) {
    double tn = -INFINITY, tf = INFINITY;
    int axis = -1, hi_side = 0;
    for (int a = 0; a < 3; ++a) {
      if (d[a] == 0.0) {
        if (!(P0[a] > b[a] && P0[a] < b[3 + a])) return 0;
        continue;
      }
      double t1 = (b[a] - P0[a]) / d[a], t2 = (b[3 + a] - P0[a]) / d[a];
      double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
      if (lo > tn) {
        tn = lo;
        axis = a;
        hi_side = d[a] < 0.0;
      }
      if (hi < tf) tf = hi;
    }
    if (axis < 0 || !(tn >= 0.0 && tn < tf)) return 0;
    *t = tn;
    for (int a = 0; a < 3; ++a) Pb[a] = P0[a] + tn * d[a];
    Pb[axis] = hi_side ? b[3 + axis] : b[axis];
    N[0] = N[1] = N[2] = 0.0;
    N[axis] = hi_side ? 1.0 : -1.0;
    *face = 2 * axis + hi_side;
    return 1;
  } else if (m->bkind == 1) {
    double r[3] = {P0[0] - b[0], P0[1] - b[1], P0[2] - b[2]};
    double t1, t2;
    if (!quad_roots(dot3(d, d), 2.0 * dot3(r, d), dot3(r, r) - b[3] * b[3], &t1, &t2)) return 0;
    if (!(t1 >= 0.0)) return 0;
    *t = t1;
    for (int a = 0; a < 3; ++a) Pb[a] = P0[a] + t1 * d[a];
    double q[3] = {Pb[0] - b[0], Pb[1] - b[1], Pb[2] - b[2]};
    normalize3(q);
    N[0] = q[0];
    N[1] = q[1];
    N[2] = q[2];
    *face = 0;
    return 1;
  } else {
    double x = P0[0] - b[0], y = P0[1] - b[1];
    double a2 = d[0] * d[0] + d[1] * d[1];
    double s1 = -INFINITY, s2 = INFINITY;
    if (a2 > 0.0) {
      if (!quad_roots(a2, 2.0 * (x * d[0] + y * d[1]), x * x + y * y - b[2] * b[2], &s1, &s2))
        return 0;
      if (!(s1 < s2)) return 0;
    } else if (!(x * x + y * y < b[2] * b[2])) {
      return 0;
    }
    double z1 = -INFINITY, z2 = INFINITY;
    if (d[2] != 0.0) {
      double u1 = (b[3] - P0[2]) / d[2], u2 = (b[4] - P0[2]) / d[2];
      z1 = u1 < u2 ? u1 : u2;
      z2 = u1 < u2 ? u2 : u1;
    } else if (!(P0[2] > b[3] && P0[2] < b[4])) {
      return 0;
    }
    int side = s1 > z1;
    double tn = side ? s1 : z1, tf = s2 < z2 ? s2 : z2;
    if (!(tn >= 0.0 && tn < tf)) return 0;
    *t = tn;
    for (int a = 0; a < 3; ++a) Pb[a] = P0[a] + tn * d[a];
    if (side) {
      N[0] = Pb[0] - b[0];
      N[1] = Pb[1] - b[1];
      N[2] = 0.0;
      normalize3(N);
      *face = 0;
    } else {
      int top = d[2] < 0.0;
      Pb[2] = top ? b[4] : b[3];
      N[0] = N[1] = 0.0;
      N[2] = top ? 1.0 : -1.0;
      *face = top ? 2 : 1;
    }
    return 1;
  }
}

/* Crossing of the segment from P (inside, or on the surface) to Q (outside):
 * the fraction t in [0, 1], the crossing point, the face and the outward
 * unit normal there. */
static void exit_root(const orc_medium* m, const double* P, const double* Q, double* t,
                      double* Pb, double* N, int* face) {
  const double* b = m->b;
  double D[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
  double best = INFINITY;
  int bf = 0;
  if (m->bkind == 0) {
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
  } else if (m->bkind == 1) {
    double r[3] = {P[0] - b[0], P[1] - b[1], P[2] - b[2]};
    double t1, t2;
    quad_roots(dot3(D, D), 2.0 * dot3(r, D), dot3(r, r) - b[3] * b[3], &t1, &t2);
    best = t2;
    bf = 0;
  } else {
    double x = P[0] - b[0], y = P[1] - b[1];
    double qx = Q[0] - b[0], qy = Q[1] - b[1];
    if (qx * qx + qy * qy >= b[2] * b[2]) {
      double t1, t2;
      quad_roots(D[0] * D[0] + D[1] * D[1], 2.0 * (x * D[0] + y * D[1]),
                 x * x + y * y - b[2] * b[2], &t1, &t2);
      best = t2;
      bf = 0;
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
  *t = best;
  *face = bf;
  for (int a = 0; a < 3; ++a) Pb[a] = P[a] + best * D[a];
  N[0] = N[1] = N[2] = 0.0;
  if (m->bkind == 0) {
    int a = bf / 2;
    Pb[a] = (bf & 1) ? b[3 + a] : b[a];
    N[a] = (bf & 1) ? 1.0 : -1.0;
  } else if (m->bkind == 1) {
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

/* ------------------------------------------------------------ local rules */

/* Vectorial Snell law, Eq. 8-9: R = mu I + gamma N with
 * gamma = -mu (N.I) + sgn(N.I) sqrt(D), D = 1 - mu^2 (1 - (N.I)^2), the
 * positive root; for D <= 0 (Sec. II (v)) the reflection I - 2 (I.N) N.
 * Returns 1 on total internal reflection.  R is renormalised. */
static int refract_or_reflect(const double* I, const double* N, double mu, double* R,
                              double* margin) {
  double c = dot3(N, I);
  double D = 1.0 - mu * mu * (1.0 - c * c);
  /* distance of |N.I| from its critical value sqrt(1 - 1/mu^2), i.e.
   * D / (mu^2 (|c| + c_crit)); no critical angle exists for mu <= 1 */
  if (mu > 1.0) {
    double cc = sqrt(1.0 - 1.0 / (mu * mu));
    *margin = fabs(D) / (mu * mu * (fabs(c) + cc));
  } else {
    *margin = INFINITY;
  }
  if (D <= 0.0) {
    for (int a = 0; a < 3; ++a) R[a] = I[a] - 2.0 * c * N[a];
    normalize3(R);
    return 1;
  }
  double s = c > 0.0 ? 1.0 : (c < 0.0 ? -1.0 : 0.0);
  double gamma = -mu * c + s * sqrt(D);
  for (int a = 0; a < 3; ++a) R[a] = mu * I[a] + gamma * N[a];
  normalize3(R);
  return 0;
}

/* Neumaier-compensated running sum. */
typedef struct {
  double s, c;
} nsum;

static void nsum_add(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

static double minf(double a, double b) { return a < b ? a : b; }

/* Distance of the level coordinate u to the nearest shell boundary: the
 * integers 1 .. L-1 (the levels clamp below 0 and above L-1, so u = 0 and
 * u = L decide nothing). */
static double level_margin(const orc_medium* m, double u) {
  double k = floor(u + 0.5);
  if (k < 1.0) k = 1.0;
  if (k > (double)m->n_levels - 1.0) k = (double)m->n_levels - 1.0;
  return m->n_levels > 1 ? fabs(u - k) : INFINITY;
}

typedef struct {
  double P[3], d[3], opl;
  int exit_id, steps, tir_int, tir_bnd;
  double mg[ORC_NM];
} ray_out;

/* Index n_i, gradient and level at P.  For layered media *lvl receives the
 * level and *u the level coordinate; otherwise *lvl = -1. */
static void sample(const orc_medium* m, const double* P, double* n, double* g, int* lvl,
                   double* u) {
  double f;
  field_eval(m, P, &f, g);
  if (m->n_levels > 0) {
    level_of(m, f, lvl, n, u);
  } else {
    *n = f;
    *lvl = -1;
    *u = 0.5;
  }
}

/* Conditioning probe: a deterministic value in [-1, 1) for (seed, ray,
 * step, axis) from the SplitMix64 finaliser (Steele, Lea and Flood 2014). */
static double probe_uniform(uint64_t seed, int64_t ray, int steps, int axis) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(4 * ((uint64_t)ray * 1000003ull +
                                                              (uint64_t)steps) + (uint64_t)axis + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

static void trace_one(const orc_medium* m, const orc_params* prm, int64_t ray, const double* o,
                      const double* d0, ray_out* out, double* path, int64_t cap,
                      int64_t* plen) {
  double P[3] = {o[0], o[1], o[2]}, d[3] = {d0[0], d0[1], d0[2]};
  nsum opl = {0.0, 0.0};
  int64_t np = 0;
  memset(out, 0, sizeof(*out));
  for (int k = 0; k < ORC_NM; ++k) out->mg[k] = INFINITY;
  out->exit_id = EXIT_INVALID;
  for (int a = 0; a < 3; ++a) {
    out->P[a] = o[a];
    out->d[a] = d0[a];
  }
  if (!finite3(P) || !finite3(d) || norm3(d) == 0.0) return;
  normalize3(d);

  double n_prev, g[3], u, Dm; /* n_prev holds n_{i-1} */
  int lvl_prev;
  if (inside(m, P)) {
    sample(m, P, &n_prev, g, &lvl_prev, &u);
  } else {
    double t, Pb[3], NB[3];
    int face;
    if (!enter(m, P, d, &t, Pb, NB, &face)) {
      out->exit_id = EXIT_MISS;
      for (int a = 0; a < 3; ++a) out->d[a] = d[a];
      return;
    }
    nsum_add(&opl, m->n_ext * t);
    for (int a = 0; a < 3; ++a) P[a] = Pb[a];
    double n_b;
    sample(m, P, &n_b, g, &lvl_prev, &u);
    double R[3];
    int tir = refract_or_reflect(d, NB, m->n_ext / n_b, R, &Dm);
    out->mg[ORC_M_CRIT] = minf(out->mg[ORC_M_CRIT], fabs(Dm));
    for (int a = 0; a < 3; ++a) d[a] = R[a];
    if (tir) {
      out->exit_id = EXIT_ENTRY_REFLECT;
      goto done;
    }
    n_prev = n_b;
  }
  if (!(isfinite(n_prev) && n_prev > 0.0)) {
    out->exit_id = EXIT_INVALID;
    goto done;
  }
  if (path && np < cap) {
    for (int a = 0; a < 3; ++a) path[3 * np + a] = P[a];
    ++np;
  }

  double dopl = prm->dopl;
  double h = dopl / n_prev; /* Eq. 3 */
  double Q[3];
  for (int a = 0; a < 3; ++a) Q[a] = P[a] + h * d[a]; /* Eq. 2 */
  int steps = 0;
  out->exit_id = EXIT_MAXSTEPS;
  const int level_root = (prm->flags & ORC_LEVEL_ROOT) && m->n_levels > 0;
  double rem = 1.0; /* fraction of the current step's dL0 still to go */
  int crossings = 0; /* shell crossings in the current step */
  while (steps < prm->max_steps) {
    if (level_root) {
      /* Layered shells with their crossings solved (the discretised media
       * of Sec. I as a stack of isoindicial surfaces).  n is constant inside
       * a shell, so the ray runs straight (Sec. II (iii)) until it meets a
       * shell boundary or the enclosing surface.  At the first point of the
       * segment outside the current shell, found by bisection, it refracts
       * by Eq. 8-9 with the normal of the isoindicial surface, grad f /
       * |grad f| of the smooth field, and mu = n_k / n_k' of the two shells,
       * or is totally reflected (Sec. II (v)), and goes on with the rest of
       * the step's optical path dL0 (rem, a fraction of it) in its new
       * direction.  A step therefore still adds dL0 (Eq. 3); the enclosing
       * surface ends a step as in Sec. II (i).  Q = P + rem h d here. */
      out->mg[ORC_M_BND] = minf(out->mg[ORC_M_BND], boundary_margin(m, Q, h));
      double E[3], tb = 1.0, Pb[3], NB[3];
      int face = 0, leaves = !inside(m, Q);
      if (leaves) {
        exit_root(m, P, Q, &tb, Pb, NB, &face);
        for (int a = 0; a < 3; ++a) E[a] = Pb[a];
      } else {
        for (int a = 0; a < 3; ++a) E[a] = Q[a];
      }
      double nE, gE[3], uE;
      int lE;
      sample(m, E, &nE, gE, &lE, &uE);
      if (lE != lvl_prev && crossings == ORC_MAX_CROSSINGS) {
        /* a ray grazing a curved shell boundary can cross it back and forth
         * at ever shorter intervals: after ORC_MAX_CROSSINGS crossings in
         * one step the rest of the step runs straight and the ray takes the
         * shell it ends in */
        lvl_prev = lE;
        n_prev = nE;
      }
      if (lE != lvl_prev) {
        ++crossings;
        double lo = 0.0, hi = 1.0, X[3], nX, gX[3], uX;
        int lX;
        for (int it = 0; it < 128; ++it) {
          double mid = 0.5 * (lo + hi);
          if (!(mid > lo && mid < hi)) break;
          for (int a = 0; a < 3; ++a) X[a] = P[a] + mid * (E[a] - P[a]);
          sample(m, X, &nX, gX, &lX, &uX);
          if (lX == lvl_prev) lo = mid;
          else hi = mid;
        }
        for (int a = 0; a < 3; ++a) X[a] = P[a] + hi * (E[a] - P[a]);
        sample(m, X, &nX, gX, &lX, &uX);
        if (prm->perturb > 0.0) {
          double gl = norm3(gX);
          for (int a = 0; a < 3; ++a)
            gX[a] += prm->perturb * gl * probe_uniform(prm->seed, ray, steps + 1000000 * crossings, a);
        }
        double used = hi * tb * rem; /* fraction of dL0 up to the crossing */
        nsum_add(&opl, used * dopl);
        rem = rem - used;
        for (int a = 0; a < 3; ++a) P[a] = X[a];
        if (path && np < cap) {
          for (int a = 0; a < 3; ++a) path[3 * np + a] = P[a];
          ++np;
        }
        if (!(isfinite(nX) && nX > 0.0)) {
          out->exit_id = EXIT_INVALID;
          break;
        }
        double gn = norm3(gX);
        if (gn == 0.0 || !isfinite(gn)) {
          /* Sec. II (ii): no normal; straight on into the new shell */
          n_prev = nX;
          lvl_prev = lX;
        } else {
          double N[3] = {gX[0] / gn, gX[1] / gn, gX[2] / gn}, R[3];
          out->mg[ORC_M_TAN] = minf(out->mg[ORC_M_TAN], fabs(dot3(N, d)));
          int tir = refract_or_reflect(d, N, n_prev / nX, R, &Dm);
          out->mg[ORC_M_CRIT] = minf(out->mg[ORC_M_CRIT], fabs(Dm));
          for (int a = 0; a < 3; ++a) d[a] = R[a];
          if (tir) {
            ++out->tir_int;
          } else {
            n_prev = nX;
            lvl_prev = lX;
          }
        }
        h = dopl / n_prev;
        for (int a = 0; a < 3; ++a) Q[a] = P[a] + rem * h * d[a];
        continue;
      }
      crossings = 0;
      if (!leaves) {
        for (int a = 0; a < 3; ++a) P[a] = Q[a];
        nsum_add(&opl, rem * dopl);
        ++steps;
        rem = 1.0;
        if (path && np < cap) {
          for (int a = 0; a < 3; ++a) path[3 * np + a] = P[a];
          ++np;
        }
        h = dopl / n_prev;
        for (int a = 0; a < 3; ++a) Q[a] = P[a] + h * d[a];
        continue;
      }
      /* the rest of the step meets the enclosing surface inside the shell:
       * the boundary event below */
    }
    out->mg[ORC_M_BND] = minf(out->mg[ORC_M_BND], boundary_margin(m, Q, h));
    if (!inside(m, Q)) {
      /* Sec. II (i): the step ends on the enclosing surface, where the
       * surface normal replaces grad n. */
      double t, Pb[3], NB[3], R[3];
      int face;
      exit_root(m, P, Q, &t, Pb, NB, &face);
      nsum_add(&opl, t * rem * dopl);
      ++steps;
      rem = 1.0;
      for (int a = 0; a < 3; ++a) P[a] = Pb[a];
      if (path && np < cap) {
        for (int a = 0; a < 3; ++a) path[3 * np + a] = P[a];
        ++np;
      }
      int tir = refract_or_reflect(d, NB, n_prev / m->n_ext, R, &Dm);
      out->mg[ORC_M_CRIT] = minf(out->mg[ORC_M_CRIT], fabs(Dm));
      for (int a = 0; a < 3; ++a) d[a] = R[a];
      if (tir) {
        ++out->tir_bnd;
        /* Sec. II (v): step Delta L_0 / n_{i-1}; then n(P_b) is the new n_{i-1}. */
        h = dopl / n_prev;
        sample(m, P, &n_prev, g, &lvl_prev, &u);
        if (!(isfinite(n_prev) && n_prev > 0.0)) {
          out->exit_id = EXIT_INVALID;
          break;
        }
        for (int a = 0; a < 3; ++a) Q[a] = P[a] + h * d[a];
        continue;
      }
      out->exit_id = face;
      break;
    }
    double step_v[3], g_prev[3];
    for (int a = 0; a < 3; ++a) {
      step_v[a] = Q[a] - P[a];
      g_prev[a] = g[a];
      P[a] = Q[a];
    }
    nsum_add(&opl, dopl);
    ++steps;
    if (path && np < cap) {
      for (int a = 0; a < 3; ++a) path[3 * np + a] = P[a];
      ++np;
    }

    double n_i;
    int lvl_i;
    sample(m, P, &n_i, g, &lvl_i, &u);
    if (prm->perturb > 0.0) {
      double gl = norm3(g);
      for (int a = 0; a < 3; ++a) g[a] += prm->perturb * gl * probe_uniform(prm->seed, ray, steps, a);
    }
    if (lvl_i >= 0) out->mg[ORC_M_LEVEL] = minf(out->mg[ORC_M_LEVEL], level_margin(m, u));
    if (!(isfinite(n_i) && n_i > 0.0)) {
      out->exit_id = EXIT_INVALID;
      break;
    }
    double gn = norm3(g);
    int homogeneous = (lvl_i >= 0 && lvl_i == lvl_prev) || gn == 0.0 || !isfinite(gn);
    if (homogeneous) {
      /* Sec. II (ii)/(iii): undefined or vanishing gradient, straight step. */
      n_prev = n_i;
      lvl_prev = lvl_i;
      h = dopl / n_i;
    } else {
      double N[3] = {g[0] / gn, g[1] / gn, g[2] / gn}; /* Eq. 5 */
      double c = dot3(N, d);
      double mu = n_prev / n_i;
      if (prm->index_rule == 1 && lvl_i < 0) {
        /* probe: n_i - n_{i-1} by the trapezoid rule on grad n */
        double dn = 0.5 * ((g_prev[0] + g[0]) * step_v[0] + (g_prev[1] + g[1]) * step_v[1] +
                           (g_prev[2] + g[2]) * step_v[2]);
        mu = 1.0 - dn / n_i;
      }
      out->mg[ORC_M_TAN] = minf(out->mg[ORC_M_TAN], fabs(c));
      if (c == 0.0) {
        /* Sec. II (iv): tangential incidence, circular arc of curvature
         * (dn / h) / n_i along N, with dn from one extra index sample. */
        double hi = dopl / n_i;
        double Pn[3] = {P[0] + hi * N[0], P[1] + hi * N[1], P[2] + hi * N[2]};
        double n2, g2[3], u2;
        int l2;
        sample(m, Pn, &n2, g2, &l2, &u2);
        double k = (n2 - n_i) / (2.0 * n_i);
        double w = 1.0 - k * k;
        double a0 = w > 0.0 ? sqrt(w) : 0.0;
        for (int a = 0; a < 3; ++a) d[a] = a0 * d[a] + k * N[a];
        normalize3(d);
        n_prev = n_i;
        lvl_prev = lvl_i;
        h = hi;
      } else {
        double R[3];
        int tir = refract_or_reflect(d, N, mu, R, &Dm);
        out->mg[ORC_M_CRIT] = minf(out->mg[ORC_M_CRIT], fabs(Dm));
        for (int a = 0; a < 3; ++a) d[a] = R[a];
        if (tir) {
          /* Sec. II (v): reflected step of length Delta L_0 / n_{i-1}. */
          ++out->tir_int;
          h = dopl / n_prev;
        } else {
          h = dopl / n_i;
        }
        n_prev = n_i;
        lvl_prev = lvl_i;
      }
    }
    for (int a = 0; a < 3; ++a) Q[a] = P[a] + h * d[a];
  }
  out->steps = steps;
done:
  for (int a = 0; a < 3; ++a) {
    out->P[a] = P[a];
    out->d[a] = d[a];
  }
  out->opl = opl.s + opl.c;
  if (plen) *plen = np;
}

/* ------------------------------------------------------------ batch API */

typedef struct {
  const orc_medium* m;
  const orc_params* p;
  int64_t n;
  const double *o, *d;
  double *P_out, *d_out, *opl, *margins;
  int32_t *exit_id, *steps, *tir_int, *tir_bnd;
  int tid, nt;
} job;

static void store(const job* j, int64_t i, const ray_out* r) {
  for (int a = 0; a < 3; ++a) {
    j->P_out[3 * i + a] = r->P[a];
    j->d_out[3 * i + a] = r->d[a];
  }
  j->opl[i] = r->opl;
  j->exit_id[i] = r->exit_id;
  j->steps[i] = r->steps;
  j->tir_int[i] = r->tir_int;
  j->tir_bnd[i] = r->tir_bnd;
  if (j->margins)
    for (int k = 0; k < ORC_NM; ++k) j->margins[ORC_NM * i + k] = r->mg[k];
}

static void* worker(void* arg) {
  job* j = (job*)arg;
  ray_out r;
  for (int64_t i = j->tid; i < j->n; i += j->nt) {
    trace_one(j->m, j->p, i, j->o + 3 * i, j->d + 3 * i, &r, NULL, 0, NULL);
    store(j, i, &r);
  }
  return NULL;
}

int orc_trace_batch(const orc_medium* m, const orc_params* p, int64_t n, const double* o,
                    const double* d, double* P_out, double* d_out, double* opl,
                    int32_t* exit_id, int32_t* steps, int32_t* tir_int, int32_t* tir_bnd,
                    double* margins, int32_t nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  job jobs[256];
  pthread_t th[256];
  for (int t = 0; t < nthreads; ++t) {
    job j = {m, p, n, o, d, P_out, d_out, opl, margins, exit_id, steps, tir_int, tir_bnd, t,
             nthreads};
    jobs[t] = j;
  }
  if (nthreads == 1) {
    worker(&jobs[0]);
    return 0;
  }
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, worker, &jobs[t]);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  return 0;
}

int orc_trace_path(const orc_medium* m, const orc_params* p, const double* o, const double* d,
                   double* P_out, double* d_out, double* opl, int32_t* exit_id,
                   int32_t* steps, int32_t* tir_int, int32_t* tir_bnd, double* margins,
                   double* path, int64_t cap, int64_t* path_len) {
  ray_out r;
  *path_len = 0;
  trace_one(m, p, 0, o, d, &r, path, cap, path_len);
  job j = {m, p, 1, o, d, P_out, d_out, opl, margins, exit_id, steps, tir_int, tir_bnd, 0, 1};
  store(&j, 0, &r);
  return 0;
}

/* ------------------------------------------------- forward-mode tangents */

/* Hessian of p in physical coordinates and, per monomial, its value phi and
 * gradient gphi at P (the derivatives of n = p and grad n with respect to
 * each coefficient); p and grad p themselves come from poly_eval. */
static void poly_second(const orc_medium* m, const double* P, double H[3][3], double* phi,
                        double (*gphi)[3]) {
  double x[3];
  for (int a = 0; a < 3; ++a) x[a] = (P[a] - m->off[a]) / m->scale[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) H[a][b] = 0.0;
  int idx = 0;
  for (int s = 0; s <= m->degree; ++s) {
    for (int i = s; i >= 0; --i) {
      for (int j = s - i; j >= 0; --j) {
        int e[3] = {i, j, s - i - j};
        double v[3], d1[3], d2[3]; /* x_a^e, its first and second derivatives */
        for (int a = 0; a < 3; ++a) {
          v[a] = ipow(x[a], e[a]);
          d1[a] = e[a] > 0 ? (double)e[a] * ipow(x[a], e[a] - 1) : 0.0;
          d2[a] = e[a] > 1 ? (double)(e[a] * (e[a] - 1)) * ipow(x[a], e[a] - 2) : 0.0;
        }
        phi[idx] = v[0] * v[1] * v[2];
        gphi[idx][0] = d1[0] * v[1] * v[2] / m->scale[0];
        gphi[idx][1] = v[0] * d1[1] * v[2] / m->scale[1];
        gphi[idx][2] = v[0] * v[1] * d1[2] / m->scale[2];
        double c = m->coeffs[idx];
        for (int a = 0; a < 3; ++a) {
          for (int b = 0; b < 3; ++b) {
            double t = 1.0;
            for (int q = 0; q < 3; ++q) {
              if (a == b && q == a) t = t * d2[q];
              else if (q == a || q == b) t = t * d1[q];
              else t = t * v[q];
            }
            H[a][b] += c * t / (m->scale[a] * m->scale[b]);
          }
        }
        ++idx;
      }
    }
  }
}

/* Tangent of refract_or_reflect's unit result R for tangents dI, dN, dmu of
 * its arguments, in the case (refraction, or reflection when tir) that the
 * value took: the chain rule through c = N.I, D, gamma (Eq. 9), R = mu I +
 * gamma N (Eq. 8) or I - 2 c N, and the renormalisation. */
static void refract_tangent(const double* I, const double* N, double mu, int tir,
                            const double* dI, const double* dN, double dmu, double* dR) {
  double c = dot3(N, I);
  double dc = dot3(dN, I) + dot3(N, dI);
  double Rr[3], dRr[3];
  if (tir) {
    for (int a = 0; a < 3; ++a) {
      Rr[a] = I[a] - 2.0 * c * N[a];
      dRr[a] = dI[a] - 2.0 * (dc * N[a] + c * dN[a]);
    }
  } else {
    double D = 1.0 - mu * mu * (1.0 - c * c);
    double dD = -2.0 * mu * dmu * (1.0 - c * c) + 2.0 * mu * mu * c * dc;
    double s = c > 0.0 ? 1.0 : (c < 0.0 ? -1.0 : 0.0);
    double sq = sqrt(D);
    double gamma = -mu * c + s * sq;
    double dgamma = -dmu * c - mu * dc + s * dD / (2.0 * sq);
    for (int a = 0; a < 3; ++a) {
      Rr[a] = mu * I[a] + gamma * N[a];
      dRr[a] = dmu * I[a] + mu * dI[a] + dgamma * N[a] + gamma * dN[a];
    }
  }
  double L = norm3(Rr);
  double R[3] = {Rr[0] / L, Rr[1] / L, Rr[2] / L};
  double p = dot3(R, dRr);
  for (int a = 0; a < 3; ++a) dR[a] = (dRr[a] - R[a] * p) / L;
}

/* Tricubic interpolant: its Hessian in physical coordinates and, for each
 * of the np samples params[] (flat index, x fastest), the derivative of f and
 * grad f with respect to that sample at P.  A sample's weight is the product
 * of its per-axis weights, each summed over the stencil taps that the edge
 * clamp maps onto it. */
static void grid_second(const orc_medium* m, const double* P, int np, const int64_t* params,
                        double H[3][3], double* phi, double (*gphi)[3]) {
  int n[3] = {m->nx, m->ny, m->nz};
  int base[3];
  double w[3][4], dw[3][4], ddw[3][4];
  for (int a = 0; a < 3; ++a) {
    double u = (P[a] - m->origin[a]) / m->spacing[a];
    if (!(u > -2.0)) u = -2.0;
    if (u > (double)n[a] + 1.0) u = (double)n[a] + 1.0;
    double fl = floor(u), t = u - fl;
    base[a] = (int)fl;
    cr_weights(t, w[a], dw[a]);
    ddw[a][0] = -3.0 * t + 2.0; /* second derivatives of the Keys weights */
    ddw[a][1] = 9.0 * t - 5.0;
    ddw[a][2] = -9.0 * t + 4.0;
    ddw[a][3] = 3.0 * t - 1.0;
  }
  double hxx = 0.0, hyy = 0.0, hzz = 0.0, hxy = 0.0, hxz = 0.0, hyz = 0.0;
  for (int c = 0; c < 4; ++c) {
    int kk = clampi(base[2] - 1 + c, 0, n[2] - 1);
    for (int b = 0; b < 4; ++b) {
      int jj = clampi(base[1] - 1 + b, 0, n[1] - 1);
      for (int a = 0; a < 4; ++a) {
        int ii = clampi(base[0] - 1 + a, 0, n[0] - 1);
        double s = (double)m->grid[((int64_t)kk * n[1] + jj) * n[0] + ii];
        hxx += ddw[0][a] * w[1][b] * w[2][c] * s;
        hyy += w[0][a] * ddw[1][b] * w[2][c] * s;
        hzz += w[0][a] * w[1][b] * ddw[2][c] * s;
        hxy += dw[0][a] * dw[1][b] * w[2][c] * s;
        hxz += dw[0][a] * w[1][b] * dw[2][c] * s;
        hyz += w[0][a] * dw[1][b] * dw[2][c] * s;
      }
    }
  }
  const double* sp = m->spacing;
  H[0][0] = hxx / (sp[0] * sp[0]);
  H[1][1] = hyy / (sp[1] * sp[1]);
  H[2][2] = hzz / (sp[2] * sp[2]);
  H[0][1] = H[1][0] = hxy / (sp[0] * sp[1]);
  H[0][2] = H[2][0] = hxz / (sp[0] * sp[2]);
  H[1][2] = H[2][1] = hyz / (sp[1] * sp[2]);
  for (int q = 0; q < np; ++q) {
    int64_t idx = params[q];
    int want[3] = {(int)(idx % n[0]), (int)((idx / n[0]) % n[1]),
                   (int)(idx / ((int64_t)n[0] * n[1]))};
    double W[3], dW[3];
    for (int a = 0; a < 3; ++a) {
      W[a] = 0.0;
      dW[a] = 0.0;
      for (int t = 0; t < 4; ++t) {
        if (clampi(base[a] - 1 + t, 0, n[a] - 1) == want[a]) {
          W[a] += w[a][t];
          dW[a] += dw[a][t];
        }
      }
    }
    phi[q] = W[0] * W[1] * W[2];
    gphi[q][0] = dW[0] * W[1] * W[2] / sp[0];
    gphi[q][1] = W[0] * dW[1] * W[2] / sp[1];
    gphi[q][2] = W[0] * W[1] * dW[2] / sp[2];
  }
}

/* The second-order data of the tangents at P (n and grad n themselves come
 * from sample(), as trace_one takes them): the Hessian of n and, per parameter (all polynomial
 * coefficients, or the grid samples params[]), dn and d(grad n).  For
 * n = sqrt(p): grad n = grad p / 2n, H_n = H_p / 2n - grad p grad p^T / 4n^3,
 * dn = dp / 2n, d grad n = d grad p / 2n - grad p dp / 4n^3.  For n = C / p:
 * grad n = -C grad p / p^2, H_n = -C H_p / p^2 + 2 C grad p grad p^T / p^3,
 * dn = -C dp / p^2, d grad n = -C d grad p / p^2 + 2 C grad p dp / p^3. */

/* The N2P lens (Sec. VI), n = w^gamma, w = 1 + u^beta,
 * u = (R^2 - rho^2 / 4) / F^2, rho from the axis through off[0], off[1]:
 * with du = (-x / 2F^2, -y / 2F^2, 0), dn/du = gamma beta w^(gamma - 1)
 * u^(beta - 1) =: nu and d nu / du = nuu, grad n = nu du and the Hessian
 * nuu du du^T + nu diag(-1 / 2F^2, -1 / 2F^2, 0).  Per parameter (R, F,
 * beta, gamma): dn/dR = nu 2R / F^2, dn/dF = -nu 2u / F,
 * dn/dbeta = gamma w^(gamma - 1) u^beta ln u, dn/dgamma = w^gamma ln w,
 * and grad n moves along du: d grad n/dR = nuu (2R / F^2) du,
 * d grad n/dF = -(2 / F) (u nuu + nu) du, d grad n/dbeta = (d nu/dbeta) du,
 * d grad n/dgamma = (d nu/dgamma) du. */
static void n2p_second(const orc_medium* m, const double* P, double H[3][3], double* phi,
                       double (*gphi)[3]) {
  double R = m->coeffs[0], F = m->coeffs[1], be = m->coeffs[2], ga = m->coeffs[3];
  double x = P[0] - m->off[0], y = P[1] - m->off[1];
  double u = (R * R - (x * x + y * y) / 4.0) / (F * F);
  double ub = pow(u, be), w = 1.0 + ub;
  double nu = ga * be * pow(w, ga - 1.0) * pow(u, be - 1.0);
  double nuu = ga * be * ((ga - 1.0) * be * pow(w, ga - 2.0) * pow(u, 2.0 * be - 2.0) +
                          (be - 1.0) * pow(w, ga - 1.0) * pow(u, be - 2.0));
  double du[3] = {-x / (2.0 * F * F), -y / (2.0 * F * F), 0.0};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) H[a][b] = nuu * du[a] * du[b];
  H[0][0] += -nu / (2.0 * F * F);
  H[1][1] += -nu / (2.0 * F * F);
  /* d nu / dbeta and d nu / dgamma, differentiated term by term */
  double dnu_dbe = ga * pow(w, ga - 1.0) * pow(u, be - 1.0) +
                   ga * be * (ga - 1.0) * pow(w, ga - 2.0) * ub * log(u) * pow(u, be - 1.0) +
                   ga * be * pow(w, ga - 1.0) * pow(u, be - 1.0) * log(u);
  double dnu_dga = be * pow(w, ga - 1.0) * pow(u, be - 1.0) + nu * log(w);
  double dn[4] = {nu * 2.0 * R / (F * F), -nu * 2.0 * u / F, ga * pow(w, ga - 1.0) * ub * log(u),
                  pow(w, ga) * log(w)};
  double c[4] = {nuu * 2.0 * R / (F * F), -(2.0 / F) * (u * nuu + nu), dnu_dbe, dnu_dga};
  for (int j = 0; j < 4; ++j) {
    phi[j] = dn[j];
    for (int a = 0; a < 3; ++a) gphi[j][a] = c[j] * du[a];
  }
}

/* The spherical freeform field (Sec. V) in sph_eval's forms: the Hessian of
 * p = a0 + a1 G1 + a2 G2 + a3 G3 and, per coefficient a_k, dp = G_k and
 * d grad p = grad G_k.  G1 = 0.3 (r^2 - 1) and G3 = x^2 - y^2 have the
 * constant Hessians 0.6 I and diag(2, -2, 0).  For G2 = z q(t), t = z^2 s,
 * s = 1 / r^2, q = 16 t^2 - 20 t + 5: s_ab = 8 x_a x_b s^3 - 2 delta_ab s^2,
 * so t_xx = z^2 (8 x^2 s^3 - 2 s^2), t_xy = 8 x y z^2 s^3,
 * t_xz = 8 x z^3 s^3 - 4 x z s^2, t_zz = 2 s - 10 z^2 s^2 + 8 z^4 s^3 (y as
 * x), and G2_ab = z (q'' t_a t_b + q' t_ab) + q' (t_a [b = z] + t_b [a = z]),
 * q' = 32 t - 20, q'' = 32.  At r = 0 t's derivatives are taken as 0, as
 * sph_eval takes the polar angle there. */
static void sph_second(const orc_medium* m, const double* P, double H[3][3], double* phi,
                       double (*gphi)[3]) {
  double X[3];
  for (int a = 0; a < 3; ++a) X[a] = (P[a] - m->off[a]) / m->scale[a];
  const double* c = m->coeffs;
  double r2 = dot3(X, X);
  double t = 1.0, dt[3] = {0.0, 0.0, 0.0}, ddt[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  double z = X[2];
  if (r2 > 0.0) {
    double s = 1.0 / r2;
    t = z * z * s;
    dt[0] = -2.0 * X[0] * t / r2;
    dt[1] = -2.0 * X[1] * t / r2;
    dt[2] = 2.0 * z * (1.0 - t) / r2;
    for (int a = 0; a < 2; ++a) {
      for (int b = 0; b < 2; ++b)
        ddt[a][b] = z * z * (8.0 * X[a] * X[b] * s * s * s - (a == b ? 2.0 * s * s : 0.0));
      ddt[a][2] = ddt[2][a] = 8.0 * X[a] * z * z * z * s * s * s - 4.0 * X[a] * z * s * s;
    }
    ddt[2][2] = 2.0 * s - 10.0 * z * z * s * s + 8.0 * z * z * z * z * s * s * s;
  }
  double q = 16.0 * t * t - 20.0 * t + 5.0, q1 = 32.0 * t - 20.0, q2 = 32.0;
  double G2H[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      G2H[a][b] = z * (q2 * dt[a] * dt[b] + q1 * ddt[a][b]);
      if (b == 2) G2H[a][b] += q1 * dt[a];
      if (a == 2) G2H[a][b] += q1 * dt[b];
    }
  double G3H[3] = {2.0, -2.0, 0.0};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      H[a][b] = (c[1] * (a == b ? 0.6 : 0.0) + c[2] * G2H[a][b] + c[3] * (a == b ? G3H[a] : 0.0)) /
                (m->scale[a] * m->scale[b]);
  double dG[4][3] = {{0.0, 0.0, 0.0},
                     {0.6 * X[0], 0.6 * X[1], 0.6 * X[2]},
                     {z * q1 * dt[0], z * q1 * dt[1], q + z * q1 * dt[2]},
                     {2.0 * X[0], -2.0 * X[1], 0.0}};
  phi[0] = 1.0;
  phi[1] = 0.3 * (r2 - 1.0);
  phi[2] = z * q;
  phi[3] = X[0] * X[0] - X[1] * X[1];
  for (int k = 0; k < 4; ++k)
    for (int a = 0; a < 3; ++a) gphi[k][a] = dG[k][a] / m->scale[a];
}

static void ref_second(const orc_medium* m, const double* P, int np, const int64_t* params,
                       double H[3][3], double* phi, double (*gphi)[3]) {
  if (m->kind == 1) {
    grid_second(m, P, np, params, H, phi, gphi);
    return;
  }
  if (m->kind == 3) {
    n2p_second(m, P, H, phi, gphi);
    return;
  }
  int nc;
  double p, gp[3];
  if (m->kind == 2) {
    sph_second(m, P, H, phi, gphi);
    nc = 4;
  } else {
    poly_second(m, P, H, phi, gphi);
    nc = (m->degree + 1) * (m->degree + 2) * (m->degree + 3) / 6;
  }
  if (m->form == 0) return;
  if (m->kind == 2) sph_eval(m, P, &p, gp);
  else poly_eval(m, P, &p, gp);
  double a1, a2; /* n' and n'' of the form at p */
  if (m->form == 1) {
    double n = sqrt(p);
    a1 = 1.0 / (2.0 * n);
    a2 = -1.0 / (4.0 * n * n * n);
  } else {
    a1 = -m->form_c / (p * p);
    a2 = 2.0 * m->form_c / (p * p * p);
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) H[a][b] = a1 * H[a][b] + a2 * gp[a] * gp[b];
  for (int j = 0; j < nc; ++j) {
    for (int a = 0; a < 3; ++a) gphi[j][a] = a1 * gphi[j][a] + a2 * gp[a] * phi[j];
    phi[j] = a1 * phi[j];
  }
}

/* n, grad n and the level as trace_one samples them (sample()), with the
 * second-order data of ref_second.  In a layered medium n is a shell's
 * constant index: its derivatives, dn/dtheta and its spatial gradient gd,
 * are zero, while grad f still sets the refraction normal (Sec. I, Eq. 5). */
static void tan_field(const orc_medium* m, const double* P, int nc, const int64_t* params,
                      double* n, double* g, double* gd, int* lvl, double H[3][3], double* phi,
                      double (*gphi)[3]) {
  double u;
  sample(m, P, n, g, lvl, &u);
  ref_second(m, P, nc, params, H, phi, gphi);
  for (int a = 0; a < 3; ++a) gd[a] = m->n_levels > 0 ? 0.0 : g[a];
  if (m->n_levels > 0)
    for (int j = 0; j < nc; ++j) phi[j] = 0.0;
}

/* Per parameter j the tangents carried along a ray. */
typedef struct {
  double P[3], d[3], Q[3], n_prev, h, opl;
} tangent;

/* One ray of a polynomial or spherical freeform medium (n = p, sqrt(p) or
 * C / p), of a grid medium or of the N2P lens, continuous or in
 * point-sampled shells (not the exact level crossings), in a box, sphere or
 * cylinder: trace_one's values and decisions
 * (the same operations, in the same order), with every continuous quantity
 * also carrying its derivative with respect to each of the nc parameters
 * (all polynomial coefficients, or the grid samples params[]).  The entry
 * point does not depend on the parameters; at the exit the crossing fraction
 * carries one (a plane face: t = (b - P_a) / (Q_a - P_a)), and on a curved
 * face so does the normal.
 * Returns 1 when the ray met a case the tangents do not follow (an arc of
 * tangential incidence whose a0 = sqrt(1 - k^2) is clamped, or a crossing
 * fraction clamped to [0, 1]). */
static int tangent_one(const orc_medium* m, const orc_params* prm, const double* o,
                       const double* d0, ray_out* out, int nc, const int64_t* params, tangent* T,
                       double* phi, double (*gphi)[3], double* phi2, double (*gphi2)[3]) {
  double P[3] = {o[0], o[1], o[2]}, d[3] = {d0[0], d0[1], d0[2]};
  nsum opl = {0.0, 0.0};
  int flag = 0;
  memset(out, 0, sizeof(*out));
  memset(T, 0, (size_t)nc * sizeof(tangent));
  out->exit_id = EXIT_INVALID;
  for (int a = 0; a < 3; ++a) {
    out->P[a] = o[a];
    out->d[a] = d0[a];
  }
  if (!finite3(P) || !finite3(d) || norm3(d) == 0.0) return 0;
  normalize3(d);
  const double zero[3] = {0.0, 0.0, 0.0};

  double n_prev, g[3], gd[3], H[3][3];
  int lvl_prev;
  if (inside(m, P)) {
    tan_field(m, P, nc, params, &n_prev, g, gd, &lvl_prev, H, phi, gphi);
    for (int j = 0; j < nc; ++j) T[j].n_prev = phi[j];
  } else {
    double t, Pb[3], NB[3], Dm;
    int face;
    if (!enter(m, P, d, &t, Pb, NB, &face)) {
      out->exit_id = EXIT_MISS;
      for (int a = 0; a < 3; ++a) out->d[a] = d[a];
      return 0;
    }
    nsum_add(&opl, m->n_ext * t);
    for (int a = 0; a < 3; ++a) P[a] = Pb[a];
    double n_b;
    tan_field(m, P, nc, params, &n_b, g, gd, &lvl_prev, H, phi, gphi);
    double R[3];
    double mu = m->n_ext / n_b;
    int tir = refract_or_reflect(d, NB, mu, R, &Dm);
    for (int j = 0; j < nc; ++j) {
      double dmu = -m->n_ext * phi[j] / (n_b * n_b);
      refract_tangent(d, NB, mu, tir, zero, zero, dmu, T[j].d);
      T[j].n_prev = phi[j];
    }
    for (int a = 0; a < 3; ++a) d[a] = R[a];
    if (tir) {
      out->exit_id = EXIT_ENTRY_REFLECT;
      goto done;
    }
    n_prev = n_b;
  }
  if (!(isfinite(n_prev) && n_prev > 0.0)) {
    out->exit_id = EXIT_INVALID;
    goto done;
  }

  double dopl = prm->dopl;
  double h = dopl / n_prev;
  double Q[3];
  for (int a = 0; a < 3; ++a) Q[a] = P[a] + h * d[a];
  for (int j = 0; j < nc; ++j) {
    T[j].h = -dopl * T[j].n_prev / (n_prev * n_prev);
    for (int a = 0; a < 3; ++a) T[j].Q[a] = T[j].P[a] + T[j].h * d[a] + h * T[j].d[a];
  }
  int steps = 0;
  out->exit_id = EXIT_MAXSTEPS;
  while (steps < prm->max_steps) {
    if (!inside(m, Q)) {
      double t, Pb[3], NB[3], R[3], Dm;
      int face;
      exit_root(m, P, Q, &t, Pb, NB, &face);
      /* a plane face (a box face, a cylinder's end) fixes its coordinate ax
       * at bv; a curved face (the sphere, the cylinder's side) is met where
       * its implicit function F(P + t (Q - P)) vanishes, so that
       * dt = -r . (dP + t (dQ - dP)) / r . (Q - P) with r = grad F at P_b,
       * and its unit normal N = r / |r| moves with P_b:
       * dN = (dr - N (N . dr)) / |r|, dr = dP_b (its xy part on the side) */
      int ax = -1;
      double bv = 0.0;
      if (m->bkind == 0) {
        ax = face / 2;
        bv = (face & 1) ? m->b[3 + ax] : m->b[ax];
      } else if (m->bkind == 2 && face != 0) {
        ax = 2;
        bv = face == 2 ? m->b[4] : m->b[3];
      }
      double r[3] = {0.0, 0.0, 0.0}, rn = 1.0, rD = 1.0;
      int clamped;
      if (ax >= 0) {
        double traw = (bv - P[ax]) / (Q[ax] - P[ax]);
        clamped = !(traw > 0.0) || traw > 1.0;
      } else {
        clamped = !(t > 0.0) || !(t < 1.0);
        for (int a = 0; a < 3; ++a) r[a] = Pb[a] - m->b[a];
        if (m->bkind == 2) r[2] = 0.0;
        rn = norm3(r);
        rD = r[0] * (Q[0] - P[0]) + r[1] * (Q[1] - P[1]) + r[2] * (Q[2] - P[2]);
      }
      if (clamped) flag = 1;
      for (int j = 0; j < nc; ++j) {
        double dt;
        if (clamped) {
          dt = 0.0;
        } else if (ax >= 0) {
          double Da = Q[ax] - P[ax], dDa = T[j].Q[ax] - T[j].P[ax];
          dt = (-T[j].P[ax] * Da - (bv - P[ax]) * dDa) / (Da * Da);
        } else {
          double s = 0.0;
          for (int a = 0; a < 3; ++a) s += r[a] * (T[j].P[a] + t * (T[j].Q[a] - T[j].P[a]));
          dt = -s / rD;
        }
        double dPb[3];
        for (int a = 0; a < 3; ++a)
          dPb[a] = T[j].P[a] + dt * (Q[a] - P[a]) + t * (T[j].Q[a] - T[j].P[a]);
        if (ax >= 0) dPb[ax] = 0.0;
        for (int a = 0; a < 3; ++a) T[j].P[a] = dPb[a];
        T[j].opl += dt * dopl;
      }
      nsum_add(&opl, t * dopl);
      ++steps;
      for (int a = 0; a < 3; ++a) P[a] = Pb[a];
      double mu = n_prev / m->n_ext;
      int tir = refract_or_reflect(d, NB, mu, R, &Dm);
      for (int j = 0; j < nc; ++j) {
        double dd[3], dNB[3] = {0.0, 0.0, 0.0};
        if (ax < 0) {
          double dr[3] = {T[j].P[0], T[j].P[1], m->bkind == 2 ? 0.0 : T[j].P[2]};
          double Ndr = dot3(NB, dr);
          for (int a = 0; a < 3; ++a) dNB[a] = (dr[a] - NB[a] * Ndr) / rn;
        }
        refract_tangent(d, NB, mu, tir, T[j].d, dNB, T[j].n_prev / m->n_ext, dd);
        for (int a = 0; a < 3; ++a) T[j].d[a] = dd[a];
      }
      for (int a = 0; a < 3; ++a) d[a] = R[a];
      if (tir) {
        ++out->tir_bnd;
        h = dopl / n_prev;
        for (int j = 0; j < nc; ++j) T[j].h = -dopl * T[j].n_prev / (n_prev * n_prev);
        tan_field(m, P, nc, params, &n_prev, g, gd, &lvl_prev, H, phi, gphi);
        if (!(isfinite(n_prev) && n_prev > 0.0)) {
          out->exit_id = EXIT_INVALID;
          break;
        }
        for (int a = 0; a < 3; ++a) Q[a] = P[a] + h * d[a];
        for (int j = 0; j < nc; ++j) {
          T[j].n_prev = phi[j] + dot3(gd, T[j].P);
          for (int a = 0; a < 3; ++a) T[j].Q[a] = T[j].P[a] + T[j].h * d[a] + h * T[j].d[a];
        }
        continue;
      }
      out->exit_id = face;
      break;
    }
    for (int a = 0; a < 3; ++a) P[a] = Q[a];
    for (int j = 0; j < nc; ++j)
      for (int a = 0; a < 3; ++a) T[j].P[a] = T[j].Q[a];
    nsum_add(&opl, dopl);
    ++steps;

    double n_i;
    int lvl_i;
    tan_field(m, P, nc, params, &n_i, g, gd, &lvl_i, H, phi, gphi);
    if (!(isfinite(n_i) && n_i > 0.0)) {
      out->exit_id = EXIT_INVALID;
      break;
    }
    double gn = norm3(g);
    if ((lvl_i >= 0 && lvl_i == lvl_prev) || gn == 0.0 || !isfinite(gn)) {
      /* a step inside one shell, or no gradient: straight */
      for (int j = 0; j < nc; ++j) {
        double dn_i = phi[j] + dot3(gd, T[j].P);
        T[j].n_prev = dn_i;
        T[j].h = -dopl * dn_i / (n_i * n_i);
      }
      n_prev = n_i;
      h = dopl / n_i;
    } else {
      double N[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
      double c = dot3(N, d);
      double mu = n_prev / n_i;
      if (c == 0.0) {
        /* tangential incidence (Sec. II (iv)): trace_one's arc,
         * d = normalize(a0 d + k N), k = (n(P'') - n_i) / 2 n_i,
         * a0 = sqrt(1 - k^2), P'' = P + hi N, hi = dL0 / n_i, with its
         * tangents: dk = dn'' / 2 n_i - n'' dn_i / 2 n_i^2,
         * dn'' = dn(P'') + grad n(P'') . dP'', dP'' = dP + dhi N + hi dN,
         * da0 = -k dk / a0 (not followed where the clamp a0 = 0 acts) */
        double hi = dopl / n_i;
        double Pn[3] = {P[0] + hi * N[0], P[1] + hi * N[1], P[2] + hi * N[2]};
        double n2, g2[3], g2d[3], H2[3][3];
        int l2;
        tan_field(m, Pn, nc, params, &n2, g2, g2d, &l2, H2, phi2, gphi2);
        double k = (n2 - n_i) / (2.0 * n_i);
        double w = 1.0 - k * k;
        double a0 = w > 0.0 ? sqrt(w) : 0.0;
        if (!(w > 0.0)) flag = 1;
        double Rr[3];
        for (int a = 0; a < 3; ++a) Rr[a] = a0 * d[a] + k * N[a];
        double L = norm3(Rr), R[3] = {Rr[0] / L, Rr[1] / L, Rr[2] / L};
        for (int j = 0; j < nc; ++j) {
          double dn_i = phi[j] + dot3(gd, T[j].P);
          double dg[3], dN[3], dPn[3], dRr[3];
          for (int a = 0; a < 3; ++a)
            dg[a] = gphi[j][a] + H[a][0] * T[j].P[0] + H[a][1] * T[j].P[1] + H[a][2] * T[j].P[2];
          double Ndg = dot3(N, dg);
          for (int a = 0; a < 3; ++a) dN[a] = (dg[a] - N[a] * Ndg) / gn;
          double dhi = -dopl * dn_i / (n_i * n_i);
          for (int a = 0; a < 3; ++a) dPn[a] = T[j].P[a] + dhi * N[a] + hi * dN[a];
          double dn2 = phi2[j] + dot3(g2d, dPn);
          double dk = dn2 / (2.0 * n_i) - n2 * dn_i / (2.0 * n_i * n_i);
          double da0 = w > 0.0 ? -k * dk / a0 : 0.0;
          for (int a = 0; a < 3; ++a) dRr[a] = da0 * d[a] + a0 * T[j].d[a] + dk * N[a] + k * dN[a];
          double pr = dot3(R, dRr);
          for (int a = 0; a < 3; ++a) T[j].d[a] = (dRr[a] - R[a] * pr) / L;
          T[j].h = dhi;
          T[j].n_prev = dn_i;
        }
        for (int a = 0; a < 3; ++a) d[a] = a0 * d[a] + k * N[a];
        normalize3(d);
        n_prev = n_i;
        h = hi;
      } else {
        double R[3], Dm;
        int tir = refract_or_reflect(d, N, mu, R, &Dm);
        for (int j = 0; j < nc; ++j) {
          double dn_i = phi[j] + dot3(gd, T[j].P);
          double dg[3], dN[3], dd[3];
          for (int a = 0; a < 3; ++a)
            dg[a] = gphi[j][a] + H[a][0] * T[j].P[0] + H[a][1] * T[j].P[1] + H[a][2] * T[j].P[2];
          double Ndg = dot3(N, dg);
          for (int a = 0; a < 3; ++a) dN[a] = (dg[a] - N[a] * Ndg) / gn;
          double dmu = T[j].n_prev / n_i - n_prev * dn_i / (n_i * n_i);
          refract_tangent(d, N, mu, tir, T[j].d, dN, dmu, dd);
          for (int a = 0; a < 3; ++a) T[j].d[a] = dd[a];
          T[j].h = tir ? -dopl * T[j].n_prev / (n_prev * n_prev) : -dopl * dn_i / (n_i * n_i);
          T[j].n_prev = dn_i;
        }
        for (int a = 0; a < 3; ++a) d[a] = R[a];
        if (tir) {
          ++out->tir_int;
          h = dopl / n_prev;
        } else {
          h = dopl / n_i;
        }
        n_prev = n_i;
      }
    }
    lvl_prev = lvl_i;
    for (int a = 0; a < 3; ++a) Q[a] = P[a] + h * d[a];
    for (int j = 0; j < nc; ++j)
      for (int a = 0; a < 3; ++a) T[j].Q[a] = T[j].P[a] + T[j].h * d[a] + h * T[j].d[a];
  }
  out->steps = steps;
done:
  for (int a = 0; a < 3; ++a) {
    out->P[a] = P[a];
    out->d[a] = d[a];
  }
  out->opl = opl.s + opl.c;
  return flag;
}

typedef struct {
  const orc_medium* m;
  const orc_params* p;
  int64_t n;
  const double *o, *d;
  double *P_out, *d_out, *opl, *tP, *td, *topl;
  int32_t *exit_id, *steps, *flag;
  const int64_t* params;
  int nc, tid, nt;
} tjob;

static void* tangent_worker(void* arg) {
  tjob* j = (tjob*)arg;
  tangent* T = (tangent*)malloc((size_t)j->nc * sizeof(tangent));
  double* phi = (double*)malloc((size_t)j->nc * sizeof(double));
  double(*gphi)[3] = (double(*)[3])malloc((size_t)j->nc * sizeof(*gphi));
  double* phi2 = (double*)malloc((size_t)j->nc * sizeof(double));
  double(*gphi2)[3] = (double(*)[3])malloc((size_t)j->nc * sizeof(*gphi2));
  ray_out r;
  for (int64_t i = j->tid; i < j->n; i += j->nt) {
    j->flag[i] = tangent_one(j->m, j->p, j->o + 3 * i, j->d + 3 * i, &r, j->nc, j->params, T,
                             phi, gphi, phi2, gphi2);
    for (int a = 0; a < 3; ++a) {
      j->P_out[3 * i + a] = r.P[a];
      j->d_out[3 * i + a] = r.d[a];
    }
    j->opl[i] = r.opl;
    j->exit_id[i] = r.exit_id;
    j->steps[i] = r.steps;
    for (int c = 0; c < j->nc; ++c) {
      for (int a = 0; a < 3; ++a) {
        j->tP[(i * j->nc + c) * 3 + a] = T[c].P[a];
        j->td[(i * j->nc + c) * 3 + a] = T[c].d[a];
      }
      j->topl[i * j->nc + c] = T[c].opl;
    }
  }
  free(T);
  free(phi);
  free(gphi);
  free(phi2);
  free(gphi2);
  return NULL;
}

int orc_trace_tangent(const orc_medium* m, const orc_params* p, int64_t n, const double* o,
                      const double* d, int32_t nparams, const int64_t* params, double* P_out,
                      double* d_out, double* opl, int32_t* exit_id, int32_t* steps, double* tP,
                      double* td, double* topl, int32_t* flag, int32_t nthreads) {
  if (m->bkind < 0 || m->bkind > 2 || (p->flags & ORC_LEVEL_ROOT)) return -1;
  int nc;
  if (m->kind == 0 && m->form >= 0 && m->form <= 2 && m->degree >= 0) {
    nc = (m->degree + 1) * (m->degree + 2) * (m->degree + 3) / 6;
  } else if (m->kind == 3 && m->form == 0) {
    nc = 4; /* R, F, beta, gamma */
  } else if (m->kind == 2 && m->form >= 0 && m->form <= 2) {
    nc = 4; /* a0 .. a3 */
  } else if (m->kind == 1 && nparams > 0 && params) {
    int64_t total = (int64_t)m->nx * m->ny * m->nz;
    for (int q = 0; q < nparams; ++q)
      if (params[q] < 0 || params[q] >= total) return -1;
    nc = nparams;
  } else {
    return -1;
  }
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  tjob jobs[256];
  pthread_t th[256];
  for (int t = 0; t < nthreads; ++t) {
    tjob j = {m, p, n, o, d, P_out, d_out, opl, tP, td, topl, exit_id, steps, flag,
              m->kind == 1 ? params : NULL, nc, t, nthreads};
    jobs[t] = j;
  }
  if (nthreads == 1) {
    tangent_worker(&jobs[0]);
    return 0;
  }
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, tangent_worker, &jobs[t]);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  return 0;
}
