// adjoint.cu -- reverse-mode derivative of the traced exit states with
// respect to the medium parameters (polynomial coefficients of n = p, or grid
// samples), for the direct-design use of VRT (Chavez-Islas et al., Sec. VI).
//
// The derivative is that of the discrete map the plain FP64 tracer computes
// (Sec. II, Eq. 1-9), with every branch decision (refraction, TIR, surface
// crossing, exit) held at the one the forward sweep took.  Forward: the plain
// step (plain_fp64.cuh, this file is built with --fmad=false like
// trace_fp64.cu, so the decisions are the plain tracer's, which are the
// oracle's), saving the ray state (P, I, n_{i-1}, step length) every K
// steps.  Backward: for each K-step segment, last first, the segment is
// recomputed from its checkpoint with the input state of every step kept in
// thread-local memory, then the adjoint state
// (dL/dP, dL/dI, dL/dn_{i-1}, dL/dh) is carried back through each step:
//   normal step   P' = P + h I; n, grad n at P'; N = grad n / |grad n|;
//                 c = N.I; mu = n_{i-1} / n; D = 1 - mu^2 (1 - c^2);
//                 R = mu I + gamma N (gamma = -mu c + sgn(c) sqrt(D)) or, on
//                 TIR, R = I - 2 c N; I' = R / |R|; h' = dL0 / n (TIR:
//                 dL0 / n_{i-1}); n'_{i-1} = n;
//   surface cross fraction t = (b - P_a) / (h I_a) of the step to the face,
//                 P_b = P + t h I; exit refraction with the face normal, or
//                 reflection (the normal component flips) and n'_{i-1} =
//                 n(P_b);
//   entry         the refraction at the entry point through mu = n_ext / n.
// Parameters enter through n, grad n (first and, for dL/dP, second
// derivatives of the interpolant or polynomial) at every point sampled.
// Supported: box boundaries; polynomial media with n = p, or grid media;
// continuous (not layered) fields.
#include "plain_fp64.cuh"

namespace grin {
namespace adj {

constexpr int kMaxK = 64;
// checkpoint words: P[3], I[3], n_{i-1}, h at the start of a step; with a
// checkpoint every step (K = 1) also the step's case and face, kind + 4 face
// (word 8), and n, grad n at the end point of a normal step (words kNg ..
// kNg + 3), which the backward step then takes instead of sampling the field
constexpr int kCk = 13;
constexpr int kNg = 9;
enum Kind : int { kNormal = 0, kCrossReflect = 1, kExit = 2 };

struct St {
  double P[3], d[3], n_prev, h;
  double n_end, g_end[3];  // n and grad n at the last normal step's end point
  int lvl, steps, full, ti, tb, exit_id;
  double frac, opl_ext;
  bool done;
};

// One iteration of the plain tracer's loop (trace_fp64.cu), on St.  A
// normal step leaves n and grad n at its end point in s.n_end and s.g_end.
template <int PC, bool GRID, bool LAY>
__device__ __forceinline__ int advance(const DevMedium& m, double dopl, St& s, int& face) {
  using namespace plain;
  double Q[3];
  for (int k = 0; k < 3; ++k) Q[k] = s.P[k] + s.h * s.d[k];
  double g[3];
  if (!inside(m, Q)) {
    double t, Pb[3], NB[3];
    leave(m, s.P, Q, t, Pb, NB, face);
    s.frac += t;
    ++s.steps;
    for (int k = 0; k < 3; ++k) s.P[k] = Pb[k];
    if (snell(s.d, NB, s.n_prev / m.n_ext)) {
      ++s.tb;
      s.h = dopl / s.n_prev;
      sample<PC, GRID, LAY>(m, s.P, s.n_prev, g, s.lvl);
      if (!(isfinite(s.n_prev) && s.n_prev > 0.0)) {
        s.exit_id = GRIN_EXIT_INVALID;
        s.done = true;
      }
      return kCrossReflect;
    }
    s.exit_id = face;
    s.done = true;
    return kExit;
  }
  for (int k = 0; k < 3; ++k) s.P[k] = Q[k];
  ++s.full;
  ++s.steps;
  double n_i;
  int lvl_i;
  sample<PC, GRID, LAY>(m, s.P, n_i, g, lvl_i);
  s.n_end = n_i;
  s.g_end[0] = g[0];
  s.g_end[1] = g[1];
  s.g_end[2] = g[2];
  if (!(isfinite(n_i) && n_i > 0.0)) {
    s.exit_id = GRIN_EXIT_INVALID;
    s.done = true;
    return kNormal;
  }
  double gn = sqrt(dot3(g, g));
  if ((LAY && lvl_i == s.lvl) || gn == 0.0 || !isfinite(gn)) {
    s.h = dopl / n_i;
  } else {
    double N[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
    double c = dot3(N, s.d);
    if (c == 0.0) {
      double hi = dopl / n_i;
      double Pn[3] = {s.P[0] + hi * N[0], s.P[1] + hi * N[1], s.P[2] + hi * N[2]};
      double n2, g2[3];
      int l2;
      sample<PC, GRID, LAY>(m, Pn, n2, g2, l2);
      double k = (n2 - n_i) / (2.0 * n_i);
      double w = 1.0 - k * k;
      double a0 = w > 0.0 ? sqrt(w) : 0.0;
      for (int q = 0; q < 3; ++q) s.d[q] = a0 * s.d[q] + k * N[q];
      normalize3(s.d);
      s.h = hi;
    } else if (snell(s.d, N, s.n_prev / n_i)) {
      ++s.ti;
      s.h = dopl / s.n_prev;
    } else {
      s.h = dopl / n_i;
    }
  }
  s.n_prev = n_i;
  s.lvl = lvl_i;
  return kNormal;
}

// Start of a ray as in the plain tracer; false if it never steps (miss,
// entry reflection, invalid).  Also returns the entry data the backward
// sweep needs.
template <int PC, bool GRID, bool LAY>
__device__ bool start(const DevMedium& m, const TraceArgs& a, int64_t r, St& s, bool& entered,
                      double* d_in, double* NB) {
  using namespace plain;
  s.P[0] = ld(a.ox, r, a.dtype);
  s.P[1] = ld(a.oy, r, a.dtype);
  s.P[2] = ld(a.oz, r, a.dtype);
  s.d[0] = ld(a.dx, r, a.dtype);
  s.d[1] = ld(a.dy, r, a.dtype);
  s.d[2] = ld(a.dz, r, a.dtype);
  s.steps = s.full = s.ti = s.tb = 0;
  s.frac = 0.0;
  s.opl_ext = 0.0;
  s.done = false;
  s.exit_id = GRIN_EXIT_MAXSTEPS;
  entered = false;
  if (!finite3(s.P) || !finite3(s.d) || sqrt(dot3(s.d, s.d)) == 0.0) {
    s.exit_id = GRIN_EXIT_INVALID;
    return false;
  }
  normalize3(s.d);
  double g[3];
  if (inside(m, s.P)) {
    sample<PC, GRID, LAY>(m, s.P, s.n_prev, g, s.lvl);
  } else {
    double t, Pb[3];
    int face;
    if (!enter(m, s.P, s.d, t, Pb, NB, face)) {
      s.exit_id = GRIN_EXIT_MISS;
      return false;
    }
    entered = true;
    s.opl_ext = m.n_ext * t;
    for (int k = 0; k < 3; ++k) {
      s.P[k] = Pb[k];
      d_in[k] = s.d[k];
    }
    sample<PC, GRID, LAY>(m, s.P, s.n_prev, g, s.lvl);
    if (snell(s.d, NB, m.n_ext / s.n_prev)) {
      s.exit_id = GRIN_EXIT_ENTRY_REFLECT;
      return false;
    }
  }
  if (!(isfinite(s.n_prev) && s.n_prev > 0.0)) {
    s.exit_id = GRIN_EXIT_INVALID;
    return false;
  }
  s.h = a.dopl / s.n_prev;
  return true;
}

// a . b with fused multiply-adds (reverse-mode arithmetic only: the forward
// sweep keeps plain::dot3's unfused rounding)
__device__ __forceinline__ double fdot3(const double* a, const double* b) {
  return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
}

// ------------------------------------------------------ field derivatives

// At P: n, grad n and the Hessian (xx, yy, zz, xy, xz, yz), then, with the
// same weights (grid) or powers (polynomial),
//   theta_bar += nb dn/dtheta + gb . d(grad n)/dtheta
// (polynomial: into the thread's accumulator acc[term]; grid: atomically
// into grad).  gb may be null (zero).  The cell choice takes the forward
// sweep's division; nothing after it feeds a decision, so the rest uses
// explicit fused multiply-adds and products by stored reciprocals.
template <int PC, bool GRID>
__device__ void field_h_adj(const DevMedium& m, const double* P, double nb, const double* gbp,
                            double& n, double* g, double* H, double* acc, double* grad) {
  const double gb[3] = {gbp ? gbp[0] : 0.0, gbp ? gbp[1] : 0.0, gbp ? gbp[2] : 0.0};
  for (int k = 0; k < 3; ++k) g[k] = 0.0;
  for (int k = 0; k < 6; ++k) H[k] = 0.0;
  n = 0.0;
  if constexpr (PC == kN2P) {
    // N2P lens (Sec. VI): n = w^gamma, w = 1 + u^beta, u = (R^2 - rho^2 / 4) / F^2.
    // With n_u = dn/du = gamma beta w^(gamma-1) u^(beta-1) and
    // n_uu = n_u ((gamma - 1) beta u^beta / w + beta - 1) / u: grad n = n_u grad u,
    // H = n_uu grad u grad u^T + n_u diag(-1/2F^2, -1/2F^2, 0).  The parameters
    // theta = (R, F, beta, gamma) move n by dn/dtheta and grad n by
    // c_theta grad u (every grad n derivative lies along grad u).
    const double R = m.cglex[0], F = m.cglex[1], be = m.cglex[2], ga = m.cglex[3];
    const double X = P[0] - m.off[0], Y = P[1] - m.off[1];
    const double iF2 = 1.0 / (F * F);
    const double u = (R * R - (X * X + Y * Y) * 0.25) * iF2;
    const double lu = log(u), A = pow(u, be), w = 1.0 + A, lw = log(w);
    n = pow(w, ga);
    const double n0 = n * A / (w * u);  // n_u / (gamma beta)
    const double nu = ga * be * n0;
    const double nuu = nu * fma((ga - 1.0) * be, A / w, be - 1.0) / u;
    const double ux = -0.5 * X * iF2, uy = -0.5 * Y * iF2, uxx = -0.5 * iF2;
    g[0] = nu * ux;
    g[1] = nu * uy;
    H[0] = fma(nuu * ux, ux, nu * uxx);
    H[1] = fma(nuu * uy, uy, nu * uxx);
    H[3] = nuu * ux * uy;
    const double gbu = fma(gb[0], ux, gb[1] * uy);
    const double dn[4] = {nu * 2.0 * R * iF2, nu * (-2.0 * u / F), ga * n * A * lu / w, n * lw};
    const double c[4] = {nuu * 2.0 * R * iF2, (-2.0 / F) * fma(u, nuu, nu),
                         fma(nu, fma((ga - 1.0) * A, lu / w, lu), ga * n0), fma(nu, lw, be * n0)};
    for (int q = 0; q < 4; ++q) acc[q] += fma(nb, dn[q], gbu * c[q]);
    return;
  }
  if constexpr (PC == kSpherical) {
    // Spherical freeform (Sec. V): p = a0 + a1 G1 + a2 G2 + a3 G3 in the
    // normalised coordinates X, G1 = 0.3 (r^2 - 1), G2 = z q(t) with
    // t = z^2 s, s = 1 / r^2, q = 16 t^2 - 20 t + 5, G3 = x^2 - y^2.  With
    // t_a and t_ab from s_ab = 8 X_a X_b s^3 - 2 delta_ab s^2,
    // G2_ab = z (32 t_a t_b + q' t_ab) + q' (t_a [b = z] + t_b [a = z]); G1 and
    // G3 have the Hessians 0.6 I and diag(2, -2, 0).  dp/da_k = G_k; the form
    // (n = p, sqrt(p), C / p) by the chain rule as for polynomials.
    const double* a = m.cglex;
    double X[3];
    for (int k = 0; k < 3; ++k) X[k] = (P[k] - m.off[k]) * m.inv_scale[k];
    const double z = X[2];
    const double r2 = fdot3(X, X);
    double t = 1.0, dt[3] = {0.0, 0.0, 0.0}, tt[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (r2 > 0.0) {
      const double sv = 1.0 / r2, s2 = sv * sv, s3 = s2 * sv, zz = z * z;
      t = zz * sv;
      dt[0] = -2.0 * X[0] * t * sv;
      dt[1] = -2.0 * X[1] * t * sv;
      dt[2] = 2.0 * z * (1.0 - t) * sv;
      tt[0] = zz * fma(8.0 * X[0] * X[0], s3, -2.0 * s2);
      tt[1] = zz * fma(8.0 * X[1] * X[1], s3, -2.0 * s2);
      tt[2] = fma(8.0 * zz * zz, s3, fma(-10.0 * zz, s2, 2.0 * sv));
      tt[3] = 8.0 * X[0] * X[1] * zz * s3;
      tt[4] = X[0] * z * fma(8.0 * zz, s3, -4.0 * s2);
      tt[5] = X[1] * z * fma(8.0 * zz, s3, -4.0 * s2);
    }
    const double q = fma(fma(16.0, t, -20.0), t, 5.0), q1 = fma(32.0, t, -20.0);
    const int hi[6] = {0, 1, 2, 0, 0, 1}, hj[6] = {0, 1, 2, 1, 2, 2};
    const double* is = m.inv_scale;
    const double G[4] = {1.0, 0.3 * (r2 - 1.0), z * q, fma(X[0], X[0], -X[1] * X[1])};
    double dG[4][3] = {{0.0, 0.0, 0.0},
                       {0.6 * X[0] * is[0], 0.6 * X[1] * is[1], 0.6 * X[2] * is[2]},
                       {z * q1 * dt[0] * is[0], z * q1 * dt[1] * is[1], fma(z * q1, dt[2], q) * is[2]},
                       {2.0 * X[0] * is[0], -2.0 * X[1] * is[1], 0.0}};
    double pv = a[0], gp[3] = {0.0, 0.0, 0.0}, Hp[6];
    for (int k = 1; k < 4; ++k) {
      pv = fma(a[k], G[k], pv);
      for (int c = 0; c < 3; ++c) gp[c] = fma(a[k], dG[k][c], gp[c]);
    }
    for (int e = 0; e < 6; ++e) {
      const int i = hi[e], j = hj[e];
      double h2 = z * fma(32.0 * dt[i], dt[j], q1 * tt[e]);
      if (j == 2) h2 = fma(q1, dt[i], h2);
      if (i == 2) h2 = fma(q1, dt[j], h2);
      const double h1 = i == j ? 0.6 : 0.0, h3 = i == j ? (i == 0 ? 2.0 : (i == 1 ? -2.0 : 0.0)) : 0.0;
      Hp[e] = fma(a[1], h1, fma(a[2], h2, a[3] * h3)) * is[i] * is[j];
    }
    double pb = nb, gscale = 1.0;
    if (m.form == GRIN_FORM_LINEAR) {
      n = pv;
      for (int c = 0; c < 3; ++c) g[c] = gp[c];
      for (int e = 0; e < 6; ++e) H[e] = Hp[e];
    } else if (m.form == GRIN_FORM_SQRT) {
      n = sqrt(pv);
      const double i2n = 0.5 / n, i4n3 = 0.25 / (n * n * n);
      for (int c = 0; c < 3; ++c) g[c] = gp[c] * i2n;
      for (int e = 0; e < 6; ++e) H[e] = fma(Hp[e], i2n, -gp[hi[e]] * gp[hj[e]] * i4n3);
      pb = fma(nb, i2n, -fdot3(gb, gp) * i4n3);
      gscale = i2n;
    } else {
      const double C = m.form_c, ip = 1.0 / pv, cp2 = C * ip * ip, c2p3 = 2.0 * cp2 * ip;
      n = C * ip;
      for (int c = 0; c < 3; ++c) g[c] = -cp2 * gp[c];
      for (int e = 0; e < 6; ++e) H[e] = fma(-cp2, Hp[e], c2p3 * gp[hi[e]] * gp[hj[e]]);
      pb = fma(-cp2, nb, c2p3 * fdot3(gb, gp));
      gscale = -cp2;
    }
    for (int k = 0; k < 4; ++k) acc[k] += fma(pb, G[k], gscale * fdot3(gb, dG[k]));
    return;
  }
  if (GRID) {
    const int nn[3] = {m.nx, m.ny, m.nz};
    int b0[3];
    double w[3][4], dw[3][4], ddw[3][4];
    for (int a = 0; a < 3; ++a) {
      double u = (P[a] - m.origin[a]) / m.spacing[a];
      if (!(u > -2.0)) u = -2.0;
      if (u > (double)nn[a] + 1.0) u = (double)nn[a] + 1.0;
      double fl = floor(u), t = u - fl;
      b0[a] = (int)fl;
      plain::keys(t, w[a], dw[a]);
      ddw[a][0] = fma(-3.0, t, 2.0);
      ddw[a][1] = fma(9.0, t, -5.0);
      ddw[a][2] = fma(-9.0, t, 4.0);
      ddw[a][3] = fma(3.0, t, -1.0);
    }
    // The tensor-product stencil separates: sums along x of the samples
    // weighted by w, w', w'' (per row), then along y, then along z, keeping
    // only the weight combinations of total derivative order <= 2.
    for (int c = 0; c < 4; ++c) {
      int kk = min(max(b0[2] - 1 + c, 0), nn[2] - 1);
      double y00 = 0.0, y10 = 0.0, y20 = 0.0, y01 = 0.0, y11 = 0.0, y02 = 0.0;
      for (int b = 0; b < 4; ++b) {
        int jj = min(max(b0[1] - 1 + b, 0), nn[1] - 1);
        const int64_t row = ((int64_t)kk * nn[1] + jj) * nn[0];
        double x0 = 0.0, x1 = 0.0, x2 = 0.0;  // row sums with w, w', w'' in x
        for (int a = 0; a < 4; ++a) {
          int ii = min(max(b0[0] - 1 + a, 0), nn[0] - 1);
          const double sv = (double)m.grid[GRIN_IDX(m, row + ii, m.grid_n, kSiteGridAdjoint)];
          x0 = fma(w[0][a], sv, x0);
          x1 = fma(dw[0][a], sv, x1);
          x2 = fma(ddw[0][a], sv, x2);
        }
        y00 = fma(w[1][b], x0, y00);
        y10 = fma(w[1][b], x1, y10);
        y20 = fma(w[1][b], x2, y20);
        y01 = fma(dw[1][b], x0, y01);
        y11 = fma(dw[1][b], x1, y11);
        y02 = fma(ddw[1][b], x0, y02);
      }
      n = fma(w[2][c], y00, n);
      g[0] = fma(w[2][c], y10, g[0]);
      g[1] = fma(w[2][c], y01, g[1]);
      g[2] = fma(dw[2][c], y00, g[2]);
      H[0] = fma(w[2][c], y20, H[0]);
      H[1] = fma(w[2][c], y02, H[1]);
      H[2] = fma(ddw[2][c], y00, H[2]);
      H[3] = fma(w[2][c], y11, H[3]);
      H[4] = fma(dw[2][c], y10, H[4]);
      H[5] = fma(dw[2][c], y01, H[5]);
    }
    const double* is = m.inv_spacing;
    for (int k = 0; k < 3; ++k) g[k] *= is[k];
    H[0] *= is[0] * is[0];
    H[1] *= is[1] * is[1];
    H[2] *= is[2] * is[2];
    H[3] *= is[0] * is[1];
    H[4] *= is[0] * is[2];
    H[5] *= is[1] * is[2];
    // d(n, grad n)/d(sample) = the tap's weight products; factored per row
    // (b, c): v = w0 A + w0' B with A = w1 (nb w2 + gb2 w2') + gb1 w1' w2 and
    // B = gb0 w1 w2 (the derivative weights in physical units)
    const double g0 = gb[0] * is[0], g1 = gb[1] * is[1], g2 = gb[2] * is[2];
    for (int c = 0; c < 4; ++c) {
      int kk = min(max(b0[2] - 1 + c, 0), nn[2] - 1);
      const double zc = fma(nb, w[2][c], g2 * dw[2][c]);
      const double g1w2 = g1 * w[2][c], g0w2 = g0 * w[2][c];
      for (int b = 0; b < 4; ++b) {
        int jj = min(max(b0[1] - 1 + b, 0), nn[1] - 1);
        const double A = fma(w[1][b], zc, g1w2 * dw[1][b]);
        const double B = g0w2 * w[1][b];
        const int64_t row = ((int64_t)kk * nn[1] + jj) * nn[0];
        for (int a = 0; a < 4; ++a) {
          int ii = min(max(b0[0] - 1 + a, 0), nn[0] - 1);
          const double v = fma(w[0][a], A, dw[0][a] * B);
          if (v != 0.0) atomicAdd(grad + GRIN_IDX(m, row + ii, m.grid_n, kSiteGridAdjoint), v);
        }
      }
    }
  } else if (m.form == GRIN_FORM_LINEAR) {
    const double* is = m.inv_scale;
    double x[3];
    for (int k = 0; k < 3; ++k) x[k] = (P[k] - m.off[k]) * is[k];
    double pw[3][PC + 1];
    for (int k = 0; k < 3; ++k) {
      pw[k][0] = 1.0;
      for (int e = 1; e <= PC; ++e) pw[k][e] = pw[k][e - 1] * x[k];
    }
    const double gx = gb[0] * is[0], gy = gb[1] * is[1], gz = gb[2] * is[2];
    int idx = 0;
    for (int s = 0; s <= PC; ++s)
      for (int i = s; i >= 0; --i)
        for (int j = s - i; j >= 0; --j) {
          const int k = s - i - j;
          const double X = pw[0][i], Y = pw[1][j], Z = pw[2][k];
          const double dX = i ? i * pw[0][i - 1] : 0.0, dY = j ? j * pw[1][j - 1] : 0.0,
                       dZ = k ? k * pw[2][k - 1] : 0.0;
          const double YZ = Y * Z, XZ = X * Z, XY = X * Y;
          acc[idx] += fma(nb, X * YZ, fma(gx, dX * YZ, fma(gy, dY * XZ, gz * dZ * XY)));
          const double c = m.cglex[idx++];
          if (c == 0.0) continue;
          const double ddX = i > 1 ? i * (i - 1) * pw[0][i - 2] : 0.0;
          const double ddY = j > 1 ? j * (j - 1) * pw[1][j - 2] : 0.0;
          const double ddZ = k > 1 ? k * (k - 1) * pw[2][k - 2] : 0.0;
          n = fma(c, X * YZ, n);
          g[0] = fma(c, dX * YZ, g[0]);
          g[1] = fma(c, dY * XZ, g[1]);
          g[2] = fma(c, dZ * XY, g[2]);
          H[0] = fma(c, ddX * YZ, H[0]);
          H[1] = fma(c, ddY * XZ, H[1]);
          H[2] = fma(c, ddZ * XY, H[2]);
          H[3] = fma(c, dX * dY * Z, H[3]);
          H[4] = fma(c, dX * dZ * Y, H[4]);
          H[5] = fma(c, dY * dZ * X, H[5]);
        }
    for (int k = 0; k < 3; ++k) g[k] *= is[k];
    H[0] *= is[0] * is[0];
    H[1] *= is[1] * is[1];
    H[2] *= is[2] * is[2];
    H[3] *= is[0] * is[1];
    H[4] *= is[0] * is[2];
    H[5] *= is[1] * is[2];
  } else {
    // n = sqrt(p) or n = form_c / p: p, grad p and its Hessian first (the
    // first pass), then n's, and the adjoints of p and grad p that n's value
    // and gradient give (the second pass puts them on the coefficients)
    const double* is = m.inv_scale;
    double x[3];
    for (int k = 0; k < 3; ++k) x[k] = (P[k] - m.off[k]) * is[k];
    double pw[3][PC + 1];
    for (int k = 0; k < 3; ++k) {
      pw[k][0] = 1.0;
      for (int e = 1; e <= PC; ++e) pw[k][e] = pw[k][e - 1] * x[k];
    }
    double p = 0.0, gp[3] = {0.0, 0.0, 0.0}, Hp[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int idx = 0;
    for (int s = 0; s <= PC; ++s)
      for (int i = s; i >= 0; --i)
        for (int j = s - i; j >= 0; --j) {
          const int k = s - i - j;
          const double c = m.cglex[idx++];
          if (c == 0.0) continue;
          const double X = pw[0][i], Y = pw[1][j], Z = pw[2][k];
          const double dX = i ? i * pw[0][i - 1] : 0.0, dY = j ? j * pw[1][j - 1] : 0.0,
                       dZ = k ? k * pw[2][k - 1] : 0.0;
          const double ddX = i > 1 ? i * (i - 1) * pw[0][i - 2] : 0.0;
          const double ddY = j > 1 ? j * (j - 1) * pw[1][j - 2] : 0.0;
          const double ddZ = k > 1 ? k * (k - 1) * pw[2][k - 2] : 0.0;
          const double YZ = Y * Z, XZ = X * Z, XY = X * Y;
          p = fma(c, X * YZ, p);
          gp[0] = fma(c, dX * YZ, gp[0]);
          gp[1] = fma(c, dY * XZ, gp[1]);
          gp[2] = fma(c, dZ * XY, gp[2]);
          Hp[0] = fma(c, ddX * YZ, Hp[0]);
          Hp[1] = fma(c, ddY * XZ, Hp[1]);
          Hp[2] = fma(c, ddZ * XY, Hp[2]);
          Hp[3] = fma(c, dX * dY * Z, Hp[3]);
          Hp[4] = fma(c, dX * dZ * Y, Hp[4]);
          Hp[5] = fma(c, dY * dZ * X, Hp[5]);
        }
    for (int k = 0; k < 3; ++k) gp[k] *= is[k];
    Hp[0] *= is[0] * is[0];
    Hp[1] *= is[1] * is[1];
    Hp[2] *= is[2] * is[2];
    Hp[3] *= is[0] * is[1];
    Hp[4] *= is[0] * is[2];
    Hp[5] *= is[1] * is[2];
    const int hi[6] = {0, 1, 2, 0, 0, 1}, hj[6] = {0, 1, 2, 1, 2, 2};
    const double gbp = fdot3(gb, gp);
    double pb, gscale;  // dL/dp, and dL/d(grad p) = gscale * gb
    if (m.form == GRIN_FORM_SQRT) {
      // n = sqrt(p): grad n = grad p / 2n, H_n = H_p / 2n - grad p grad p^T / 4n^3
      n = sqrt(p);
      const double i2n = 0.5 / n, i4n3 = 0.25 / (n * n * n);
      for (int k = 0; k < 3; ++k) g[k] = gp[k] * i2n;
      for (int q = 0; q < 6; ++q) H[q] = fma(Hp[q], i2n, -gp[hi[q]] * gp[hj[q]] * i4n3);
      pb = fma(nb, i2n, -gbp * i4n3);
      gscale = i2n;
    } else {
      // n = C / p: grad n = -C grad p / p^2, H_n = -C H_p / p^2 + 2 C grad p grad p^T / p^3
      const double C = m.form_c, ip = 1.0 / p, cp2 = C * ip * ip, c2p3 = 2.0 * cp2 * ip;
      n = C * ip;
      for (int k = 0; k < 3; ++k) g[k] = -cp2 * gp[k];
      for (int q = 0; q < 6; ++q) H[q] = fma(-cp2, Hp[q], c2p3 * gp[hi[q]] * gp[hj[q]]);
      pb = fma(-cp2, nb, c2p3 * gbp);
      gscale = -cp2;
    }
    const double gx = gscale * gb[0] * is[0], gy = gscale * gb[1] * is[1],
                 gz = gscale * gb[2] * is[2];
    idx = 0;
    for (int s = 0; s <= PC; ++s)
      for (int i = s; i >= 0; --i)
        for (int j = s - i; j >= 0; --j) {
          const int k = s - i - j;
          const double X = pw[0][i], Y = pw[1][j], Z = pw[2][k];
          const double dX = i ? i * pw[0][i - 1] : 0.0, dY = j ? j * pw[1][j - 1] : 0.0,
                       dZ = k ? k * pw[2][k - 1] : 0.0;
          const double YZ = Y * Z, XZ = X * Z, XY = X * Y;
          acc[idx++] += fma(pb, X * YZ, fma(gx, dX * YZ, fma(gy, dY * XZ, gz * dZ * XY)));
        }
  }
}

// ------------------------------------------------------- adjoint pieces

struct Adj {
  double P[3], d[3], n, h;  // dL/dP, dL/dI, dL/dn_{i-1}, dL/dh
};

// Back through R -> R / |R| given the unit result u and 1 / |R|.
__device__ __forceinline__ void unit_back(const double* u, double inv_Rn, const double* ub, double* Rb) {
  double s = fdot3(u, ub);
  for (int k = 0; k < 3; ++k) Rb[k] = fma(-u[k], s, ub[k]) * inv_Rn;
}

// Back through the Snell refraction R = mu I + gamma N (Eq. 8-9) at fixed
// branch; adds into Ib, Nb and returns mub.
__device__ __forceinline__ double snell_back(const double* I, const double* N, double mu,
                                             const double* Rb, double* Ib, double* Nb) {
  // c, D and gamma exactly as the forward step formed them (unfused): near
  // critical incidence D is tiny, and 1 / sqrt(D) below would amplify any
  // other rounding of it (or take the square root of a negative one)
  double c = plain::dot3(N, I);
  const double omc2 = 1.0 - c * c;
  double D = 1.0 - mu * mu * omc2;
  double s = c > 0.0 ? 1.0 : (c < 0.0 ? -1.0 : 0.0);
  double sq = sqrt(D);
  double gamma = -mu * c + s * sq;
  double mub = fdot3(Rb, I);
  double gammab = fdot3(Rb, N);
  mub = fma(-c, gammab, mub);
  double cb = -mu * gammab;
  double Db = sq > 0.0 ? s * gammab * (0.5 / sq) : 0.0;
  mub = fma(-2.0 * mu * omc2, Db, mub);
  cb = fma(2.0 * mu * mu * c, Db, cb);
  for (int k = 0; k < 3; ++k) {
    Ib[k] = fma(cb, N[k], fma(mu, Rb[k], Ib[k]));
    Nb[k] = fma(cb, I[k], fma(gamma, Rb[k], Nb[k]));
  }
  return mub;
}

// The refracted or reflected unit vector of the forward pass (plain snell
// without the normalisation) and its length.
__device__ __forceinline__ double fwd_R(const double* I, const double* N, double mu, bool tir,
                                        double* R) {
  double c = plain::dot3(N, I);
  if (tir) {
    for (int k = 0; k < 3; ++k) R[k] = I[k] - 2.0 * c * N[k];
  } else {
    double D = 1.0 - mu * mu * (1.0 - c * c);
    double s = c > 0.0 ? 1.0 : (c < 0.0 ? -1.0 : 0.0);
    double gamma = -mu * c + s * sqrt(D);
    for (int k = 0; k < 3; ++k) R[k] = mu * I[k] + gamma * N[k];
  }
  return sqrt(plain::dot3(R, R));
}

// Back through a step that crossed face `face` of the box from state (P, I,
// h): t = (b - P_a) / (Q_a - P_a), P_b = P + t (Q - P), Q = P + h I.  Takes
// dL/dP_b (component a ignored: P_b,a = b) and dL/dt; adds into lam.
__device__ void cross_back(const DevMedium& m, const double* P, const double* I, double h, int face,
                           const double* Pbb, double tb, Adj& lam) {
  const int ax = face >> 1;
  const double b = (face & 1) ? m.b[3 + ax] : m.b[ax];
  double D[3], Db[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < 3; ++k) D[k] = h * I[k];
  const double t = (b - P[ax]) / D[ax];
  for (int k = 0; k < 3; ++k) {
    if (k == ax) continue;
    tb += Pbb[k] * D[k];
    Db[k] += t * Pbb[k];
    lam.P[k] += Pbb[k];
  }
  lam.P[ax] += -tb / D[ax];
  Db[ax] += -tb * t / D[ax];
  for (int k = 0; k < 3; ++k) {
    lam.h += Db[k] * I[k];
    lam.d[k] += h * Db[k];
  }
}

// The surface geometry of a crossing at P_b on face `face`: r, a normal
// direction of the surface's implicit function there (so that r . dP_b = 0
// along the surface), |r|, and for a plane face its axis, whose coordinate
// the forward sweep sets to the plane's exactly (-1 for a curved face, whose
// unit normal N = r / |r| moves with P_b).
struct CrossGeom {
  double r[3];
  double rn;
  int plane_axis;
  bool z_free = false;  // r does not depend on P_b's z (a cylinder side)
};

__device__ __forceinline__ CrossGeom cross_geom(const DevMedium& m, const double* Pb, int face) {
  CrossGeom g;
  const double* b = m.b;
  g.r[0] = g.r[1] = g.r[2] = 0.0;
  g.rn = 1.0;
  if (m.bkind == GRIN_BOUNDARY_BOX) {
    g.plane_axis = face >> 1;
    g.r[g.plane_axis] = (face & 1) ? 1.0 : -1.0;
  } else if (m.bkind == GRIN_BOUNDARY_SPHERE) {
    g.plane_axis = -1;
    for (int k = 0; k < 3; ++k) g.r[k] = Pb[k] - b[k];
    g.rn = sqrt(plain::dot3(g.r, g.r));
  } else if (face == 0) {  // cylinder side
    g.plane_axis = -1;
    g.z_free = true;
    g.r[0] = Pb[0] - b[0];
    g.r[1] = Pb[1] - b[1];
    g.rn = sqrt(g.r[0] * g.r[0] + g.r[1] * g.r[1]);
  } else {  // cylinder end planes
    g.plane_axis = 2;
    g.r[2] = face == 2 ? 1.0 : -1.0;
  }
  return g;
}

// Back through the unit normal N = r / |r| of a curved face: dL/dN into
// dL/dP_b, (1 - N N^T) dL/dN / |r| on the coordinates r depends on.
__device__ __forceinline__ void surface_normal_back(const CrossGeom& g, const double* N,
                                                    const double* Nb, double* Pbb) {
  if (g.plane_axis >= 0) return;
  const double s = fdot3(N, Nb), inv = 1.0 / g.rn;
  for (int k = 0; k < (g.z_free ? 2 : 3); ++k) Pbb[k] = fma(fma(-N[k], s, Nb[k]), inv, Pbb[k]);
}

// Back through a step that crossed the surface at the fraction t of D = h I
// from P (P_b = P + t D, t the root of the surface's implicit function along
// the segment): takes dL/dP_b (a plane face's own coordinate ignored, as the
// forward sweep sets it) and dL/dt; adds into lam.  With r the surface normal
// direction at P_b, dt = -(r . dP + t r . dD) / (r . D).
__device__ void cross_back_general(const double* P, const double* I, double h, double t,
                                   const CrossGeom& g, const double* Pbb, double tb, Adj& lam) {
  double D[3], Db[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < 3; ++k) D[k] = h * I[k];
  for (int k = 0; k < 3; ++k) {
    if (k == g.plane_axis) continue;
    tb = fma(Pbb[k], D[k], tb);
    Db[k] = fma(t, Pbb[k], Db[k]);
    lam.P[k] += Pbb[k];
  }
  const double inv_rD = 1.0 / fdot3(g.r, D);
  for (int k = 0; k < 3; ++k) {
    lam.P[k] = fma(-tb * inv_rD, g.r[k], lam.P[k]);
    Db[k] = fma(-tb * t * inv_rD, g.r[k], Db[k]);
  }
  for (int k = 0; k < 3; ++k) {
    lam.h = fma(Db[k], I[k], lam.h);
    lam.d[k] = fma(h, Db[k], lam.d[k]);
  }
}

// Back through one normal step from its input state rec (P, I, n_{i-1}, h).
// have: n0 and (g0, g1, g2) are n and grad n at the step's end point as the
// forward recompute sampled them (taken by value), else they are sampled
// here with the same arithmetic; either way the branch decisions below are
// the forward sweep's.
template <int PC, bool GRID, bool LAY>
__device__ void normal_back(const DevMedium& m, double dopl, const double* rec, Adj& lam,
                            double* acc, double* grad, bool have = false, double n0 = 0.0,
                            double g0 = 0.0, double g1 = 0.0, double g2 = 0.0) {
  const double* P = rec;
  const double* I = rec + 3;
  const double n_prev = rec[6], h = rec[7];
  double Pn[3];
  for (int k = 0; k < 3; ++k) Pn[k] = P[k] + h * I[k];
  double n, g[3];
  int lvl_i = -1, lvl_prev = -1;
  if (have) {
    n = n0;
    g[0] = g0;
    g[1] = g1;
    g[2] = g2;
  } else {
    plain::sample<PC, GRID, LAY>(m, Pn, n, g, lvl_i);
  }
  if (LAY) {
    // shells: the levels at the step's two ends decide whether it stayed in
    // one (the level of the current point is always the one sampled there)
    double nx, gx[3];
    if (have) plain::sample<PC, GRID, LAY>(m, Pn, nx, gx, lvl_i);
    plain::sample<PC, GRID, LAY>(m, P, nx, gx, lvl_prev);
  }
  double gn = sqrt(plain::dot3(g, g));
  Adj in = lam;  // adjoint of the state after the step
  Adj out;
  for (int k = 0; k < 3; ++k) out.P[k] = out.d[k] = 0.0;
  out.n = out.h = 0.0;
  // a shell's index is a constant: nothing flows into n in a layered medium
  double nb = LAY ? 0.0 : in.n;
  double gb[3] = {0.0, 0.0, 0.0};
  double Pxb[3] = {0.0, 0.0, 0.0};  // dL/dP' through the arc's P'' (tangential incidence)
  const double inv_n = 1.0 / n;
  if (LAY && lvl_i == lvl_prev) {
    // inside one shell: straight, h = dL0 / n_i a constant
    for (int k = 0; k < 3; ++k) out.d[k] += in.d[k];
  } else if (gn == 0.0 || !isfinite(gn)) {
    nb = fma(-in.h * dopl, inv_n * inv_n, nb);
    for (int k = 0; k < 3; ++k) out.d[k] += in.d[k];
  } else {
    // (the decisions take the forward sweep's arithmetic: N, c and D as the
    // plain step forms them; the rest is reverse-mode only)
    double N[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
    double c = plain::dot3(N, I);
    double mu = n_prev / n;
    double Nb[3] = {0.0, 0.0, 0.0};
    if (c == 0.0) {
      // tangential incidence (Sec. II (iv)): the arc's direction
      // R = a0 I + k N, renormalised, with k = (n(P'') - n) / 2n,
      // a0 = sqrt(1 - k^2), P'' = P' + hi N and the step hi = dL0 / n, as the
      // forward sweep forms them; back through n(P''), n, N and I
      const double hi = dopl / n;
      double Pa[3];
      for (int k = 0; k < 3; ++k) Pa[k] = Pn[k] + hi * N[k];
      double n2, g2[3];
      int l2;
      plain::sample<PC, GRID, LAY>(m, Pa, n2, g2, l2);
      const double kk = (n2 - n) / (2.0 * n);
      const double w = 1.0 - kk * kk;
      const double a0 = w > 0.0 ? sqrt(w) : 0.0;
      double R[3];
      for (int k = 0; k < 3; ++k) R[k] = fma(a0, I[k], kk * N[k]);
      const double inv_Rn = 1.0 / sqrt(fdot3(R, R));
      double u[3] = {R[0] * inv_Rn, R[1] * inv_Rn, R[2] * inv_Rn};
      double Rb[3];
      unit_back(u, inv_Rn, in.d, Rb);
      const double a0b = fdot3(Rb, I);
      double kb = fdot3(Rb, N);
      if (w > 0.0) kb = fma(-a0b, kk / a0, kb);
      for (int k = 0; k < 3; ++k) {
        out.d[k] = fma(a0, Rb[k], out.d[k]);
        Nb[k] = kk * Rb[k];
      }
      // k = (n2 - n) / 2n; n2 = n(P''): its parameters, dL/dP'' = n2b grad n(P'')
      if (!LAY) {  // (in shells k is a constant: n, n'' and hi are levels' indices)
        const double n2b = kb * (0.5 * inv_n);
        nb = fma(-kb * n2 * 0.5, inv_n * inv_n, nb);
        double nh2, gh2[3], H2[6];
        field_h_adj<PC, GRID>(m, Pa, n2b, nullptr, nh2, gh2, H2, acc, grad);
        double hib = in.h;  // the next step's length is hi
        for (int k = 0; k < 3; ++k) {
          const double pab = n2b * gh2[k];
          Pxb[k] += pab;
          hib = fma(pab, N[k], hib);
          Nb[k] = fma(hi, pab, Nb[k]);
        }
        nb = fma(-hib * dopl, inv_n * inv_n, nb);
      }
    } else {
      double D = 1.0 - mu * mu * (1.0 - c * c);
      bool tir = D <= 0.0;
      double R[3];
      const double inv_Rn = 1.0 / fwd_R(I, N, mu, tir, R);
      double u[3] = {R[0] * inv_Rn, R[1] * inv_Rn, R[2] * inv_Rn};
      double Rb[3];
      unit_back(u, inv_Rn, in.d, Rb);
      if (tir) {
        const double inv_p = 1.0 / n_prev;
        out.n = fma(-in.h * dopl, inv_p * inv_p, out.n);
        double cb = -2.0 * fdot3(Rb, N);
        for (int k = 0; k < 3; ++k) {
          out.d[k] += fma(cb, N[k], Rb[k]);
          Nb[k] += fma(-2.0 * c, Rb[k], cb * I[k]);
        }
      } else {
        nb = fma(-in.h * dopl, inv_n * inv_n, nb);
        double mub = snell_back(I, N, mu, Rb, out.d, Nb);
        out.n = fma(mub, inv_n, out.n);
        nb = fma(-mub * mu, inv_n, nb);
      }
    }
    double s = fdot3(N, Nb);
    const double inv_gn = 1.0 / gn;
    for (int k = 0; k < 3; ++k) gb[k] = fma(-N[k], s, Nb[k]) * inv_gn;
  }
  // field at P': dL/dP' = in.P + nb grad n + H gb (+ the arc's P''); parameters
  if (LAY) nb = 0.0;
  double nh, gh[3], H[6];
  field_h_adj<PC, GRID>(m, Pn, nb, gb, nh, gh, H, acc, grad);
  double Pb[3];
  Pb[0] = fma(H[4], gb[2], fma(H[3], gb[1], fma(H[0], gb[0], fma(nb, gh[0], in.P[0] + Pxb[0]))));
  Pb[1] = fma(H[5], gb[2], fma(H[1], gb[1], fma(H[3], gb[0], fma(nb, gh[1], in.P[1] + Pxb[1]))));
  Pb[2] = fma(H[2], gb[2], fma(H[5], gb[1], fma(H[4], gb[0], fma(nb, gh[2], in.P[2] + Pxb[2]))));
  // P' = P + h I
  for (int k = 0; k < 3; ++k) {
    out.P[k] += Pb[k];
    out.h = fma(Pb[k], I[k], out.h);
    out.d[k] = fma(h, Pb[k], out.d[k]);
  }
  lam = out;
}

// Back through a surface crossing with boundary reflection.
template <int PC, bool GRID, bool LAY>
__device__ void reflect_back(const DevMedium& m, double dopl, const double* rec, int face,
                             double fb, Adj& lam, double* acc, double* grad) {
  const double* P = rec;
  const double* I = rec + 3;
  const double n_prev = rec[6], h = rec[7];
  double Q[3], t, Pb[3], NB[3];
  int f2;
  for (int k = 0; k < 3; ++k) Q[k] = P[k] + h * I[k];
  plain::leave(m, P, Q, t, Pb, NB, f2);
  // R = I - 2 (I.N) N, as the forward reflection forms it
  const double cI = plain::dot3(NB, I);
  double R[3];
  for (int k = 0; k < 3; ++k) R[k] = I[k] - 2.0 * cI * NB[k];
  const double inv_Rn = 1.0 / sqrt(plain::dot3(R, R));
  double u[3] = {R[0] * inv_Rn, R[1] * inv_Rn, R[2] * inv_Rn};
  Adj in = lam;
  Adj out;
  for (int k = 0; k < 3; ++k) out.P[k] = out.d[k] = 0.0;
  const double inv_p = 1.0 / n_prev;
  out.n = -in.h * dopl * inv_p * inv_p;
  out.h = 0.0;
  // n'_{i-1} = n(P_b)
  double nh, gh[3], H[6];
  const double nbb = LAY ? 0.0 : in.n;  // (a shell's index: a constant)
  field_h_adj<PC, GRID>(m, Pb, nbb, nullptr, nh, gh, H, acc, grad);
  double Pbb[3];
  for (int k = 0; k < 3; ++k) Pbb[k] = fma(nbb, gh[k], in.P[k]);
  double Rb[3];
  unit_back(u, inv_Rn, in.d, Rb);
  // dR = (1 - 2 N N^T) dI - 2 ((I.N) dN + N (I . dN))
  const double rN = fdot3(Rb, NB);
  double Nb[3];
  for (int k = 0; k < 3; ++k) {
    out.d[k] += fma(-2.0 * rN, NB[k], Rb[k]);
    Nb[k] = -2.0 * fma(cI, Rb[k], rN * I[k]);
  }
  if (m.bkind == GRIN_BOUNDARY_BOX) {
    cross_back(m, P, I, h, face, Pbb, fb, out);
  } else {
    const CrossGeom g = cross_geom(m, Pb, face);
    surface_normal_back(g, NB, Nb, Pbb);
    cross_back_general(P, I, h, t, g, Pbb, fb, out);
  }
  lam = out;
}

// Back through the exit step from the seeds (dL/dP_exit, dL/dI_exit).
__device__ void exit_back(const DevMedium& m, const double* rec, int face, const double* Pob,
                          const double* dob, double fb, Adj& lam) {
  const double* P = rec;
  const double* I = rec + 3;
  const double n_prev = rec[6], h = rec[7];
  double N[3] = {0.0, 0.0, 0.0}, t = 0.0, Pb[3];
  if (m.bkind == GRIN_BOUNDARY_BOX) {
    const int ax = face >> 1;
    N[ax] = (face & 1) ? 1.0 : -1.0;
  } else {
    double Q[3];
    int f2;
    for (int k = 0; k < 3; ++k) Q[k] = P[k] + h * I[k];
    plain::leave(m, P, Q, t, Pb, N, f2);
  }
  const double mu = n_prev / m.n_ext;
  double R[3];
  const double inv_Rn = 1.0 / fwd_R(I, N, mu, false, R);
  double u[3] = {R[0] * inv_Rn, R[1] * inv_Rn, R[2] * inv_Rn};
  double Rb[3];
  unit_back(u, inv_Rn, dob, Rb);
  for (int k = 0; k < 3; ++k) lam.P[k] = lam.d[k] = 0.0;
  lam.h = 0.0;
  double Nb[3] = {0.0, 0.0, 0.0};
  double mub = snell_back(I, N, mu, Rb, lam.d, Nb);
  lam.n = mub / m.n_ext;
  if (m.bkind == GRIN_BOUNDARY_BOX) {
    cross_back(m, P, I, h, face, Pob, fb, lam);
  } else {
    // the exit normal moves with the exit point
    const CrossGeom g = cross_geom(m, Pb, face);
    double Pbb[3] = {Pob[0], Pob[1], Pob[2]};
    surface_normal_back(g, N, Nb, Pbb);
    cross_back_general(P, I, h, t, g, Pbb, fb, lam);
  }
}

// Back through the ray's start: the entry refraction (mu = n_ext / n(P_b))
// or, for a ray starting inside, n(P_0).
template <int PC, bool GRID, bool LAY>
__device__ void entry_back(const DevMedium& m, double dopl, const St& s0, bool entered,
                           const double* d_in, const double* NB, const Adj& lam, double* acc,
                           double* grad) {
  const double n0 = s0.n_prev;
  double nb = lam.n - lam.h * (dopl / n0) / n0;
  if (entered) {
    double mu = m.n_ext / n0;
    double R[3];
    const double inv_Rn = 1.0 / fwd_R(d_in, NB, mu, false, R);
    double u[3] = {R[0] * inv_Rn, R[1] * inv_Rn, R[2] * inv_Rn};
    double Rb[3], Ib[3] = {0.0, 0.0, 0.0}, Nb[3] = {0.0, 0.0, 0.0};
    unit_back(u, inv_Rn, lam.d, Rb);
    double mub = snell_back(d_in, NB, mu, Rb, Ib, Nb);
    nb += -mub * mu / n0;
  }
  double nh, gh[3], H[6];
  if (LAY) nb = 0.0;  // the entry shell's index is a constant
  field_h_adj<PC, GRID>(m, s0.P, nb, nullptr, nh, gh, H, acc, grad);
}

// ---------------------------------------------------------------- kernels

struct AdjArgs {
  TraceArgs a;       // rays in; outputs of the forward sweep
  double* ckpt;      // [ray][segment][kCk]
  int32_t* meta;     // [ray][2]: exit id, steps
  int k, nseg;       // checkpoint interval, segments per ray
  const double *gpx, *gpy, *gpz, *gdx, *gdy, *gdz, *gopl;  // dL/d(outputs)
  double* grad;      // dL/d(parameters), accumulated
  int nterms;
  void* order_ws = nullptr;         // scratch of the backward order (or nullptr)
  const uint32_t* order = nullptr;  // backward sweep: thread t takes ray order[t]
};

template <int PC, bool GRID, bool LAY>
__global__ void __launch_bounds__(128) k_adj_forward(DevMedium m, AdjArgs A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.a.count) return;
  St s;
  bool entered;
  double d_in[3], NB[3];
  bool live = start<PC, GRID, LAY>(m, A.a, r, s, entered, d_in, NB);
  double* ck = A.ckpt + (size_t)r * A.nseg * kCk;
  if (live) {
    int face = 0;
    while (!s.done && s.steps < A.a.max_steps) {
      double* c = nullptr;
      if (s.steps % A.k == 0) {
        c = ck + (size_t)(s.steps / A.k) * kCk;
        for (int q = 0; q < 3; ++q) {
          c[q] = s.P[q];
          c[3 + q] = s.d[q];
        }
        c[6] = s.n_prev;
        c[7] = s.h;
      }
      const int kind = advance<PC, GRID, LAY>(m, A.a.dopl, s, face);
      if (A.k == 1) {
        c[8] = (double)(kind + 4 * face);
        c[kNg] = s.n_end;
        c[kNg + 1] = s.g_end[0];
        c[kNg + 2] = s.g_end[1];
        c[kNg + 3] = s.g_end[2];
      }
    }
  }
  double opl = s.opl_ext + A.a.dopl * (double)s.full + A.a.dopl * s.frac;
  plain::put(A.a, r, s.P, s.d, opl, s.exit_id, s.steps, s.ti, s.tb);
  A.meta[2 * r] = s.exit_id;
  A.meta[2 * r + 1] = s.steps;
}

template <int PC, bool GRID, bool LAY>
__global__ void __launch_bounds__(128) k_adj_backward(DevMedium m, AdjArgs A) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.a.count) return;
  const int64_t r = A.order ? (int64_t)A.order[t] : t;
  const int exit_id = A.meta[2 * r], nsteps = A.meta[2 * r + 1];
  if (exit_id == GRIN_EXIT_INVALID || exit_id == GRIN_EXIT_MISS ||
      exit_id == GRIN_EXIT_ENTRY_REFLECT)
    return;
  const double dopl = A.a.dopl;
  double acc[GRID ? 1 : kMaxTerms];
  if (!GRID)
    for (int q = 0; q < A.nterms; ++q) acc[q] = 0.0;
  const double Pob[3] = {A.gpx[r], A.gpy[r], A.gpz[r]};
  const double dob[3] = {A.gdx[r], A.gdy[r], A.gdz[r]};
  const double fb = dopl * A.gopl[r];  // dL/d(sum of cut fractions)
  Adj lam;
  for (int q = 0; q < 3; ++q) {
    lam.P[q] = Pob[q];
    lam.d[q] = dob[q];
  }
  lam.n = lam.h = 0.0;
  const double* ck = A.ckpt + (size_t)r * A.nseg * kCk;
  // each recomputed step's start state and n, grad n at its end point, in
  // the checkpoint's word layout
  double rec[kMaxK][kCk];
  int kind[kMaxK], fc[kMaxK];
  if (nsteps > 0 && A.k == 1) {
    // every step's start state, case and face were stored: no recompute
    for (int i = nsteps - 1; i >= 0; --i) {
      const double* c = ck + (size_t)i * kCk;
      const int code = (int)c[8], kd = code & 3, face = code >> 2;
      if (i == nsteps - 1 && exit_id >= 0)
        exit_back(m, c, face, Pob, dob, fb, lam);
      else if (kd == kCrossReflect)
        reflect_back<PC, GRID, LAY>(m, dopl, c, face, fb, lam, acc, A.grad);
      else
        normal_back<PC, GRID, LAY>(m, dopl, c, lam, acc, A.grad, true, c[kNg], c[kNg + 1], c[kNg + 2],
                              c[kNg + 3]);
    }
  } else if (nsteps > 0) {
    const int last = (nsteps - 1) / A.k;
    for (int seg = last; seg >= 0; --seg) {
      const int s0 = seg * A.k, s1 = min(s0 + A.k, nsteps);
      St s;
      const double* c = ck + (size_t)seg * kCk;
      for (int q = 0; q < 3; ++q) {
        s.P[q] = c[q];
        s.d[q] = c[3 + q];
      }
      s.n_prev = c[6];
      s.h = c[7];
      s.steps = s0;
      s.full = s.ti = s.tb = 0;
      s.frac = 0.0;
      s.done = false;
      s.lvl = 0;
      if (LAY) {  // the current point's level, as the forward sweep sampled it there
        double nx, gx[3];
        plain::sample<PC, GRID, LAY>(m, s.P, nx, gx, s.lvl);
      }
      for (int i = s0; i < s1; ++i) {
        double* rr = rec[i - s0];
        for (int q = 0; q < 3; ++q) {
          rr[q] = s.P[q];
          rr[3 + q] = s.d[q];
        }
        rr[6] = s.n_prev;
        rr[7] = s.h;
        int face = 0;
        kind[i - s0] = advance<PC, GRID, LAY>(m, dopl, s, face);
        fc[i - s0] = face;
        rr[kNg] = s.n_end;
        rr[kNg + 1] = s.g_end[0];
        rr[kNg + 2] = s.g_end[1];
        rr[kNg + 3] = s.g_end[2];
      }
      int i = s1 - 1;
      if (seg == last && exit_id >= 0) {
        exit_back(m, rec[i - s0], fc[i - s0], Pob, dob, fb, lam);
        --i;
      }
      for (; i >= s0; --i) {
        if (kind[i - s0] == kCrossReflect)
          reflect_back<PC, GRID, LAY>(m, dopl, rec[i - s0], fc[i - s0], fb, lam, acc, A.grad);
        else
          normal_back<PC, GRID, LAY>(m, dopl, rec[i - s0], lam, acc, A.grad, true, rec[i - s0][kNg],
                                rec[i - s0][kNg + 1], rec[i - s0][kNg + 2], rec[i - s0][kNg + 3]);
      }
    }
  }
  St s;
  bool entered;
  double d_in[3], NB[3];
  start<PC, GRID, LAY>(m, A.a, r, s, entered, d_in, NB);
  entry_back<PC, GRID, LAY>(m, dopl, s, entered, d_in, NB, lam, acc, A.grad);
  if (!GRID)
    for (int q = 0; q < A.nterms; ++q)
      if (acc[q] != 0.0) atomicAdd(A.grad + q, acc[q]);
}

template <int PC, bool GRID, bool LAY>
static int run_t(const DevMedium& m, const AdjArgs& A, cudaStream_t st, int phase) {
  const unsigned blocks = (unsigned)((A.a.count + 127) / 128);
  if (phase != kAdjBackward &&
      launch_kernel(k_adj_forward<PC, GRID, LAY>, blocks, 128, st, m, A) < 0)
    return GRIN_ERR_CUDA;
  if (phase == kAdjForward) return 1;
  // The backward sweep walks each ray back through all its steps, one
  // thread a ray: in a gridded medium, where path lengths vary with the exit
  // face, take the rays longest first, bucketed by step count, so the threads
  // of a warp have similar amounts of work (measured 6x on the 128^3 blob
  // grid; on the polynomial block, whose rays have nearly equal lengths, the
  // permutation only cost locality).
  AdjArgs B = A;
  int lo = 0;
  if (GRID && A.order_ws) {
    lo = launch_order_by_steps(A.meta, A.a.count, A.order_ws, st, &B.order);
    if (lo < 0) {
      B.order = nullptr;
      lo = 0;
    }
  }
  if (launch_kernel(k_adj_backward<PC, GRID, LAY>, blocks, 128, st, m, B) < 0) return GRIN_ERR_CUDA;
  return (phase == kAdjBackward ? 1 : 2) + lo;
}

}  // namespace adj

bool adjoint_supported(const DevMedium& m) {
  if (m.bkind != GRIN_BOUNDARY_BOX && m.bkind != GRIN_BOUNDARY_SPHERE &&
      m.bkind != GRIN_BOUNDARY_CYLINDER)
    return false;
  if (m.kind == GRIN_MEDIUM_GRID || m.kind == GRIN_MEDIUM_N2P) return true;
  return (m.kind == GRIN_MEDIUM_POLY || m.kind == GRIN_MEDIUM_SPHERICAL) &&
         (m.form == GRIN_FORM_LINEAR || m.form == GRIN_FORM_SQRT || m.form == GRIN_FORM_RECIP);
}

// Workspace: checkpoints [ray][segment][kCk] | meta [ray][2] | (256-byte
// aligned) the backward order's scratch, for fewer than 2^31 rays.
static size_t adjoint_order_offset(int64_t rays, int32_t max_steps, int32_t k) {
  const int64_t nseg = max_steps / k + 1;
  const size_t end = (size_t)rays * (size_t)nseg * adj::kCk * sizeof(double) +
                     (size_t)rays * 2 * sizeof(int32_t);
  return (end + 255) & ~size_t(255);
}

size_t adjoint_workspace(int64_t rays, int32_t max_steps, int32_t k) {
  size_t bytes = adjoint_order_offset(rays, max_steps, k);
  if (rays > 0 && rays < (int64_t(1) << 31)) bytes += order_scratch_bytes(rays);
  return bytes + 256;
}

// The medium kinds, continuous (LAY = false) or in point-sampled shells.
template <bool LAY>
static int launch_adjoint_t(const DevMedium& m, const adj::AdjArgs& A, cudaStream_t st, int phase) {
  if (m.kind == GRIN_MEDIUM_GRID) return adj::run_t<0, true, LAY>(m, A, st, phase);
  if (m.kind == GRIN_MEDIUM_N2P) return adj::run_t<kN2P, false, LAY>(m, A, st, phase);
  if (m.kind == GRIN_MEDIUM_SPHERICAL) return adj::run_t<kSpherical, false, LAY>(m, A, st, phase);
  switch (m.pclass) {
    case kPoly2: return adj::run_t<2, false, LAY>(m, A, st, phase);
    case kPoly4: return adj::run_t<4, false, LAY>(m, A, st, phase);
    default: return adj::run_t<6, false, LAY>(m, A, st, phase);
  }
}

int launch_adjoint(const DevMedium& m, const TraceArgs& a, int32_t k, void* ws, const double* const* gout,
                   double* grad, int nterms, cudaStream_t st, int phase) {
  adj::AdjArgs A;
  A.a = a;
  A.k = k;
  A.nseg = a.max_steps / k + 1;
  A.ckpt = (double*)ws;
  A.meta = (int32_t*)((char*)ws + (size_t)a.count * A.nseg * adj::kCk * sizeof(double));
  static const double* const kNone[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (!gout) gout = kNone;  // the forward sweep alone reads no gradients
  A.gpx = gout[0];
  A.gpy = gout[1];
  A.gpz = gout[2];
  A.gdx = gout[3];
  A.gdy = gout[4];
  A.gdz = gout[5];
  A.gopl = gout[6];
  A.grad = grad;
  A.nterms = nterms;
  if (a.count < (int64_t(1) << 31))
    A.order_ws = (char*)ws + adjoint_order_offset(a.count, a.max_steps, k);
  if (m.n_levels > 0) return launch_adjoint_t<true>(m, A, st, phase);
  return launch_adjoint_t<false>(m, A, st, phase);
}


}  // namespace grin
