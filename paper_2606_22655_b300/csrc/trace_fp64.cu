// trace_fp64.cu -- the plain FP64 VRT tracer: one thread per ray, every
// quantity of the method in double precision (Chavez-Islas et al., Sec. II).
//
// This file is compiled with --fmad=false, and every expression is written
// as the plain formula in a fixed left-to-right order with IEEE division and
// square root: polynomials as sums of monomials c x^i y^j z^k (powers by
// repeated multiplication), the tricubic interpolant as the 64-term sum of
// weight products, the vectorial Snell law as R = mu I + gamma N with
// gamma = -mu c + sgn(c) sqrt(D).  Each result is therefore a function of
// the inputs alone, independent of compiler contraction choices, which makes
// it the GPU reference that the mixed-precision tracer is gated against.
//
// Per step, at the new point P_i: n_i and grad n (Eq. 5); then, in this
// order: crossing of the enclosing surface (Sec. II (i), boundary normal,
// mu = n_{i-1} / n_ext); zero or undefined gradient ((ii)/(iii), straight
// on); N.I == 0 ((iv), circular arc); D <= 0 ((v), reflection with a step of
// dL0 / n_{i-1}); else refraction (Eq. 8-9) with a step of dL0 / n_i.
// n_{i-1} is n at the previous point (also after a reflection).
#include "plain_fp64.cuh"

namespace grin {
namespace plain {

// Shell crossings within one step, at most (GRIN_TRACE_LEVEL_ROOT): a ray
// grazing a curved shell boundary can cross it back and forth at ever shorter
// intervals; after this many the rest of the step runs straight.
constexpr int kMaxCrossings = 16;

// Point recorder of grin_trace_path: the first interior point, every full
// step and every surface cut, at most cap points (ray-major, xyz).
struct PathTap {
  double* pts;
  int64_t cap, n;
  __device__ __forceinline__ void put(const double* P) {
    if (n < cap) {
      pts[3 * n] = P[0];
      pts[3 * n + 1] = P[1];
      pts[3 * n + 2] = P[2];
    }
    ++n;
  }
};

template <int PC, bool GRID, bool LAYERED, bool TAP = false>
__device__ void trace_one(const DevMedium& m, const TraceArgs& a, int64_t r,
                          PathTap* tap = nullptr) {
  // decision margins are kept only when the caller asked for them
  const bool keep = a.margin != nullptr;
  Margins mg;
  mg.init();
  double dm = INFINITY;
  auto finish = [&](const double* P, const double* d, double opl, int exit_id, int steps, int ti,
                    int tb) {
    put(a, r, P, d, opl, exit_id, steps, ti, tb);
    if (keep)
      for (int k = 0; k < 4; ++k) a.margin[4 * r + k] = mg.v[k];
  };
  double P[3] = {ld(a.ox, r, a.dtype), ld(a.oy, r, a.dtype), ld(a.oz, r, a.dtype)};
  double d[3] = {ld(a.dx, r, a.dtype), ld(a.dy, r, a.dtype), ld(a.dz, r, a.dtype)};
  if (!finite3(P) || !finite3(d) || sqrt(dot3(d, d)) == 0.0) {
    finish(P, d, 0.0, GRIN_EXIT_INVALID, 0, 0, 0);
    return;
  }
  normalize3(d);
  double n_prev, g[3], opl_ext = 0.0, u;
  int lvl_prev;
  if (inside(m, P)) {
    sample<PC, GRID, LAYERED>(m, P, n_prev, g, lvl_prev);
  } else {
    double t, Pb[3], NB[3];
    int face;
    if (!enter(m, P, d, t, Pb, NB, face)) {
      finish(P, d, 0.0, GRIN_EXIT_MISS, 0, 0, 0);
      return;
    }
    opl_ext = m.n_ext * t;
    P[0] = Pb[0];
    P[1] = Pb[1];
    P[2] = Pb[2];
    sample<PC, GRID, LAYERED>(m, P, n_prev, g, lvl_prev);
    const bool refl = snell(d, NB, m.n_ext / n_prev, keep ? &dm : nullptr);
    if (keep) mg.take(0, fabs(dm));
    if (refl) {
      finish(P, d, opl_ext, GRIN_EXIT_ENTRY_REFLECT, 0, 0, 0);
      return;
    }
  }
  if (!(isfinite(n_prev) && n_prev > 0.0)) {
    finish(P, d, opl_ext, GRIN_EXIT_INVALID, 0, 0, 0);
    return;
  }
  if (TAP) tap->put(P);
  const double dopl = a.dopl;
  double h = dopl / n_prev;
  double Q[3];
  for (int k = 0; k < 3; ++k) Q[k] = P[k] + h * d[k];
  int steps = 0, full = 0, ti = 0, tb = 0, exit_id = GRIN_EXIT_MAXSTEPS;
  double frac = 0.0;
  const bool level_root = LAYERED && (a.flags & GRIN_TRACE_LEVEL_ROOT);
  double rem = 1.0;   // fraction of the current step's dL0 still to go
  int crossings = 0;  // shell crossings in the current step
  while (steps < a.max_steps) {
    if (LAYERED && level_root) {
      // Shells with their crossings solved: straight inside a shell (Sec. II
      // (iii)); where the ray leaves its shell, the first point outside it
      // (bisection on the segment) is where it refracts (Eq. 8-9) with the
      // isoindicial normal grad f / |grad f| and mu = n_k / n_k', or is
      // totally reflected (Sec. II (v)), and it goes on with the rest of the
      // step's optical path (rem, a fraction of dL0; Q = P + rem h d).  At
      // most kMaxCrossings crossings a step; then the rest of the step runs
      // straight into the shell it ends in.
      if (keep) mg.take(2, bmargin(m, Q, h));
      double E[3], tq = 1.0, Pb[3], NB[3];
      int face = 0;
      const bool leaves = !inside(m, Q);
      if (leaves) {
        leave(m, P, Q, tq, Pb, NB, face);
        E[0] = Pb[0];
        E[1] = Pb[1];
        E[2] = Pb[2];
      } else {
        E[0] = Q[0];
        E[1] = Q[1];
        E[2] = Q[2];
      }
      double nE, gE[3];
      int lE;
      sample<PC, GRID, LAYERED>(m, E, nE, gE, lE);
      if (lE != lvl_prev && crossings == kMaxCrossings) {
        lvl_prev = lE;
        n_prev = nE;
      }
      if (lE != lvl_prev) {
        ++crossings;
        double lo = 0.0, hi = 1.0, X[3], nX, gX[3];
        int lX;
        for (int it = 0; it < 128; ++it) {
          double mid = 0.5 * (lo + hi);
          if (!(mid > lo && mid < hi)) break;
          for (int k = 0; k < 3; ++k) X[k] = P[k] + mid * (E[k] - P[k]);
          sample<PC, GRID, LAYERED>(m, X, nX, gX, lX);
          if (lX == lvl_prev) lo = mid;
          else hi = mid;
        }
        for (int k = 0; k < 3; ++k) X[k] = P[k] + hi * (E[k] - P[k]);
        sample<PC, GRID, LAYERED>(m, X, nX, gX, lX);
        const double used = hi * tq * rem;
        frac += used;
        rem = rem - used;
        P[0] = X[0];
        P[1] = X[1];
        P[2] = X[2];
        if (TAP) tap->put(P);
        if (!(isfinite(nX) && nX > 0.0)) {
          exit_id = GRIN_EXIT_INVALID;
          break;
        }
        double gn = sqrt(dot3(gX, gX));
        if (gn == 0.0 || !isfinite(gn)) {
          n_prev = nX;
          lvl_prev = lX;
        } else {
          double N[3] = {gX[0] / gn, gX[1] / gn, gX[2] / gn};
          if (keep) mg.take(1, fabs(dot3(N, d)));
          const bool refl = snell(d, N, n_prev / nX, keep ? &dm : nullptr);
          if (keep) mg.take(0, fabs(dm));
          if (refl) {
            ++ti;
          } else {
            n_prev = nX;
            lvl_prev = lX;
          }
        }
        h = dopl / n_prev;
        for (int k = 0; k < 3; ++k) Q[k] = P[k] + rem * h * d[k];
        continue;
      }
      crossings = 0;
      if (!leaves) {
        P[0] = Q[0];
        P[1] = Q[1];
        P[2] = Q[2];
        if (rem == 1.0) ++full;
        else frac += rem;
        ++steps;
        rem = 1.0;
        if (TAP) tap->put(P);
        h = dopl / n_prev;
        for (int k = 0; k < 3; ++k) Q[k] = P[k] + h * d[k];
        continue;
      }
      // the rest of the step meets the enclosing surface inside the shell:
      // below
    }
    if (keep) mg.take(2, bmargin(m, Q, h));
    if (!inside(m, Q)) {
      double t, Pb[3], NB[3];
      int face;
      leave(m, P, Q, t, Pb, NB, face);
      frac += t * rem;
      rem = 1.0;
      ++steps;
      P[0] = Pb[0];
      P[1] = Pb[1];
      P[2] = Pb[2];
      if (TAP) tap->put(P);
      const bool refl = snell(d, NB, n_prev / m.n_ext, keep ? &dm : nullptr);
      if (keep) mg.take(0, fabs(dm));
      if (refl) {
        ++tb;
        h = dopl / n_prev;
        sample<PC, GRID, LAYERED>(m, P, n_prev, g, lvl_prev);
        if (!(isfinite(n_prev) && n_prev > 0.0)) {
          exit_id = GRIN_EXIT_INVALID;
          break;
        }
        for (int k = 0; k < 3; ++k) Q[k] = P[k] + h * d[k];
        continue;
      }
      exit_id = face;
      break;
    }
    P[0] = Q[0];
    P[1] = Q[1];
    P[2] = Q[2];
    ++full;
    ++steps;
    if (TAP) tap->put(P);
    double n_i;
    int lvl_i;
    sample<PC, GRID, LAYERED>(m, P, n_i, g, lvl_i, &u);
    if (keep && LAYERED) mg.take(3, lmargin(m, u));
    if (!(isfinite(n_i) && n_i > 0.0)) {
      exit_id = GRIN_EXIT_INVALID;
      break;
    }
    double gn = sqrt(dot3(g, g));
    if ((LAYERED && lvl_i == lvl_prev) || gn == 0.0 || !isfinite(gn)) {
      h = dopl / n_i;
    } else {
      double N[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
      double c = dot3(N, d);
      if (keep) mg.take(1, fabs(c));
      if (c == 0.0) {
        double hi = dopl / n_i;
        double Pn[3] = {P[0] + hi * N[0], P[1] + hi * N[1], P[2] + hi * N[2]};
        double n2, g2[3];
        int l2;
        sample<PC, GRID, LAYERED>(m, Pn, n2, g2, l2);
        double k = (n2 - n_i) / (2.0 * n_i);
        double w = 1.0 - k * k;
        double a0 = w > 0.0 ? sqrt(w) : 0.0;
        for (int q = 0; q < 3; ++q) d[q] = a0 * d[q] + k * N[q];
        normalize3(d);
        h = hi;
      } else {
        const bool refl = snell(d, N, n_prev / n_i, keep ? &dm : nullptr);
        if (keep) mg.take(0, fabs(dm));
        if (refl) {
          ++ti;
          h = dopl / n_prev;
        } else {
          h = dopl / n_i;
        }
      }
    }
    n_prev = n_i;
    lvl_prev = lvl_i;
    for (int k = 0; k < 3; ++k) Q[k] = P[k] + h * d[k];
  }
  double opl = opl_ext + dopl * (double)full + dopl * frac;
  finish(P, d, opl, exit_id, steps, ti, tb);
}

template <int PC, bool GRID, bool LAYERED>
__global__ void __launch_bounds__(128) k_trace_fp64(DevMedium m, TraceArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.count; r += stride)
    trace_one<PC, GRID, LAYERED>(m, a, r);
}

// grin_trace_path: the same trace with the point recorder; ray r's points
// go to path + 3 cap r, its point count (which may exceed cap) to plen[r].
template <int PC, bool GRID, bool LAYERED>
__global__ void __launch_bounds__(128) k_trace_fp64_path(DevMedium m, TraceArgs a, double* path,
                                                         int64_t cap, int64_t* plen) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.count; r += stride) {
    PathTap tap{path + 3 * cap * r, cap, 0};
    trace_one<PC, GRID, LAYERED, true>(m, a, r, &tap);
    plen[r] = tap.n;
  }
}

template <int PC, bool GRID, bool LAYERED>
int launch_path_t(const DevMedium& m, const TraceArgs& a, double* path, int64_t cap,
                  int64_t* plen, cudaStream_t s) {
  const int block = 128;
  int64_t blocks = (a.count + block - 1) / block;
  if (blocks > (1 << 30)) blocks = 1 << 30;
  return launch_kernel(k_trace_fp64_path<PC, GRID, LAYERED>, (unsigned)blocks, block, s, m, a,
                       path, cap, plen);
}

template <int PC, bool GRID, bool LAYERED>
int launch_t(const DevMedium& m, const TraceArgs& a, cudaStream_t s) {
  const int block = 128;
  int64_t blocks = (a.count + block - 1) / block;
  if (blocks > (1 << 30)) blocks = 1 << 30;
  return launch_kernel(k_trace_fp64<PC, GRID, LAYERED>, (unsigned)blocks, block, s, m, a);
}

}  // namespace plain

int launch_fp64(const DevMedium& m, const TraceArgs& a, cudaStream_t s, int) {
  using namespace plain;
  const bool lay = m.n_levels > 0;
  if (m.kind == GRIN_MEDIUM_GRID)
    return lay ? launch_t<0, true, true>(m, a, s) : launch_t<0, true, false>(m, a, s);
  switch (m.pclass) {
    case kSpherical:
      return lay ? launch_t<1, false, true>(m, a, s) : launch_t<1, false, false>(m, a, s);
    case kN2P:
      return lay ? launch_t<3, false, true>(m, a, s) : launch_t<3, false, false>(m, a, s);
    case kPoly2:
      return lay ? launch_t<2, false, true>(m, a, s) : launch_t<2, false, false>(m, a, s);
    case kPoly4:
      return lay ? launch_t<4, false, true>(m, a, s) : launch_t<4, false, false>(m, a, s);
    default:
      return lay ? launch_t<6, false, true>(m, a, s) : launch_t<6, false, false>(m, a, s);
  }
}

int launch_fp64_path(const DevMedium& m, const TraceArgs& a, double* path, int64_t cap,
                     int64_t* plen, cudaStream_t s) {
  using namespace plain;
  const bool lay = m.n_levels > 0;
  if (m.kind == GRIN_MEDIUM_GRID)
    return lay ? launch_path_t<0, true, true>(m, a, path, cap, plen, s)
               : launch_path_t<0, true, false>(m, a, path, cap, plen, s);
  switch (m.pclass) {
    case kSpherical:
      return lay ? launch_path_t<1, false, true>(m, a, path, cap, plen, s)
                 : launch_path_t<1, false, false>(m, a, path, cap, plen, s);
    case kN2P:
      return lay ? launch_path_t<3, false, true>(m, a, path, cap, plen, s)
                 : launch_path_t<3, false, false>(m, a, path, cap, plen, s);
    case kPoly2:
      return lay ? launch_path_t<2, false, true>(m, a, path, cap, plen, s)
                 : launch_path_t<2, false, false>(m, a, path, cap, plen, s);
    case kPoly4:
      return lay ? launch_path_t<4, false, true>(m, a, path, cap, plen, s)
                 : launch_path_t<4, false, false>(m, a, path, cap, plen, s);
    default:
      return lay ? launch_path_t<6, false, true>(m, a, path, cap, plen, s)
                 : launch_path_t<6, false, false>(m, a, path, cap, plen, s);
  }
}

}  // namespace grin
