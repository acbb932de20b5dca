// trace_fp64_fast.cu -- FP64 VRT tracer with fused, reordered arithmetic: one
// thread per ray, polynomials by nested Horner with FMAs.  It computes the
// same steps as the plain FP64 tracer (trace_fp64.cu) with fewer FP64
// operations, so it is the fair FP64 speed baseline; its results differ from
// the plain tracer's by rounding order only (amplified near critical
// incidence, where gamma goes like sqrt(D)).
//
// Per step, at the new point P_i: evaluate n_i and grad n (Eq. 5); then, in
// this order: a crossing of the enclosing surface (Sec. II (i), boundary
// normal, mu = n_{i-1} / n_ext); zero or undefined gradient (ii)/(iii),
// straight on; N.I == 0 (iv), circular arc; D <= 0 (v), reflection with a
// step of dL0 / n_{i-1}; else refraction R = mu I + gamma N (Eq. 8-9) with a
// step of dL0 / n_i (Eq. 2-3).  n_{i-1} is always n at the previous point.
#include "grin_device.cuh"

namespace grin {


template <int PC, bool GRID, bool LAYERED>
__device__ void trace_one_fp64_fast(const DevMedium& m, const TraceArgs& a, int64_t r) {
  using F = Field64Fast<PC, GRID, LAYERED>;
  V3 p = mk(ld(a.ox, r, a.dtype), ld(a.oy, r, a.dtype), ld(a.oz, r, a.dtype));
  V3 d = mk(ld(a.dx, r, a.dtype), ld(a.dy, r, a.dtype), ld(a.dz, r, a.dtype));
  if (!finite3(p) || !finite3(d) || dot(d, d) == 0.0) {
    store_ray(a, r, p, d, 0.0, GRIN_EXIT_INVALID, 0, 0, 0);
    return;
  }
  d = unit(d);
  double opl_ext = 0.0, n_prev;
  V3 g;
  int lvl_prev;
  if (inside64(m, p)) {
    F::eval(m, p, n_prev, g, lvl_prev);
  } else {
    double t;
    V3 pb, nb;
    int face;
    if (!enter64(m, p, d, t, pb, nb, face)) {
      store_ray(a, r, p, d, 0.0, GRIN_EXIT_MISS, 0, 0, 0);
      return;
    }
    opl_ext = m.n_ext * t;
    p = pb;
    F::eval(m, p, n_prev, g, lvl_prev);
    if (refract64(d, nb, m.n_ext / n_prev)) {
      store_ray(a, r, p, d, opl_ext, GRIN_EXIT_ENTRY_REFLECT, 0, 0, 0);
      return;
    }
  }
  if (!(isfinite(n_prev) && n_prev > 0.0)) {
    store_ray(a, r, p, d, opl_ext, GRIN_EXIT_INVALID, 0, 0, 0);
    return;
  }
  const double dopl = a.dopl;
  double h = dopl / n_prev;
  V3 q = axpy(h, d, p);
  int steps = 0, full = 0, tir_i = 0, tir_b = 0, exit_id = GRIN_EXIT_MAXSTEPS;
  double frac = 0.0;
  while (steps < a.max_steps) {
    if (!inside64(m, q)) {
      double t;
      V3 pb, nb;
      int face;
      exit64(m, p, q, t, pb, nb, face);
      frac += t;
      ++steps;
      p = pb;
      if (refract64(d, nb, n_prev / m.n_ext)) {
        ++tir_b;
        h = dopl / n_prev;
        F::eval(m, p, n_prev, g, lvl_prev);
        if (!(isfinite(n_prev) && n_prev > 0.0)) {
          exit_id = GRIN_EXIT_INVALID;
          break;
        }
        q = axpy(h, d, p);
        continue;
      }
      exit_id = face;
      break;
    }
    p = q;
    ++full;
    ++steps;
    double n_i;
    int lvl_i;
    F::eval(m, p, n_i, g, lvl_i);
    if (!(isfinite(n_i) && n_i > 0.0)) {
      exit_id = GRIN_EXIT_INVALID;
      break;
    }
    double gn = sqrt(dot(g, g));
    if ((LAYERED && lvl_i == lvl_prev) || gn == 0.0 || !isfinite(gn)) {
      h = dopl / n_i;
    } else {
      V3 N = mk(g.x / gn, g.y / gn, g.z / gn);
      double c = dot(N, d);
      if (c == 0.0) {
        double hi = dopl / n_i;
        double n2;
        V3 g2;
        int l2;
        F::eval(m, axpy(hi, N, p), n2, g2, l2);
        double k = (n2 - n_i) / (2.0 * n_i);
        double w = 1.0 - k * k;
        d = unit(axpy(k, N, scale(w > 0.0 ? sqrt(w) : 0.0, d)));
        h = hi;
      } else if (refract64(d, N, n_prev / n_i)) {
        ++tir_i;
        h = dopl / n_prev;
      } else {
        h = dopl / n_i;
      }
    }
    n_prev = n_i;
    lvl_prev = lvl_i;
    q = axpy(h, d, p);
  }
  double opl = opl_ext + dopl * (double)full + dopl * frac;
  store_ray(a, r, p, d, opl, exit_id, steps, tir_i, tir_b);
}

template <int PC, bool GRID, bool LAYERED>
__global__ void __launch_bounds__(128) k_trace_fp64_fast(DevMedium m, TraceArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.count; r += stride)
    trace_one_fp64_fast<PC, GRID, LAYERED>(m, a, r);
}

template <int PC, bool GRID, bool LAYERED>
static int launch_t(const DevMedium& m, const TraceArgs& a, cudaStream_t s) {
  const int block = 128;
  int64_t blocks = (a.count + block - 1) / block;
  if (blocks > (1 << 30)) blocks = 1 << 30;
  return launch_kernel(k_trace_fp64_fast<PC, GRID, LAYERED>, (unsigned)blocks, block, s, m, a);
}

int launch_fp64_fast(const DevMedium& m, const TraceArgs& a, cudaStream_t s, int) {
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

}  // namespace grin
