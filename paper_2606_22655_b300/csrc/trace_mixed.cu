// trace_mixed.cu -- mixed-precision persistent ray-pool VRT tracer.
//
// The VRT step (Chavez-Islas et al., Sec. II; Eq. 1-9) runs in FP32:
//   - the point is kept as an unevaluated sum ph + pl of two floats and each
//     step's increment h d is added with Dekker's Fast2Sum (on polynomial
//     media, into pl alone, the pair normalised every kStepQuantum steps),
//     so rounding does not pile up over thousands of steps;
//   - the unit direction is kept the same way (dh + dl): a refraction adds
//     the small vector R - I = gamma N - (1 - mu) I, a reflection -2 c N, by
//     Fast2Sum, so the direction does not random-walk by one FP32
//     rounding per step (that walk, a few 1e-6 after 3000 steps, would decide
//     on which side of a turning point of n the discrete map kinks); R is a
//     unit vector whenever I and N are, so no per-step renormalisation;
//   - the index difference n_i - n_{i-1}, which sets 1 - mu and hence the
//     whole deflection, is taken by the trapezoid rule on grad n along the
//     step, (grad n_{i-1} + grad n_i) . (P_i - P_{i-1}) / 2, which equals the
//     point difference to O(step^3) but keeps FP32 relative accuracy where
//     the difference of two rounded indices would not (near turning points,
//     where gamma ~ sqrt(D) amplifies any error in 1 - mu^2); layered media
//     use the exact level values; the index itself is carried as
//     nu = n - base;
//   - the refraction uses gamma = sgn(c) (1 - mu^2) / (sqrt(D) + mu |c|), an
//     algebraically equal form of Eq. 9 without the cancellation of
//     -mu c + sgn(c) sqrt(D); D = (1 - mu^2) + mu^2 c^2; steps with D at or
//     below the near-critical band, total internal reflection included (a
//     few per ray), take the out-of-line step, so the common step refracts
//     without a branch;
//   - when |D| is within a few FP32 roundings of zero (near critical or
//     grazing incidence) the discriminant and gamma are recomputed in FP64;
//   - the optical path is exact: dL0 times the count of full steps (all steps
//     but those cut at the surface, which are the only ones counted apart), plus the
//     FP64 exterior segment and the fractions of steps cut at the surface;
//   - everything at the enclosing surface (the entry intersection and
//     refraction, the exit root, boundary refraction or TIR) runs in FP64.
// This file is built with -prec-div=false -prec-sqrt=false: FP32 divisions
// and square roots use the hardware approximations (a few ulp), which is far
// inside the FP32 path's error budget and removes their slow-path branches.
//
// Work distribution: a persistent grid sized to the resident capacity of the
// GPU; each warp keeps 32 rays in flight and, every kStepQuantum steps, lanes
// whose ray finished claim new rays from a global counter (one atomicAdd per
// warp, ranks from a ballot), so long and short rays do not idle lanes.
//
// Template parameters: polynomial degree class PC (or GRID), LAYERED, and the
// boundary kind BK and index form FORM, either fixed at compile time (the
// common box / n = p case, which drops their run-time switches from the step)
// or -1 for "read from the medium at run time".
#include <climits>
#include <type_traits>

#include "grin_device.cuh"

namespace grin {

// Resident blocks of 128 threads per SM the register allocation aims for:
// 5 (at most 102 registers a thread) for polynomial and grid media, 4 (128
// registers) for the shells of a layered grid, whose level logic spills at
// 96; the measured optimum between register spills and resident warps
// (256^3 grid at 1,048,576 rays: 4, 5, 6 blocks 5.26e10, 5.52e10, 5.33e10
// ray-steps/s; its 32 shells 5.11e10, 4.94e10, 5.02e10).
#ifndef GRIN_MIXED_MIN_BLOCKS
#define GRIN_MIXED_MIN_BLOCKS 5
#endif
#ifndef GRIN_MIXED_MIN_BLOCKS_GRID
#define GRIN_MIXED_MIN_BLOCKS_GRID 5
#endif
#ifndef GRIN_MIXED_MIN_BLOCKS_LAYERED_GRID
#define GRIN_MIXED_MIN_BLOCKS_LAYERED_GRID 4
#endif
constexpr int kStepQuantum = 32;
// Tap cache of the gridded fast step: 16 rows (one per (z, y) pair of the
// stencil) of 128 float4 columns, one column per thread; the 4-float pad
// between rows spreads one column's rows over the banks.
constexpr int kTapRow = 128 * 4 + 4;
constexpr float kCritBand = 1.0e-5f;  // relative |D| below which FP64 decides

#define GRIN_UNLIKELY(x) __builtin_expect(!!(x), 0)

struct RayF;

// The value and partials of a total-degree-D polynomial (Horner layout, see
// hidx; coefficient t at c[2 t], DevMedium::c32s) in FP32: poly_vg's nested
// Horner with derivative accumulators, with the outermost level's value and
// z-partial, which both advance as (P, PZ) <- (P, PZ) x + (A, AZ), taken two
// at a time by the packed fma.rn.f32x2.  The same FMAs in the same order as
// poly_vg<D, float>, in fewer instructions.
template <int D>
__device__ __forceinline__ void poly_vg2(const float* __restrict__ c, float x, float y, float z,
                                         float& p, float& px, float& py, float& pz) {
  const float2 xx = make_float2(x, x);
  float2 P = make_float2(0.0f, 0.0f);  // (P, PZ)
  float PX = 0.0f, PY = 0.0f;
#pragma unroll
  for (int i = D; i >= 0; --i) {
    float2 A = make_float2(0.0f, 0.0f);  // (A, AZ)
    float AY = 0.0f;
#pragma unroll
    for (int j = D - i; j >= 0; --j) {
      const int top = D - i - j;
      float B = c[2 * hidx(D, i, j, top)], BZ = 0.0f;
#pragma unroll
      for (int k = top - 1; k >= 0; --k) {
        BZ = (k == top - 1) ? B : fmaf(BZ, z, B);
        B = fmaf(B, z, c[2 * hidx(D, i, j, k)]);
      }
      if (j == D - i) {
        A = make_float2(B, BZ);
      } else {
        AY = (j == D - i - 1) ? A.x : fmaf(AY, y, A.x);
        A = make_float2(fmaf(A.x, y, B), fmaf(A.y, y, BZ));
      }
    }
    if (i == D) {
      P = A;
      PY = AY;
    } else {
      PX = (i == D - 1) ? P.x : fmaf(PX, x, P.x);
      P = __ffma2_rn(P, xx, A);
      PY = fmaf(PY, x, AY);
    }
  }
  p = P.x;
  pz = P.y;
  px = PX;
  py = PY;
}

// MG: the kernel also keeps each ray's decision margins (grin_out.margin).
template <int PC, bool GRID, bool LAYERED, int BK, int FORM, bool MG = false>
struct Cfg {
  static constexpr bool kGrid = GRID;
  static constexpr int kPC = PC;
  static constexpr bool kLayered = LAYERED;
  static constexpr bool kMG = MG;
  // Polynomial media read only the hi part of a point, so their fast step
  // carries it lazily: ph stays put for a quantum of steps while pl
  // accumulates them (see step_point); a gridded medium's cell needs the
  // pair normalised after every step.
  static constexpr bool kLazyPos = !GRID;
  static constexpr int kMinBlocks = GRID ? GRIN_MIXED_MIN_BLOCKS_GRID : GRIN_MIXED_MIN_BLOCKS;
  static constexpr int kMinBlocksLayered = GRID ? GRIN_MIXED_MIN_BLOCKS_LAYERED_GRID : kMinBlocks;
  static __device__ __forceinline__ int bk(const DevMedium& m) { return BK >= 0 ? BK : m.bkind; }
  static __device__ __forceinline__ int form(const DevMedium& m) { return FORM >= 0 ? FORM : m.form; }

  // nu = n - base (after layering), the gradient of the smooth field, level,
  // at the point (px + lx, py + ly, pz + lz) (a hi + lo pair; polynomial
  // media read the hi part).
  static __device__ __forceinline__ void eval(const DevMedium& m, float px, float py, float pz,
                                              float lx, float ly, float lz, float& nu,
                                              float& gx, float& gy, float& gz, int& lvl,
                                              float* uo = nullptr) {
    float f;
    field(m, px, py, pz, lx, ly, lz, f, gx, gy, gz);
    level(m, f, nu, lvl, uo);
  }

  // The smooth field f = n - base (before any layering) and its gradient.
  static __device__ __forceinline__ void field(const DevMedium& m, float px, float py, float pz,
                                               float lx, float ly, float lz, float& f,
                                               float& gx, float& gy, float& gz) {
    if (GRID) {
      const float ph[3] = {px, py, pz}, pl[3] = {lx, ly, lz};
      int i0[3];
      float fr[3];
      cell(m, ph, pl, i0, fr);
      grid_gather(m, i0, fr, f, gx, gy, gz);
    } else {
      float x = fmaf(px, m.inv_scale_f[0], m.noff_f[0]);
      float y = fmaf(py, m.inv_scale_f[1], m.noff_f[1]);
      float z = fmaf(pz, m.inv_scale_f[2], m.noff_f[2]);
      float q, qx, qy, qz;
      if constexpr (PC == kPoly2 || PC == kPoly4 || PC == kPoly6)
        poly_vg2<PC>(m.c32s, x, y, z, q, qx, qy, qz);
      else
        field_vg<PC, float>(m.c32, x, y, z, q, qx, qy, qz);
      qx *= m.inv_scale_f[0];
      qy *= m.inv_scale_f[1];
      qz *= m.inv_scale_f[2];
      const int fm = form(m);
      if (fm == GRIN_FORM_LINEAR) {
        f = q;  // constant term already shifted by base
        gx = qx;
        gy = qy;
        gz = qz;
      } else if (fm == GRIN_FORM_SQRT) {
        // q = p - base^2: n = sqrt(q + base^2), nu = q / (n + base)
        float n = sqrtf(fmaf(m.base_f, m.base_f, q));
        f = q / (n + m.base_f);
        float s = 0.5f / n;
        gx = qx * s;
        gy = qy * s;
        gz = qz * s;
      } else {
        float n = m.form_c_f / q;
        f = n - m.base_f;
        float s = -n / q;
        gx = qx * s;
        gy = qy * s;
        gz = qz * s;
      }
    }
  }

  // f = n - base of the smooth field -> nu = n - base of the medium and its
  // level (a layered medium takes the centre value of f's shell).
  // (uo: the level coordinate, for the level margin)
  static __device__ __forceinline__ void level(const DevMedium& m, float f, float& nu, int& lvl,
                                               float* uo = nullptr) {
    if (LAYERED) {
      float u = (f - m.lvl_lo_rel_f) * m.lvl_scale_f;
      float fl = floorf(u);
      int k = fl >= 0.0f ? (fl > (float)(m.n_levels - 1) ? m.n_levels - 1 : (int)fl) : 0;
      lvl = k;
      nu = shell_nu(m, k);
      if (uo) *uo = u;
    } else {
      lvl = 0;
      nu = f;
      if (uo) *uo = 0.5f;
    }
  }

  // n - base of shell k of a layered medium.
  static __device__ __forceinline__ float shell_nu(const DevMedium& m, int k) {
    return fmaf((float)k + 0.5f, m.lvl_step_f, m.lvl_lo_rel_f);
  }

  // Gridded media.  The cell of the 64-tap stencil at the point ph + pl and
  // the fractions inside it.  The grid coordinate u = (p - origin) / spacing
  // is formed as u_h + corr: u_h = fl(fl(ph - origin_f) * inv_spacing_f) picks
  // the cell (clamped to [-2, n + 1], a NaN to -2) and corr collects, by
  // TwoSum and a fused product residual, every part that u_h drops (the
  // subtraction's and the product's rounding, the point's low part and the
  // residuals of origin_f and inv_spacing_f).  An FP32 point near 10 mm is
  // only good to about 1e-6 mm, 1e-5 of a 256^3 cell; with corr the fraction
  // is good to FP32 resolution within the cell, which keeps grad n and hence
  // N.I at about 1e-7 (near turning points of n, where Eq. 9 is steep in
  // N.I, that error is what the path accumulates).  The fraction may leave
  // [0, 1) by corr; the cell's polynomial is then taken a hair outside it.
  static __device__ __forceinline__ void cell(const DevMedium& m, const float* ph, const float* pl,
                                              int* i0, float* fr) {
    const int n[3] = {m.nx, m.ny, m.nz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float s = m.inv_spacing_f[k];
      const float a = ph[k] - m.origin_f[k];
      const float bp = a - ph[k];
      const float ea = (ph[k] - (a - bp)) + (-m.origin_f[k] - bp);  // a + ea = ph - origin_f
      float u = a * s;
      const float eu = fmaf(a, s, -u);                              // u + eu = a s
      float corr = fmaf(a, m.inv_spacing_lo_f[k], fmaf((ea + pl[k]) - m.origin_lo_f[k], s, eu));
      if (!(u > -2.0f)) {
        u = -2.0f;
        corr = 0.0f;
      }
      if (u > (float)(n[k] + 1)) {
        u = (float)(n[k] + 1);
        corr = 0.0f;
      }
      const float fl = floorf(u);
      i0[k] = (int)fl;
      fr[k] = (u - fl) + corr;
    }
  }

  // The sample at the stencil's centre tap (cell corner i0, edge-clamped):
  // every tap is taken relative to it, so the sums of the interpolant and
  // its gradient carry the local variation of the samples (a few 1e-3 on a
  // 256^3 blob field) instead of their offset from a global base (5e-2),
  // with ten times fewer rounding errors in grad n.
  static __device__ __forceinline__ float centre_tap(const DevMedium& m, const int* i0) {
    const int ix = min(max(i0[0], 0), m.nx - 1), iy = min(max(i0[1], 0), m.ny - 1),
              iz = min(max(i0[2], 0), m.nz - 1);
    return __ldg(m.grid + GRIN_IDX(m, ((int64_t)iz * m.ny + iy) * m.nx + ix, m.grid_n, kSiteGridMixed));
  }

  // Catmull-Rom value (f = n - base) and gradient (physical units) at cell
  // i0 and fractions fr, gathering the 64 edge-clamped taps from the grid:
  // the same products summed in the same order as eval_taps from the tap
  // cache, so both give the same bits.
  static __device__ __forceinline__ void grid_gather(const DevMedium& m, const int* i0,
                                                     const float* fr, float& f, float& gx,
                                                     float& gy, float& gz) {
    float w[3][4], dw[3][4];
#pragma unroll
    for (int k = 0; k < 3; ++k) cr_w(fr[k], w[k], dw[k]);
    const float lb = centre_tap(m, i0);
    const int ix[4] = {min(max(i0[0] - 1, 0), m.nx - 1), min(max(i0[0], 0), m.nx - 1),
                       min(max(i0[0] + 1, 0), m.nx - 1), min(max(i0[0] + 2, 0), m.nx - 1)};
    float V = 0.0f, GX = 0.0f, GY = 0.0f, GZ = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int iz = min(max(i0[2] - 1 + c, 0), m.nz - 1);
      float sv = 0.0f, sx = 0.0f, sy = 0.0f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int iy = min(max(i0[1] - 1 + b, 0), m.ny - 1);
        const int64_t row = ((int64_t)iz * m.ny + iy) * m.nx;
        float r = 0.0f, rx = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float t = __ldg(m.grid + GRIN_IDX(m, row + ix[k], m.grid_n, kSiteGridMixed)) - lb;
          r = fmadd(w[0][k], t, r);
          rx = fmadd(dw[0][k], t, rx);
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
    f = V + (lb - m.base_f);
    gx = GX * m.inv_spacing_f[0];
    gy = GY * m.inv_spacing_f[1];
    gz = GZ * m.inv_spacing_f[2];
  }

  // eval for a gridded medium from the cell's 64 taps (sample - lb, lb the
  // centre tap; layout at tap_fill): the same products summed in the same
  // order as grid_gather's, so the same value and gradient bit for bit.
  static __device__ __forceinline__ void eval_taps(const DevMedium& m, const float* fr,
                                                   const float* col, float lb, float& nu,
                                                   float& gx, float& gy, float& gz, int& lvl,
                                                   float* uo = nullptr) {
    float f;
    taps_field(m, fr, col, lb, f, gx, gy, gz);
    level(m, f, nu, lvl, uo);
  }

  // The smooth field f = n - base and its gradient from the cached taps (the
  // part of eval_taps before the level).  Row 2 (4 p + b) + h of the column
  // holds, for the z planes c = 2p and 2p + 1 of stencil row b, the taps
  // x = 2h and 2h + 1 as (x: c, c + 1, x + 1: c, c + 1), so each float4 read
  // gives two plane pairs: the x and y sums of planes 2p and 2p + 1 go
  // together through packed FMAs (fma.rn.f32x2, each half an IEEE fma) with
  // the weight in both halves, and each plane's sums keep grid_gather's order.
  static __device__ __forceinline__ void taps_field(const DevMedium& m, const float* fr,
                                                    const float* col, float lb, float& f,
                                                    float& gx, float& gy, float& gz) {
    float w[3][4], dw[3][4];
#pragma unroll
    for (int k = 0; k < 3; ++k) cr_w(fr[k], w[k], dw[k]);
    float2 wx[4], dwx[4], wy[4], dwy[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      wx[k] = make_float2(w[0][k], w[0][k]);
      dwx[k] = make_float2(dw[0][k], dw[0][k]);
      wy[k] = make_float2(w[1][k], w[1][k]);
      dwy[k] = make_float2(dw[1][k], dw[1][k]);
    }
    const float2 z2 = make_float2(0.0f, 0.0f);
#ifdef GRIN_CHECKED
    // the column must lie in the block's cache (16 rows of kTapRow floats)
    col = col - (int64_t)threadIdx.x * 4 + GRIN_IDX(m, (int64_t)threadIdx.x * 4, kTapRow - 4, kSiteTapCache);
#endif
    float sv[4], sx[4], sy[4];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      float2 SV = z2, SX = z2, SY = z2;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float* row = col + (2 * (4 * p + b)) * kTapRow;
        const float4 q0 = *reinterpret_cast<const float4*>(row);
        const float4 q1 = *reinterpret_cast<const float4*>(row + kTapRow);
        const float2 t[4] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w),
                             make_float2(q1.x, q1.y), make_float2(q1.z, q1.w)};
        float2 r = z2, rx = z2;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          r = __ffma2_rn(wx[k], t[k], r);
          rx = __ffma2_rn(dwx[k], t[k], rx);
        }
        SV = __ffma2_rn(wy[b], r, SV);
        SX = __ffma2_rn(wy[b], rx, SX);
        SY = __ffma2_rn(dwy[b], r, SY);
      }
      sv[2 * p] = SV.x;
      sv[2 * p + 1] = SV.y;
      sx[2 * p] = SX.x;
      sx[2 * p + 1] = SX.y;
      sy[2 * p] = SY.x;
      sy[2 * p + 1] = SY.y;
    }
    float V = 0.0f, GX = 0.0f, GY = 0.0f, GZ = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      V = fmadd(w[2][c], sv[c], V);
      GX = fmadd(w[2][c], sx[c], GX);
      GY = fmadd(w[2][c], sy[c], GY);
      GZ = fmadd(dw[2][c], sv[c], GZ);
    }
    gx = GX * m.inv_spacing_f[0];
    gy = GY * m.inv_spacing_f[1];
    gz = GZ * m.inv_spacing_f[2];
    f = V + (lb - m.base_f);
  }

  static __device__ __forceinline__ bool inside(const DevMedium& m, const float* q) {
    const float* b = m.b_f;
    const int k = bk(m);
    if (k == GRIN_BOUNDARY_BOX)
      return q[0] > b[0] && q[0] < b[3] && q[1] > b[1] && q[1] < b[4] && q[2] > b[2] &&
             q[2] < b[5];
    if (k == GRIN_BOUNDARY_SPHERE) {
      float x = q[0] - b[0], y = q[1] - b[1], z = q[2] - b[2];
      return fmaf(x, x, fmaf(y, y, z * z)) < b[3] * b[3];
    }
    float x = q[0] - b[0], y = q[1] - b[1];
    return fmaf(x, x, y * y) < b[2] * b[2] && q[2] > b[3] && q[2] < b[4];
  }
};

struct RayF {
  float ph[3], pl[3], d[3], dl[3];  // point and direction as hi + lo pairs
  float gp[3];                      // grad n at the previous point
  float nu_prev, inv_prev, h;       // n_{i-1} - base, 1 / n_{i-1}, step length
  float frac;                       // sum of the fractions of steps cut at the surface
  int lvl_prev, steps, cut, tir_i, tir_b;  // cut: steps ended early at the surface
  double opl_x;  // exterior segment, in optical length
  // layered media with GRIN_TRACE_LEVEL_ROOT: the fraction of the current
  // step's dL0 spent before its shell crossings, and their number
  float used;
  int xc;
  // kernels with MG: the ray's decision margins (grin_out.margin, in FP32 on
  // this path's own trajectory), the minimum over the trace of [0] |N.I|
  // minus its critical value at refractions with mu > 1, [1] |N.I| at
  // gradient steps, [2] the distance of a step end to the surface in steps,
  // [3] the distance of the level coordinate to the nearest shell boundary
  // (the other kernels never touch them, and they take no registers there)
  float mg[4];
};

template <class C>
__device__ __forceinline__ void mg_init(RayF& s) {
  if constexpr (C::kMG)
    for (int k = 0; k < 4; ++k) s.mg[k] = INFINITY;
}

template <class C>
__device__ __forceinline__ void mg_take(RayF& s, int k, float v) {
  if constexpr (C::kMG) s.mg[k] = fminf(s.mg[k], v);
}

// |N.I| minus its critical value for a refraction test with
// c = N.I, mu = 1 - om, omm = 1 - mu^2 and discriminant D = mu^2 c^2 + omm:
// D / (mu^2 (|c| + c_crit)) with c_crit = sqrt(-omm) / mu when mu > 1.
__device__ __forceinline__ float crit_margin(float c, float mu, float omm, float D) {
  return omm < 0.0f ? fabsf(D) / (mu * fmaf(mu, fabsf(c), sqrtf(-omm))) : INFINITY;
}

// Distance of the level coordinate u to the nearest shell boundary, the
// integers 1 .. L-1 (the levels clamp below 0 and above L-1).
__device__ __forceinline__ float lvl_margin(const DevMedium& m, float u) {
  const float k = fminf(fmaxf(rintf(u), 1.0f), (float)(m.n_levels - 1));
  return m.n_levels > 1 ? fabsf(u - k) : INFINITY;
}

// Distance of a point to the enclosing surface, in steps of length h (first
// order for the curved surfaces).
template <class C>
__device__ __forceinline__ float bnd_margin(const DevMedium& m, const float* q, float h) {
  const float* b = m.b_f;
  const int k = C::bk(m);
  float r;
  if (k == GRIN_BOUNDARY_BOX) {
    r = fminf(fminf(fminf(fabsf(q[0] - b[0]), fabsf(b[3] - q[0])),
                    fminf(fabsf(q[1] - b[1]), fabsf(b[4] - q[1]))),
              fminf(fabsf(q[2] - b[2]), fabsf(b[5] - q[2])));
  } else if (k == GRIN_BOUNDARY_SPHERE) {
    float x = q[0] - b[0], y = q[1] - b[1], z = q[2] - b[2];
    r = fabsf(fmaf(x, x, fmaf(y, y, z * z)) - b[3] * b[3]) / (2.0f * b[3]);
  } else {
    float x = q[0] - b[0], y = q[1] - b[1];
    r = fminf(fabsf(fmaf(x, x, y * y) - b[2] * b[2]) / (2.0f * b[2]),
              fminf(fabsf(q[2] - b[3]), fabsf(b[4] - q[2])));
  }
  return r / h;
}

__device__ __forceinline__ V3 pos64(const RayF& s) {
  return mk((double)s.ph[0] + (double)s.pl[0], (double)s.ph[1] + (double)s.pl[1],
            (double)s.ph[2] + (double)s.pl[2]);
}

__device__ __forceinline__ void set_pos(RayF& s, V3 p) {
  s.ph[0] = (float)p.x;
  s.ph[1] = (float)p.y;
  s.ph[2] = (float)p.z;
  s.pl[0] = (float)(p.x - (double)s.ph[0]);
  s.pl[1] = (float)(p.y - (double)s.ph[1]);
  s.pl[2] = (float)(p.z - (double)s.ph[2]);
}

__device__ __forceinline__ V3 dir64(const RayF& s) {
  return mk((double)s.d[0] + (double)s.dl[0], (double)s.d[1] + (double)s.dl[1],
            (double)s.d[2] + (double)s.dl[2]);
}

__device__ __forceinline__ void set_dir(RayF& s, V3 d) {
  s.d[0] = (float)d.x;
  s.d[1] = (float)d.y;
  s.d[2] = (float)d.z;
  s.dl[0] = (float)(d.x - (double)s.d[0]);
  s.dl[1] = (float)(d.y - (double)s.d[1]);
  s.dl[2] = (float)(d.z - (double)s.d[2]);
}

// (hi, lo) += x: the carried residual lo is folded into x, then Dekker's
// Fast2Sum leaves hi = fl(hi + x) and the new residual in lo, so hi stays the
// rounded value of the pair.  Fast2Sum is exact when |hi| >= |x|; when a
// component of the unit direction is smaller than the step's increment (it
// passes through zero) the residual it returns is off by at most about one
// ulp of x, the size of the rounding of x + lo itself, so Knuth's six-operation
// TwoSum would buy nothing here.
__device__ __forceinline__ void add_ff(float& hi, float& lo, float x) {
  x += lo;
  const float s = hi + x;
  lo = x - (s - hi);
  hi = s;
}

// (hi, lo) <- TwoSum(hi, lo): an unevaluated pair normalised again, exactly.
__device__ __forceinline__ void two_sum(float& hi, float& lo) {
  const float s = hi + lo;
  const float bp = s - hi;
  lo = (hi - (s - bp)) + (lo - bp);
  hi = s;
}

// A lazily carried position (Cfg::kLazyPos) as a normalised pair again.
__device__ __forceinline__ void norm_pos(RayF& s) {
#pragma unroll
  for (int k = 0; k < 3; ++k) two_sum(s.ph[k], s.pl[k]);
}

__device__ __forceinline__ void finish(const TraceArgs& a, int64_t r, const RayF& s, V3 p, V3 d,
                                       int exit_id) {
  // every step but the cut ones adds exactly dL0 (Eq. 3)
  double opl = s.opl_x + a.dopl * ((double)(s.steps - s.cut) + (double)s.frac);
  store_ray(a, r, p, d, opl, exit_id, s.steps, s.tir_i, s.tir_b);
}

// finish, and the margins when the kernel keeps them and the caller asked.
template <class C>
__device__ __forceinline__ void fin(const TraceArgs& a, int64_t r, const RayF& s, V3 p, V3 d,
                                    int exit_id) {
  finish(a, r, s, p, d, exit_id);
  if constexpr (C::kMG)
    if (a.margin)
      for (int k = 0; k < 4; ++k) a.margin[4 * r + k] = (double)s.mg[k];
}

// (n_{i-1} - base) -> the state's index fields; false if n is not usable.
__device__ __forceinline__ bool set_index(const DevMedium& m, RayF& s, float nu) {
  s.nu_prev = nu;
  float n = m.base_f + nu;
  s.inv_prev = 1.0f / n;
  return isfinite(n) && n > 0.0f;
}

__device__ __forceinline__ void renorm(float* v) {
  float r = rsqrtf(fmaf(v[0], v[0], fmaf(v[1], v[1], v[2] * v[2])));
  v[0] *= r;
  v[1] *= r;
  v[2] *= r;
}

__device__ __forceinline__ V3 v3f(const float* v) { return mk((double)v[0], (double)v[1], (double)v[2]); }

// eval at an FP64 point, split into a hi + lo float pair.
template <class C>
__device__ __forceinline__ void eval64(const DevMedium& m, V3 p, float& nu, float* g, int& lvl) {
  const float hx = (float)p.x, hy = (float)p.y, hz = (float)p.z;
  C::eval(m, hx, hy, hz, (float)(p.x - (double)hx), (float)(p.y - (double)hy),
          (float)(p.z - (double)hz), nu, g[0], g[1], g[2], lvl);
}

// Box entry in FP32.  With an axis-aligned face the incidence cosine is one
// direction component, the crossing a slab parameter and the reflection a
// sign flip, so FP32 carries them to its own rounding; the entry point is
// an ordinary FP32 product, accurate to one rounding of the ray's origin.
template <class C>
__device__ bool init_ray_box32(const DevMedium& m, const TraceArgs& a, int64_t r, RayF& s, V3 p64,
                               V3 d64) {
  const float* b = m.b_f;
  float o[3] = {(float)p64.x, (float)p64.y, (float)p64.z};
  float d[3] = {(float)d64.x, (float)d64.y, (float)d64.z};
  float dd = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
  if (!finite3(p64) || !finite3(d64) || !(dd > 0.0f) || !isfinite(dd)) {
    fin<C>(a, r, s, p64, d64, GRIN_EXIT_INVALID);
    return false;
  }
  renorm(d);
  float nu;
  const bool in = o[0] > b[0] && o[0] < b[3] && o[1] > b[1] && o[1] < b[4] && o[2] > b[2] &&
                  o[2] < b[5];
  if (!in) {
    float tn = -INFINITY, tf = INFINITY;
    int axis = -1, hi = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (d[k] == 0.0f) {
        if (!(o[k] > b[k] && o[k] < b[3 + k])) axis = -2;
        continue;
      }
      float t1 = (b[k] - o[k]) / d[k], t2 = (b[3 + k] - o[k]) / d[k];
      float lo = fminf(t1, t2), up = fmaxf(t1, t2);
      if (lo > tn) {
        tn = lo;
        if (axis != -2) axis = k;
        hi = d[k] < 0.0f;
      }
      tf = fminf(tf, up);
    }
    if (axis < 0 || !(tn >= 0.0f && tn < tf)) {
      fin<C>(a, r, s, p64, v3f(d), GRIN_EXIT_MISS);
      return false;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = fmaf(tn, d[k], o[k]);
    o[axis] = hi ? b[3 + axis] : b[axis];
    s.opl_x = m.n_ext * (double)tn;
    C::eval(m, o[0], o[1], o[2], 0.0f, 0.0f, 0.0f, nu, s.gp[0], s.gp[1], s.gp[2], s.lvl_prev);
    // Snell at the face: N = outward axis, c = N.I, mu = n_ext / n(P_b)
    const float mu = m.n_ext_f / (m.base_f + nu);
    const float c = hi ? d[axis] : -d[axis];
    const float D = 1.0f - mu * mu * fmaf(-c, c, 1.0f);
    mg_take<C>(s, 0, crit_margin(c, mu, fmaf(-mu, mu, 1.0f), D));
    if (D <= 0.0f) {
      d[axis] = -d[axis];
      fin<C>(a, r, s, v3f(o), v3f(d), GRIN_EXIT_ENTRY_REFLECT);
      return false;
    }
    const float gamma = fmaf(-mu, c, copysignf(sqrtf(D), c));
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] *= mu;
    d[axis] += hi ? gamma : -gamma;
    renorm(d);
  } else {
    C::eval(m, o[0], o[1], o[2], 0.0f, 0.0f, 0.0f, nu, s.gp[0], s.gp[1], s.gp[2], s.lvl_prev);
  }
  if (!set_index(m, s, nu)) {
    fin<C>(a, r, s, v3f(o), v3f(d), GRIN_EXIT_INVALID);
    return false;
  }
  if (a.max_steps <= 0) {
    fin<C>(a, r, s, v3f(o), v3f(d), GRIN_EXIT_MAXSTEPS);
    return false;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s.ph[k] = o[k];
    s.pl[k] = 0.0f;
    s.d[k] = d[k];
    s.dl[k] = 0.0f;
  }
  s.h = (float)a.dopl * s.inv_prev;
  return true;
}

// A step ends on the enclosing surface a fraction t of the way along what was
// left of it: it counts as a step and adds that part of dL0 (plus, in a
// layered medium with its crossings solved, what the step spent before them).
template <class C>
__device__ __forceinline__ void cut_step(RayF& s, float t) {
  if constexpr (C::kLayered) {
    s.frac += fmaf(t, 1.0f - s.used, s.used);
    s.used = 0.0f;
    s.xc = 0;
  } else {
    s.frac += t;
  }
  ++s.steps;
  ++s.cut;
}

// Box crossing in FP32 (see init_ray_box32): the fraction of the step to
// the first face beyond, from the compensated point; Snell or reflection
// with the face normal.  Same return codes as surface_event.
template <class C>
__device__ __forceinline__ int surface_event_box32(const DevMedium& m, const TraceArgs& a,
                                                   int64_t r, RayF& s, float dopl_f,
                                                   const float* qh) {
  const float* b = m.b_f;
  float dv[3];
  float best = INFINITY;
  int bf = -1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dv[k] = fmaf(s.h, s.d[k], s.h * s.dl[k]);
    if (qh[k] <= b[k]) {
      float t = ((b[k] - s.ph[k]) - s.pl[k]) / dv[k];
      if (t < best) {
        best = t;
        bf = 2 * k;
      }
    }
    if (qh[k] >= b[3 + k]) {
      float t = ((b[3 + k] - s.ph[k]) - s.pl[k]) / dv[k];
      if (t < best) {
        best = t;
        bf = 2 * k + 1;
      }
    }
  }
  if (bf < 0 || best > 1.0f) return 0;  // the compensated end point is inside
  best = fmaxf(best, 0.0f);
  cut_step<C>(s, best);
  const int axis = bf >> 1, hi = bf & 1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float y = fmaf(best, dv[k], s.pl[k]);
    float t = s.ph[k] + y;
    s.pl[k] = y - (t - s.ph[k]);
    s.ph[k] = t;
  }
  s.ph[axis] = hi ? b[3 + axis] : b[axis];
  s.pl[axis] = 0.0f;
  // Sec. II (i): N = outward face normal, mu = n_{i-1} / n_ext
  const float mu = (m.base_f + s.nu_prev) / m.n_ext_f;
  const float c = hi ? s.d[axis] : -s.d[axis];
  const float D = 1.0f - mu * mu * fmaf(-c, c, 1.0f);
  mg_take<C>(s, 0, crit_margin(c, mu, fmaf(-mu, mu, 1.0f), D));
  bool tir = D <= 0.0f;
  if (GRIN_UNLIKELY(fabsf(D) <= kCritBand)) {
    double mu64 = ((double)m.base_f + (double)s.nu_prev) / m.n_ext;
    double c64 = (double)c + (double)(hi ? s.dl[axis] : -s.dl[axis]);
    tir = 1.0 - mu64 * mu64 * (1.0 - c64 * c64) <= 0.0;
  }
  if (tir) {
    // Sec. II (v): reflection flips the normal component exactly
    s.d[axis] = -s.d[axis];
    s.dl[axis] = -s.dl[axis];
    ++s.tir_b;
    s.h = dopl_f * s.inv_prev;
    float nu;
    C::eval(m, s.ph[0], s.ph[1], s.ph[2], s.pl[0], s.pl[1], s.pl[2], nu, s.gp[0], s.gp[1], s.gp[2],
            s.lvl_prev);
    if (!set_index(m, s, nu)) {
      fin<C>(a, r, s, pos64(s), dir64(s), GRIN_EXIT_INVALID);
      return 2;
    }
    if (s.steps >= a.max_steps) {
      fin<C>(a, r, s, pos64(s), dir64(s), GRIN_EXIT_MAXSTEPS);
      return 2;
    }
    return 1;
  }
  float R[3];
  const float gamma = fmaf(-mu, c, copysignf(sqrtf(fmaxf(D, 0.0f)), c));
#pragma unroll
  for (int k = 0; k < 3; ++k) R[k] = mu * (s.d[k] + s.dl[k]);
  R[axis] += hi ? gamma : -gamma;
  renorm(R);
  fin<C>(a, r, s, pos64(s), v3f(R), bf);
  return 2;
}

// Start ray r: entry through the surface (FP64, or FP32 for a box).
// Returns false when the ray is already finished (its output is written).
template <class C>
__device__ bool init_ray(const DevMedium& m, const TraceArgs& a, int64_t r, RayF& s) {
  V3 p = mk(ld(a.ox, r, a.dtype), ld(a.oy, r, a.dtype), ld(a.oz, r, a.dtype));
  V3 d = mk(ld(a.dx, r, a.dtype), ld(a.dy, r, a.dtype), ld(a.dz, r, a.dtype));
  s.steps = s.cut = s.tir_i = s.tir_b = 0;
  s.opl_x = 0.0;
  s.frac = 0.0f;
  if constexpr (C::kLayered) {
    s.used = 0.0f;
    s.xc = 0;
  }
  mg_init<C>(s);
  if (C::bk(m) == GRIN_BOUNDARY_BOX) return init_ray_box32<C>(m, a, r, s, p, d);
  if (!finite3(p) || !finite3(d) || dot(d, d) == 0.0) {
    fin<C>(a, r, s, p, d, GRIN_EXIT_INVALID);
    return false;
  }
  d = unit(d);
  float nu;
  if (!inside64(m, p)) {
    double t;
    V3 pb, nb;
    int face;
    if (!enter64(m, p, d, t, pb, nb, face)) {
      fin<C>(a, r, s, p, d, GRIN_EXIT_MISS);
      return false;
    }
    s.opl_x = m.n_ext * t;
    p = pb;
    eval64<C>(m, p, nu, s.gp, s.lvl_prev);
    double nb_in = (double)m.base_f + (double)nu;
    double cm = INFINITY;
    const bool refl = refract64(d, nb, m.n_ext / nb_in, C::kMG ? &cm : nullptr);
    mg_take<C>(s, 0, (float)cm);
    if (refl) {
      fin<C>(a, r, s, p, d, GRIN_EXIT_ENTRY_REFLECT);
      return false;
    }
  } else {
    eval64<C>(m, p, nu, s.gp, s.lvl_prev);
  }
  if (!set_index(m, s, nu)) {
    fin<C>(a, r, s, p, d, GRIN_EXIT_INVALID);
    return false;
  }
  if (a.max_steps <= 0) {
    fin<C>(a, r, s, p, d, GRIN_EXIT_MAXSTEPS);
    return false;
  }
  set_pos(s, p);
  set_dir(s, d);
  s.h = (float)a.dopl * s.inv_prev;
  return true;
}


// The step would end outside the surface (by FP32): crossing (Sec. II (i)),
// in FP32 for a box, else in FP64.  Returns 0 if FP64 puts the end inside after all (take the
// ordinary step), 1 if the ray reflected and goes on, 2 if it finished.
template <class C>
__device__ __forceinline__ int surface_event(const DevMedium& m, const TraceArgs& a, int64_t r,
                                             RayF& s, float dopl_f, const float* qh) {
  if (C::bk(m) == GRIN_BOUNDARY_BOX) return surface_event_box32<C>(m, a, r, s, dopl_f, qh);
  V3 p = pos64(s), d = dir64(s);
  V3 q = axpy((double)s.h, d, p);
  if (inside64(m, q)) return 0;
  double t;
  V3 pb, nb;
  int face;
  exit64(m, p, q, t, pb, nb, face);
  cut_step<C>(s, (float)t);
  double n_prev = (double)m.base_f + (double)s.nu_prev;
  double cm = INFINITY;
  const bool refl = refract64(d, nb, n_prev / m.n_ext, C::kMG ? &cm : nullptr);
  mg_take<C>(s, 0, (float)cm);
  if (refl) {
    ++s.tir_b;
    s.h = dopl_f * s.inv_prev;
    float nu;
    eval64<C>(m, pb, nu, s.gp, s.lvl_prev);
    bool ok = set_index(m, s, nu);
    set_pos(s, pb);
    set_dir(s, d);
    if (!ok) {
      fin<C>(a, r, s, pb, d, GRIN_EXIT_INVALID);
      return 2;
    }
    if (s.steps >= a.max_steps) {
      fin<C>(a, r, s, pb, d, GRIN_EXIT_MAXSTEPS);
      return 2;
    }
    return 1;
  }
  fin<C>(a, r, s, pb, d, face);
  return 2;
}

// The index difference n_i - n_{i-1} of a step dv by the trapezoid rule on
// grad n at its ends (gp, g).
__device__ __forceinline__ float trapezoid(const float* gp, const float* g, const float* dv) {
  return 0.5f * fmaf(gp[0] + g[0], dv[0], fmaf(gp[1] + g[1], dv[1], (gp[2] + g[2]) * dv[2]));
}

// Near critical or grazing incidence: D and gamma from the same FP32 inputs
// in FP64.  Returns true on total internal reflection.
__device__ __forceinline__ bool crit64(const float* N, const float* d, float dn, float n_i,
                                       float& gamma) {
  double c64 = (double)N[0] * d[0] + (double)N[1] * d[1] + (double)N[2] * d[2];
  double om64 = (double)dn / (double)n_i;
  double mu64 = 1.0 - om64;
  double omm64 = om64 * (2.0 - om64);
  double mc64 = mu64 * c64;
  double D64 = fma(mc64, mc64, omm64);
  if (D64 <= 0.0) return true;
  gamma = (float)((c64 > 0.0 ? omm64 : -omm64) / (sqrt(D64) + fabs(mc64)));
  return false;
}

// The smooth field f = n - base and its gradient at an FP64 point.
template <class C>
__device__ __forceinline__ void field64(const DevMedium& m, V3 p, float& f, float* g) {
  const float hx = (float)p.x, hy = (float)p.y, hz = (float)p.z;
  C::field(m, hx, hy, hz, (float)(p.x - (double)hx), (float)(p.y - (double)hy),
           (float)(p.z - (double)hz), f, g[0], g[1], g[2]);
}

// The thread's tap cache as the out-of-line step sees it: its column, the
// centre tap and the cell it holds (col == nullptr: no cache).
struct TapView {
  const float* col = nullptr;
  float lb = 0.0f;
  int kx = 0, ky = 0, kz = 0;
};

// field64 from the tap cache when the point lies in the cached cell (the
// same bits, see eval_taps), else from the grid.
template <class C>
__device__ __forceinline__ void field64c(const DevMedium& m, V3 p, float& f, float* g,
                                         const TapView& tv) {
  if constexpr (C::kGrid) {
    if (tv.col) {
      const float ph[3] = {(float)p.x, (float)p.y, (float)p.z};
      const float pl[3] = {(float)(p.x - (double)ph[0]), (float)(p.y - (double)ph[1]),
                           (float)(p.z - (double)ph[2])};
      int i0[3];
      float fr[3];
      C::cell(m, ph, pl, i0, fr);
      if (i0[0] == tv.kx && i0[1] == tv.ky && i0[2] == tv.kz)
        C::taps_field(m, fr, tv.col, tv.lb, f, g[0], g[1], g[2]);
      else
        C::grid_gather(m, i0, fr, f, g[0], g[1], g[2]);
      return;
    }
  }
  field64<C>(m, p, f, g);
}

// Shell crossings within one step, at most (GRIN_TRACE_LEVEL_ROOT): a ray
// grazing a curved shell boundary can cross it back and forth at ever shorter
// intervals; after this many the rest of the step runs straight into the
// shell it ends in.
constexpr int kMaxCrossings = 16;

// The rest of a step in a layered medium with its shell crossings solved
// (GRIN_TRACE_LEVEL_ROOT; Q = P + h I is what is left of the step, h =
// (1 - used) dL0 / n_k).  Inside the shell the ray runs straight (Sec. II
// (iii)).  If Q (or the point where the segment meets the enclosing surface)
// lies in another shell, the segment first meets the boundary f = f_b of
// the ray's shell where safeguarded Newton iterations on the segment put it
// (regula falsi start; a bracket kept by the sign of f - f_b; bisection when
// a Newton step leaves it); the ray refracts there in FP64 by Eq. 8-9 with
// the isoindicial normal grad f / |grad f| and mu = n_k / n_k', or is
// totally reflected and stays in its shell (Sec. II (v)), and goes on with
// the rest of the step's optical path.  Returns false when the ray finished.
template <class C>
__device__ __forceinline__ bool level_root_step(const DevMedium& m, const TraceArgs& a, int64_t r,
                                                RayF& s, float dopl_f, const float* qh,
                                                const float* ql, const TapView& tv) {
  const V3 p = pos64(s);
  const V3 q = mk((double)qh[0] + (double)ql[0], (double)qh[1] + (double)ql[1],
                  (double)qh[2] + (double)ql[2]);
  mg_take<C>(s, 2, bnd_margin<C>(m, qh, s.h));
  double tb = 1.0;
  V3 e = q, pb, nb;
  int face = 0;
  const bool leaves = !inside64(m, q);
  if (leaves) {
    exit64(m, p, q, tb, pb, nb, face);
    e = pb;
  }
  float fE, gE[3], nuE;
  int lE;
  field64c<C>(m, e, fE, gE, tv);
  C::level(m, fE, nuE, lE);
  if (lE != s.lvl_prev && s.xc == kMaxCrossings) {
    s.lvl_prev = lE;
    if (!set_index(m, s, nuE)) {
      fin<C>(a, r, s, pos64(s), dir64(s), GRIN_EXIT_INVALID);
      return false;
    }
  }
  const int k = s.lvl_prev;
  if (lE == k) {
    s.xc = 0;
    if (leaves) {
      const int rc = surface_event<C>(m, a, r, s, dopl_f, qh);
      if (rc == 2) return false;
      if (rc == 1) return true;
    }
    // straight on to the end of the step inside the shell
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      s.ph[j] = qh[j];
      s.pl[j] = ql[j];
    }
    ++s.steps;
    s.used = 0.0f;
    s.h = dopl_f * s.inv_prev;
    if (s.steps >= a.max_steps) {
      fin<C>(a, r, s, pos64(s), dir64(s), GRIN_EXIT_MAXSTEPS);
      return false;
    }
    return true;
  }
  ++s.xc;
  // the boundary of shell k towards the end's shell: f_b; inside shell k
  // means f < f_b going up, f >= f_b going down
  const bool up = lE > k;
  const int k2 = up ? k + 1 : k - 1;
  // in FP64, as the level values below: lo + k span / L, less base
  const double L = (double)m.n_levels;
  const double fb = (m.lvl_lo - m.base) + (double)(up ? k + 1 : k) * m.lvl_span / L;
  float fP, gX[3];
  field64c<C>(m, p, fP, gX, tv);
  const V3 seg = mk(e.x - p.x, e.y - p.y, e.z - p.z);
  double lo = 0.0, hi = 1.0;
  const double a0 = (double)fP - fb, a1 = (double)fE - fb;
  double t = (a0 != a1) ? a0 / (a0 - a1) : 0.5;
  if (!(t > lo && t < hi)) t = 0.5;
  V3 x = axpy(t, seg, p);
  for (int it = 0; it < 10; ++it) {
    float fX;
    field64c<C>(m, x, fX, gX, tv);
    const double phi = (double)fX - fb;
    if (up ? phi < 0.0 : phi >= 0.0) lo = t;
    else hi = t;
    const double dphi = (double)gX[0] * seg.x + (double)gX[1] * seg.y + (double)gX[2] * seg.z;
    double tn = t - phi / dphi;
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    const bool done = fabs(tn - t) <= 1e-7 * fabs(t) + 1e-12;
    t = tn;
    x = axpy(t, seg, p);
    if (done) break;
  }
  // the ray is at x, a fraction t tb of what was left of the step further on
  set_pos(s, x);
  s.used = fmaf((float)(t * tb), 1.0f - s.used, s.used);
  // (the normal is that of the last iterate's gradient)
  const V3 gx64 = mk(gX[0], gX[1], gX[2]);
  const double gn = sqrt(dot(gx64, gx64));
  bool tir = false;
  if (gn > 0.0 && isfinite(gn)) {
    const V3 N = mk(gx64.x / gn, gx64.y / gn, gx64.z / gn);
    V3 d = dir64(s);
    mg_take<C>(s, 1, (float)fabs(dot(N, d)));
    const double nk = m.lvl_lo + ((double)k + 0.5) * m.lvl_span / L;
    const double nk2 = m.lvl_lo + ((double)k2 + 0.5) * m.lvl_span / L;
    double cm = INFINITY;
    tir = refract64(d, N, nk / nk2, C::kMG ? &cm : nullptr);
    mg_take<C>(s, 0, (float)cm);
    set_dir(s, d);
  }
  if (tir) {
    ++s.tir_i;
  } else {
    s.lvl_prev = k2;
    if (!set_index(m, s, C::shell_nu(m, k2))) {
      fin<C>(a, r, s, pos64(s), dir64(s), GRIN_EXIT_INVALID);
      return false;
    }
  }
  // the rest of the step's optical path in the (new) shell
  s.h = (1.0f - s.used) * dopl_f * s.inv_prev;
  return true;
}

// One VRT step of an active ray, every case tested in order; returns false
// when the ray finished.  Taken only when the fast step below meets a case
// it does not handle.
template <class C, bool LAYERED>
__device__ __noinline__ bool step_slow(const DevMedium& m, const TraceArgs& a, int64_t r,
                                       RayF& s, float dopl_f, TapView tv = TapView()) {
  // the exact pair form of step_point, on a normalised position
  if constexpr (C::kLazyPos) norm_pos(s);
  float qh[3], ql[3], dv[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dv[k] = s.h * s.d[k];
    float y = fmaf(s.h, s.d[k], fmaf(s.h, s.dl[k], s.pl[k]));
    float t = s.ph[k] + y;
    ql[k] = y - (t - s.ph[k]);
    qh[k] = t;
  }
  if constexpr (LAYERED)
    if (a.flags & GRIN_TRACE_LEVEL_ROOT) return level_root_step<C>(m, a, r, s, dopl_f, qh, ql, tv);
  mg_take<C>(s, 2, bnd_margin<C>(m, qh, s.h));
  if (GRIN_UNLIKELY(!C::inside(m, qh))) {
    int rc = surface_event<C>(m, a, r, s, dopl_f, qh);
    if (rc == 2) return false;
    if (rc == 1) return true;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s.ph[k] = qh[k];
    s.pl[k] = ql[k];
  }
  ++s.steps;
  float nu_i, g[3], u_i;
  int lvl_i;
  C::eval(m, qh[0], qh[1], qh[2], ql[0], ql[1], ql[2], nu_i, g[0], g[1], g[2], lvl_i,
          C::kMG ? &u_i : nullptr);
  if (LAYERED) mg_take<C>(s, 3, lvl_margin(m, u_i));
  const float n_i = m.base_f + nu_i;
  if (GRIN_UNLIKELY(!(isfinite(n_i) && n_i > 0.0f))) {
    fin<C>(a, r, s, pos64(s), dir64(s), GRIN_EXIT_INVALID);
    return false;
  }
  const float inv_n = 1.0f / n_i;
  float gn2 = fmaf(g[0], g[0], fmaf(g[1], g[1], g[2] * g[2]));
  if (GRIN_UNLIKELY((LAYERED && lvl_i == s.lvl_prev) || gn2 == 0.0f || !isfinite(gn2))) {
    s.h = dopl_f * inv_n;  // Sec. II (ii)/(iii)
  } else {
    float ri = rsqrtf(gn2);
    float N[3] = {g[0] * ri, g[1] * ri, g[2] * ri};
    float c = fmaf(N[0], s.d[0], fmaf(N[1], s.d[1], N[2] * s.d[2]));
    mg_take<C>(s, 1, fabsf(c));
    if (GRIN_UNLIKELY(c == 0.0f)) {
      // Sec. II (iv): circular arc from one extra index sample along N.
      float hi = dopl_f * inv_n;
      float nu2, g2x, g2y, g2z;
      int l2;
      C::eval(m, fmaf(hi, N[0], qh[0]), fmaf(hi, N[1], qh[1]), fmaf(hi, N[2], qh[2]), ql[0], ql[1],
              ql[2], nu2, g2x, g2y, g2z, l2);
      float k = (nu2 - nu_i) * 0.5f * inv_n;
      float w = fmaf(-k, k, 1.0f);
      float a0 = w > 0.0f ? sqrtf(w) : 0.0f;
      float nd[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) nd[j] = fmaf(a0, s.d[j], k * N[j]);
      renorm(nd);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        s.d[j] = nd[j];
        s.dl[j] = 0.0f;
      }
      s.h = hi;
    } else {
      float dn = nu_i - s.nu_prev;
      if (!LAYERED) {
        float dt = trapezoid(s.gp, g, dv);
        if (isfinite(dt)) dn = dt;
      }
      const float om = dn * inv_n;           // 1 - mu
      const float mu = 1.0f - om;
      const float omm = om * (2.0f - om);    // 1 - mu^2
      const float mc = mu * c;
      const float D = fmaf(mc, mc, omm);
      mg_take<C>(s, 0, crit_margin(c, mu, omm, D));
      bool tir = D <= 0.0f;
      float gamma = (c > 0.0f ? omm : -omm) / (sqrtf(fmaxf(D, 0.0f)) + fabsf(mc));
      if (GRIN_UNLIKELY(fabsf(D) <= kCritBand * (fabsf(omm) + mc * mc)))
        tir = crit64(N, s.d, dn, n_i, gamma);
      // Eq. 8, R = I + (gamma N - (1 - mu) I), or Sec. II (v), R = I - 2 c N
      // with a step of dL0 / n_{i-1}
      const float kn = tir ? -2.0f * c : gamma;
      const float kd = tir ? 0.0f : -om;
#pragma unroll
      for (int j = 0; j < 3; ++j) add_ff(s.d[j], s.dl[j], fmaf(kn, N[j], kd * s.d[j]));
      s.h = dopl_f * (tir ? s.inv_prev : inv_n);
      s.tir_i += tir ? 1 : 0;
    }
  }
  s.nu_prev = nu_i;
  s.inv_prev = inv_n;
  s.lvl_prev = lvl_i;
  s.gp[0] = g[0];
  s.gp[1] = g[1];
  s.gp[2] = g[2];
  if (GRIN_UNLIKELY(s.steps >= a.max_steps)) {
    fin<C>(a, r, s, pos64(s), dir64(s), GRIN_EXIT_MAXSTEPS);
    return false;
  }
  return true;
}

// The common step: the end point is inside, n is usable, N.I is nonzero and
// D is above the near-critical band, so the step refracts (or, in a layered
// medium, the level did not change and it goes straight on).
// Everything is computed without a branch and one flag routes the rare cases
// (surface crossing, invalid n, zero or undefined gradient, tangency,
// D at or below the near-critical band, the step limit) to step_slow, which
// redoes the step from the unchanged state.
//
// step_point gives the end point Q = P + h I; step_from finishes the step from n and grad n at Q, and commit_point makes
// Q the ray's point.  Q is the pair qh + ql by Fast2Sum, or, with a lazily
// carried position, the low part alone moves: ql = pl + h I and qh =
// fl(ph + ql), the rounded point the field is read at.  The low part then
// grows by a quantum's steps at most (run_quantum normalises the pair at
// each quantum's start, step_slow before it steps), so each step rounds at
// an ulp of that sum instead of an ulp of the step: still well below the
// rounding of qh itself.
template <class C>
__device__ __forceinline__ void step_point(const RayF& s, float* qh, float* ql) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float y = fmaf(s.h, s.d[k], fmaf(s.h, s.dl[k], s.pl[k]));
    if constexpr (C::kLazyPos) {
      ql[k] = y;
      qh[k] = s.ph[k] + y;
    } else {
      float t = s.ph[k] + y;
      ql[k] = y - (t - s.ph[k]);
      qh[k] = t;
    }
  }
}

template <class C>
__device__ __forceinline__ void commit_point(RayF& s, const float* qh, const float* ql) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if constexpr (!C::kLazyPos) s.ph[k] = qh[k];
    s.pl[k] = ql[k];
  }
}

template <class C, bool LAYERED>
__device__ __forceinline__ bool step_from(const DevMedium& m, const TraceArgs& a, int64_t r,
                                          RayF& s, float dopl_f, const float* qh,
                                          const float* ql, float nu_i,
                                          const float* g, int lvl_i, float u_i = 0.5f,
                                          const TapView& tv = TapView()) {
  const bool in = C::inside(m, qh);
  const float n_i = m.base_f + nu_i;
  // (the fast step's two divisions take the approximate reciprocal without
  // the full-range scaling of '/': both divisors are of order one here, and
  // any other value routes the step to step_slow)
  const float inv_n = __fdividef(1.0f, n_i);
  const float gn2 = fmaf(g[0], g[0], fmaf(g[1], g[1], g[2] * g[2]));
  const bool homog = LAYERED && lvl_i == s.lvl_prev;
  const float ri = rsqrtf(gn2);
  float N[3] = {g[0] * ri, g[1] * ri, g[2] * ri};
  const float c = fmaf(N[0], s.d[0], fmaf(N[1], s.d[1], N[2] * s.d[2]));
  // 1 - mu = (n_i - n_{i-1}) / n_i, the index difference by the trapezoid
  // rule as (grad n_{i-1} + grad n_i) . I times h / 2 (layered media: the
  // level values)
  float om;
  if constexpr (!LAYERED)
    om = fmaf(s.gp[0] + g[0], s.d[0], fmaf(s.gp[1] + g[1], s.d[1], (s.gp[2] + g[2]) * s.d[2])) *
         (0.5f * s.h) * inv_n;
  else
    om = (nu_i - s.nu_prev) * inv_n;
  const float mu = 1.0f - om;
  const float omm = om * (2.0f - om);  // 1 - mu^2
  const float mc = mu * c;
  const float D = fmaf(mc, mc, omm);
  const float gamma = __fdividef(c > 0.0f ? omm : -omm, sqrtf(D) + fabsf(mc));
  // A zero, infinite or undefined gradient, or an undefined index
  // difference, makes D a NaN (rsqrt(0) = inf and 0 * inf, or inf - inf),
  // which fails the comparison with the near-critical band; a gradient that
  // overflows while its components stay finite gives N = 0 and c == 0.
  const bool special =
      !in || !(n_i > 0.0f && n_i < INFINITY) || s.steps + 1 >= a.max_steps ||
      (!homog && (c == 0.0f || !(D > kCritBand * (fabsf(omm) + mc * mc)))) ||
      (LAYERED && !homog && (a.flags & GRIN_TRACE_LEVEL_ROOT));
  if (GRIN_UNLIKELY(special)) {
    // out of line, on a copy: only the copy's address escapes, the live
    // state stays in registers
    RayF t = s;
    bool alive = step_slow<C, LAYERED>(m, a, r, t, dopl_f, tv);
    s = t;
    return alive;
  }
  if constexpr (C::kMG) {
    mg_take<C>(s, 2, bnd_margin<C>(m, qh, s.h));
    if (LAYERED && !(a.flags & GRIN_TRACE_LEVEL_ROOT)) mg_take<C>(s, 3, lvl_margin(m, u_i));
    if (!homog) {
      mg_take<C>(s, 1, fabsf(c));
      mg_take<C>(s, 0, crit_margin(c, mu, omm, D));
    }
  }
  commit_point<C>(s, qh, ql);
  ++s.steps;
  // Eq. 8, R = I + (gamma N - (1 - mu) I); Sec. II (v), R = I - 2 c N with a
  // step of dL0 / n_{i-1}; inside one shell of a layered medium, straight on
  const float kn = homog ? 0.0f : gamma;
  const float kd = homog ? 0.0f : -om;
#pragma unroll
  for (int j = 0; j < 3; ++j) add_ff(s.d[j], s.dl[j], fmaf(kn, N[j], kd * s.d[j]));
  s.h = dopl_f * inv_n;
  if constexpr (LAYERED) {
    s.used = 0.0f;
    s.xc = 0;
  }
  s.nu_prev = nu_i;
  s.inv_prev = inv_n;
  s.lvl_prev = lvl_i;
  s.gp[0] = g[0];
  s.gp[1] = g[1];
  s.gp[2] = g[2];
  return true;
}

template <class C, bool LAYERED>
__device__ __forceinline__ bool step_ray(const DevMedium& m, const TraceArgs& a, int64_t r,
                                         RayF& s, float dopl_f) {
  float qh[3], ql[3];
  step_point<C>(s, qh, ql);
  float nu_i, g[3], u_i = 0.5f;
  int lvl_i;
  C::eval(m, qh[0], qh[1], qh[2], ql[0], ql[1], ql[2], nu_i, g[0], g[1], g[2], lvl_i,
          C::kMG ? &u_i : nullptr);
  return step_from<C, LAYERED>(m, a, r, s, dopl_f, qh, ql, nu_i, g, lvl_i, u_i);
}

// Warp-collective: the lanes in `need` get their column of the tap cache
// refilled for the cell in their key[] (the 64 edge-clamped stencil samples
// of grid_gather, minus the centre tap, which the lane keeps in lb).  The
// whole warp loads one such lane's taps at a time, lane 2 r + e filling the
// pair of floats e of cache row r = 2 (4 p + b) + h: the samples at
// x = 2 h + e of stencil row b in the z planes 2 p and 2 p + 1 (the layout
// taps_field reads).  Lanes 4 j .. 4 j + 3 read four x-adjacent samples of
// one grid row, and lane 5 holds the centre tap (kx, ky, kz) as its second,
// so a refill costs the warp two gathers instead of the lane's 64.
__device__ __forceinline__ void tap_fill(const DevMedium& m, bool need, const int* key,
                                         float& lb, float* taps, unsigned lane) {
  unsigned mask = __ballot_sync(0xffffffffu, need);
  if (!mask) return;
  __syncwarp();  // the owners' reads of their old taps come first
  const int row = (int)(lane >> 1), e = (int)(lane & 1u);
  const int p = row >> 3, b = (row >> 1) & 3, x = 2 * (row & 1) + e;
  const int wbase = (int)(threadIdx.x & ~31u);
  while (mask) {
    const int src = __ffs(mask) - 1;
    mask &= mask - 1u;
    const int kx = __shfl_sync(0xffffffffu, key[0], src);
    const int ky = __shfl_sync(0xffffffffu, key[1], src);
    const int kz = __shfl_sync(0xffffffffu, key[2], src);
    const int iz0 = min(max(kz - 1 + 2 * p, 0), m.nz - 1);
    const int iz1 = min(max(kz + 2 * p, 0), m.nz - 1);
    const int iy = min(max(ky - 1 + b, 0), m.ny - 1);
    const int ix = min(max(kx - 1 + x, 0), m.nx - 1);
    const float v0 = __ldg(m.grid + GRIN_IDX(m, ((int64_t)iz0 * m.ny + iy) * m.nx + ix, m.grid_n, kSiteGridMixed));
    const float v1 = __ldg(m.grid + GRIN_IDX(m, ((int64_t)iz1 * m.ny + iy) * m.nx + ix, m.grid_n, kSiteGridMixed));
    const float sub = __shfl_sync(0xffffffffu, v1, 5);  // plane 1, row 1, x = kx
    if ((int)lane == src) lb = sub;
    *reinterpret_cast<float2*>(
        taps + GRIN_IDX(m, row * kTapRow + (wbase + src) * 4 + 2 * e, 16 * kTapRow - 1, kSiteTapCache)) =
        make_float2(v0 - sub, v1 - sub);
  }
  __syncwarp();
}

// Up to kStepQuantum steps of the lane's ray; returns how many rays ended.
// On a gridded medium the fast step reads its taps from the lane's column of
// the tap cache (key[] = the cell they belong to): a ray stays in one cell
// for many steps, and a shared-memory row read replaces the gathers.  The
// out-of-line cases still gather from the grid, with the same result.
template <class C, bool LAYERED>
__device__ __forceinline__ unsigned run_quantum(const DevMedium& m, const TraceArgs& a,
                                                int64_t ray, RayF& s, bool& active,
                                                float dopl_f, int* key, float& lb, float* taps,
                                                unsigned lane) {
  unsigned ended = 0;
  if constexpr (!C::kGrid) {
    if (active) norm_pos(s);
    // (four steps an iteration: the measured optimum of 1, 2, 4 and 8)
#pragma unroll 4
    for (int j = 0; j < kStepQuantum; ++j) {
      if (active) {
        active = step_ray<C, LAYERED>(m, a, ray, s, dopl_f);
        if (!active) ++ended;
      }
    }
  } else {
    const float* col = taps + threadIdx.x * 4;
#pragma unroll 1
    for (int j = 0; j < kStepQuantum; ++j) {
      float qh[3], ql[3], fr[3];
      bool need = false;
      if (active) {
        step_point<C>(s, qh, ql);
        int i0[3];
        C::cell(m, qh, ql, i0, fr);
        need = i0[0] != key[0] || i0[1] != key[1] || i0[2] != key[2];
        key[0] = i0[0];
        key[1] = i0[1];
        key[2] = i0[2];
      }
      tap_fill(m, need, key, lb, taps, lane);
      if (active) {
        float nu_i, g[3], u_i = 0.5f;
        int lvl_i;
        C::eval_taps(m, fr, col, lb, nu_i, g[0], g[1], g[2], lvl_i, C::kMG ? &u_i : nullptr);
        TapView tv;
        if constexpr (LAYERED) {
          // (only the shell-crossing solve reads it)
          tv.col = col;
          tv.lb = lb;
          tv.kx = key[0];
          tv.ky = key[1];
          tv.kz = key[2];
        }
        active = step_from<C, LAYERED>(m, a, ray, s, dopl_f, qh, ql, nu_i, g, lvl_i, u_i, tv);
        if (!active) ++ended;
      }
    }
  }
  return ended;
}

template <class C, bool LAYERED>
__global__ void __launch_bounds__(128, LAYERED ? C::kMinBlocksLayered : C::kMinBlocks) k_trace_mixed(DevMedium m, TraceArgs a,
                                                     unsigned long long* queue) {
  const unsigned lane = threadIdx.x & 31u;
  const float dopl_f = (float)a.dopl;
  __shared__ __align__(16) float taps[C::kGrid ? 16 * kTapRow : 4];
  int key[3] = {INT_MIN, INT_MIN, INT_MIN};
  float lb = 0.0f;  // centre tap of the cached cell
  RayF s;
  bool active = false;
  bool exhausted = false;
  int64_t ray = 0;
  for (;;) {
    const unsigned need = __ballot_sync(0xffffffffu, !active);
    if (need && !exhausted) {
      const int leader = __ffs(need) - 1;
      const unsigned cnt = __popc(need);
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(queue, (unsigned long long)cnt);
      base = __shfl_sync(0xffffffffu, base, leader);
      exhausted = base + cnt >= (unsigned long long)a.count;
      if (!active) {
        const unsigned long long rr = base + __popc(need & ((1u << lane) - 1u));
        if (rr < (unsigned long long)a.count) {
          ray = a.perm ? (int64_t)GRIN_IDX(m, a.perm[rr], a.count, kSiteRay) : (int64_t)rr;
          active = init_ray<C>(m, a, ray, s);
        }
      }
    }
    if (!__any_sync(0xffffffffu, active)) {
      if (exhausted) break;
      continue;
    }
    run_quantum<C, LAYERED>(m, a, ray, s, active, dopl_f, key, lb, taps, lane);
  }
}

template <int PC, bool GRID, bool LAYERED, int BK, int FORM, bool MG = false>
static int launch_t(const DevMedium& m, const TraceArgs& a, unsigned long long* queue,
                    cudaStream_t st, int sm_count) {
  using C = Cfg<PC, GRID, LAYERED, BK, FORM, MG>;
  auto kern = k_trace_mixed<C, LAYERED>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t warps_needed = (a.count + 31) / 32;
  int block = 128;
  int64_t blocks = (int64_t)sm_count * per_sm;
  // Small batches: one warp per block so that the warps spread over all SMs.
  if (warps_needed <= (int64_t)sm_count * 4) {
    block = 32;
    blocks = warps_needed;
  } else {
    blocks = blocks < (warps_needed + 3) / 4 ? blocks : (warps_needed + 3) / 4;
  }
  if (cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st) != cudaSuccess) return GRIN_ERR_CUDA;
  return launch_kernel(kern, (unsigned)blocks, block, st, m, a, queue);
}

template <int PC, bool GRID>
static int launch_pc(const DevMedium& m, const TraceArgs& a, unsigned long long* q,
                     cudaStream_t s, int sm) {
  // decision margins: the kernels with run-time boundary and form, which
  // also keep the margins
  if (a.margin)
    return m.n_levels > 0 ? launch_t<PC, GRID, true, -1, -1, true>(m, a, q, s, sm)
                          : launch_t<PC, GRID, false, -1, -1, true>(m, a, q, s, sm);
  if (m.n_levels > 0) {
    if constexpr (GRID)
      if (m.bkind == GRIN_BOUNDARY_BOX)
        return launch_t<PC, GRID, true, GRIN_BOUNDARY_BOX, GRIN_FORM_LINEAR>(m, a, q, s, sm);
    return launch_t<PC, GRID, true, -1, -1>(m, a, q, s, sm);
  }
  const bool fast = m.bkind == GRIN_BOUNDARY_BOX && (GRID || m.form == GRIN_FORM_LINEAR);
  return fast ? launch_t<PC, GRID, false, GRIN_BOUNDARY_BOX, GRIN_FORM_LINEAR>(m, a, q, s, sm)
              : launch_t<PC, GRID, false, -1, -1>(m, a, q, s, sm);
}

int launch_mixed(const DevMedium& m, const TraceArgs& a, unsigned long long* queue,
                 cudaStream_t s, int sm_count) {
  if (m.kind == GRIN_MEDIUM_GRID) return launch_pc<0, true>(m, a, queue, s, sm_count);
  switch (m.pclass) {
    case kSpherical: return launch_pc<1, false>(m, a, queue, s, sm_count);
    case kN2P: return launch_pc<3, false>(m, a, queue, s, sm_count);
    case kPoly2: return launch_pc<2, false>(m, a, queue, s, sm_count);
    case kPoly4: return launch_pc<4, false>(m, a, queue, s, sm_count);
    default: return launch_pc<6, false>(m, a, queue, s, sm_count);
  }
}

// ------------------------------------------------------------- serving
//
// One tick of the continuous-batching server: the job's resident slots (one
// per thread) each run up to `quantum` steps, claiming the job's next ray
// from counters[0] whenever their ray ends; finished rays are counted into
// counters[1].  The full per-ray FP32 state stays in HBM between ticks, so
// the arithmetic of a ray does not depend on how its steps are split into
// ticks: results are bitwise those of grin_trace.

struct SlotState {
  RayF s;
  long long ray;
  int active;
  int pad;
};

template <class C, bool LAYERED>
__global__ void __launch_bounds__(128, LAYERED ? C::kMinBlocksLayered : C::kMinBlocks) k_serve_tick(DevMedium m, TraceArgs a,
                                                                   SlotState* slots,
                                                                   unsigned long long* counters,
                                                                   int quantum) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31u;
  const float dopl_f = (float)a.dopl;
  SlotState* me = slots + t;
  __shared__ __align__(16) float taps[C::kGrid ? 16 * kTapRow : 4];
  int key[3] = {INT_MIN, INT_MIN, INT_MIN};
  float lb = 0.0f;  // centre tap of the cached cell
  RayF s = me->s;
  bool active = me->active != 0;
  int64_t ray = me->ray;
  bool exhausted = false;
  unsigned done = 0;
  for (int k = 0; k < quantum; k += kStepQuantum) {
    const unsigned need = __ballot_sync(0xffffffffu, !active);
    if (need && !exhausted) {
      const int leader = __ffs(need) - 1;
      const unsigned cnt = __popc(need);
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(counters, (unsigned long long)cnt);
      base = __shfl_sync(0xffffffffu, base, leader);
      exhausted = base + cnt >= (unsigned long long)a.count;
      if (!active) {
        const unsigned long long rr = base + __popc(need & ((1u << lane) - 1u));
        if (rr < (unsigned long long)a.count) {
          ray = a.perm ? (int64_t)GRIN_IDX(m, a.perm[rr], a.count, kSiteRay) : (int64_t)rr;
          active = init_ray<C>(m, a, ray, s);
          if (!active) ++done;
        }
      }
    }
    if (!__any_sync(0xffffffffu, active)) {
      if (exhausted) break;
      continue;
    }
    done += run_quantum<C, LAYERED>(m, a, ray, s, active, dopl_f, key, lb, taps, lane);
  }
  me->s = s;
  me->active = active ? 1 : 0;
  me->ray = ray;
  done = __reduce_add_sync(0xffffffffu, done);
  if (lane == 0 && done) atomicAdd(counters + 1, (unsigned long long)done);
}

size_t serve_slot_bytes() { return sizeof(SlotState); }

template <int PC, bool GRID, bool LAYERED, int BK, int FORM>
static int tick_t(const DevMedium& m, const TraceArgs& a, void* slots, int nslots,
                  unsigned long long* counters, int quantum, cudaStream_t st) {
  using C = Cfg<PC, GRID, LAYERED, BK, FORM>;
  return launch_kernel(k_serve_tick<C, LAYERED>, (unsigned)(nslots / 128), 128, st, m, a,
                       (SlotState*)slots, counters, quantum);
}

template <int PC, bool GRID>
static int tick_pc(const DevMedium& m, const TraceArgs& a, void* slots, int nslots,
                   unsigned long long* counters, int quantum, cudaStream_t st) {
  if (m.n_levels > 0) {
    if constexpr (GRID)
      if (m.bkind == GRIN_BOUNDARY_BOX)
        return tick_t<PC, GRID, true, GRIN_BOUNDARY_BOX, GRIN_FORM_LINEAR>(m, a, slots, nslots,
                                                                          counters, quantum, st);
    return tick_t<PC, GRID, true, -1, -1>(m, a, slots, nslots, counters, quantum, st);
  }
  const bool fast = m.bkind == GRIN_BOUNDARY_BOX && (GRID || m.form == GRIN_FORM_LINEAR);
  return fast ? tick_t<PC, GRID, false, GRIN_BOUNDARY_BOX, GRIN_FORM_LINEAR>(m, a, slots, nslots,
                                                                             counters, quantum, st)
              : tick_t<PC, GRID, false, -1, -1>(m, a, slots, nslots, counters, quantum, st);
}

int launch_serve_tick(const DevMedium& m, const TraceArgs& a, void* slots, int nslots,
                      unsigned long long* counters, int quantum, cudaStream_t s) {
  if (nslots <= 0 || nslots % 128 != 0 || quantum <= 0) return GRIN_ERR_INVALID_ARG;
  if (m.kind == GRIN_MEDIUM_GRID) return tick_pc<0, true>(m, a, slots, nslots, counters, quantum, s);
  switch (m.pclass) {
    case kSpherical: return tick_pc<1, false>(m, a, slots, nslots, counters, quantum, s);
    case kN2P: return tick_pc<3, false>(m, a, slots, nslots, counters, quantum, s);
    case kPoly2: return tick_pc<2, false>(m, a, slots, nslots, counters, quantum, s);
    case kPoly4: return tick_pc<4, false>(m, a, slots, nslots, counters, quantum, s);
    default: return tick_pc<6, false>(m, a, slots, nslots, counters, quantum, s);
  }
}

}  // namespace grin
