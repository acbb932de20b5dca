/*
 * vrt_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow FP64 CPU tracer of Vectorial Ray Tracing (VRT) in gradient-index
 * media (Chavez-Islas et al., "Generalized vectorial ray tracing for optical
 * analysis and design in freeform gradient-index media", Sec. II).  It exists
 * to check the CUDA library; only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header or
 * constant with the CUDA path.
 *
 * Conventions (the oracle's own; they describe the same problem the library
 * solves):
 *   - medium kinds: 0 = polynomial field, 1 = sampled grid (Catmull-Rom
 *     tricubic), either optionally quantised into layered shells;
 *   - polynomial forms: 0: n = p, 1: n = sqrt(p), 2: n = c / p;
 *   - boundary kinds: 0 = box, 1 = sphere, 2 = finite cylinder along z;
 *   - exit ids: >= 0 face id, -1 miss, -2 reflected at entry, -3 step limit,
 *     -4 invalid ray.
 */
#ifndef VRT_ORACLE_H
#define VRT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t kind;          /* 0 polynomial, 1 grid, 2 spherical freeform (Sec. V),
                            3 N2P cylinder lens (Sec. VI) */
  int32_t form;          /* 0 n=p, 1 n=sqrt(p), 2 n=form_c/p */
  double form_c;
  int32_t degree;        /* polynomial total degree */
  const double* coeffs;  /* graded-lex monomials of the normalised coordinates;
                            kind 2: a0, a1, a2, a3; kind 3: R, F, beta, gamma
                            (axis through off[0], off[1], parallel to z) */
  double off[3];         /* x' = (x - off) / scale */
  double scale[3];
  int32_t nx, ny, nz;    /* grid sizes, x fastest */
  const float* grid;     /* host samples */
  double origin[3];      /* position of sample (0,0,0) */
  double spacing[3];
  int32_t n_levels;      /* 0: continuous; L > 0: L isoindicial shells */
  double level_lo, level_hi;
  int32_t bkind;         /* 0 box, 1 sphere, 2 cylinder */
  double b[8];           /* box: lo[3],hi[3]; sphere: c[3],R; cylinder: cx,cy,R,z0,z1 */
  double n_ext;          /* index of the surrounding homogeneous medium */
} orc_medium;

typedef struct {
  double dopl;           /* Delta L_0: optical path per step */
  int32_t max_steps;
  int32_t flags;         /* 0, or ORC_LEVEL_ROOT (below) */
  /* Conditioning probe, for judging which rays a less precise tracer can be
   * held to (0, 0.0 for the method itself): index_rule 1 takes the index
   * difference n_i - n_{i-1} of a refraction (continuous media) by the
   * trapezoid rule on grad n along the step instead of from the two point
   * values; perturb > 0 adds to every sampled gradient a pseudo-random
   * vector of at most perturb |grad n| per component (SplitMix64 of seed,
   * ray index, step and axis). */
  int32_t index_rule;
  double perturb;
  uint64_t seed;
} orc_params;

/* Per-ray decision margins: min distance of |N.I| from its critical value
 * over refraction tests, min |N.I| over gradient steps, min distance of a step
 * endpoint to the boundary in units of the step, min distance of the level
 * coordinate to a shell boundary (the integers 1 .. n_levels - 1). */
enum { ORC_M_CRIT = 0, ORC_M_TAN = 1, ORC_M_BND = 2, ORC_M_LEVEL = 3, ORC_NM = 4 };

/* orc_params.flags: for layered media, refract where the ray meets a shell
 * boundary (found by bisection on the step) instead of at the first sampled
 * point beyond it, and go on with the rest of the step's optical path. */
enum { ORC_LEVEL_ROOT = 1 };
/* Shell crossings within one step, at most (then the rest of the step runs
 * straight and the ray takes the shell it ends in). */
enum { ORC_MAX_CROSSINGS = 16 };

/* Index and its gradient at a point.  Returns 0. */
int orc_medium_eval(const orc_medium* m, const double* P, double* n, double* g);

/* Trace n rays (origins o[3n], directions d[3n], row-major xyz) with nthreads
 * POSIX threads.  Outputs: P_out[3n], d_out[3n], opl[n], exit_id[n], steps[n],
 * tir_int[n], tir_bnd[n], margins[4n]. */
int orc_trace_batch(const orc_medium* m, const orc_params* p, int64_t n,
                    const double* o, const double* d, double* P_out,
                    double* d_out, double* opl, int32_t* exit_id,
                    int32_t* steps, int32_t* tir_int, int32_t* tir_bnd,
                    double* margins, int32_t nthreads);

/* One ray, recording every point reached inside the medium (entry point
 * first) into path[3*cap].  *path_len receives the number recorded. */
int orc_trace_path(const orc_medium* m, const orc_params* p, const double* o,
                   const double* d, double* P_out, double* d_out, double* opl,
                   int32_t* exit_id, int32_t* steps, int32_t* tir_int,
                   int32_t* tir_bnd, double* margins, double* path,
                   int64_t cap, int64_t* path_len);

/* Forward-mode derivatives (tangents) of each ray's exit point, direction
 * and optical path with respect to nc parameters, in a box without layering:
 * every coefficient of a polynomial medium with n = p (nc = (degree + 1)
 * (degree + 2)(degree + 3) / 6; nparams and params unused), or the nparams
 * grid samples params[] (flat index, x fastest) of a grid medium (nc =
 * nparams).  The values and decisions are those of orc_trace_batch, each
 * continuous quantity carrying its derivative through the step (Eq. 2-9), the
 * exit crossing and the boundary refraction.  tP[3 nc n] and td[3 nc n] are
 * laid out ray, then parameter, then component; topl[nc n].  flag[i] = 1
 * when ray i met tangential incidence (N.I == 0) or a crossing fraction
 * clamped to [0, 1], which the tangents do not follow.  Returns -1 for any
 * other medium or an out-of-range sample, else 0. */
int orc_trace_tangent(const orc_medium* m, const orc_params* p, int64_t n,
                      const double* o, const double* d, int32_t nparams,
                      const int64_t* params, double* P_out, double* d_out,
                      double* opl, int32_t* exit_id, int32_t* steps, double* tP,
                      double* td, double* topl, int32_t* flag, int32_t nthreads);

#ifdef __cplusplus
}
#endif
#endif
