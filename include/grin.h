/*
 * grin.h -- C ABI of the B300 Vectorial Ray Tracing (VRT) library.
 *
 * The library traces batches of independent rays through a gradient-index
 * (GRIN) medium bounded by a closed surface in a homogeneous surround, by the
 * method of Chavez-Islas et al., "Generalized vectorial ray tracing for
 * optical analysis and design in freeform gradient-index media":
 *   - each step advances the point by Delta_i = Delta L_0 / n_i along the
 *     current direction (Sec. II, Eq. 2-3), so every full step adds Delta L_0
 *     of optical path;
 *   - at each new point P_i the direction is refracted by the vectorial Snell
 *     law R = mu I + gamma N (Eq. 1, 8-9) with mu = n(P_{i-1}) / n(P_i) and
 *     N = grad n / |grad n| (Eq. 5);
 *   - special cases (Sec. II (i)-(v)): the enclosing-surface normal at the
 *     boundary, straight steps where grad n is zero or undefined, a circular
 *     arc at tangential incidence, and total internal reflection (TIR) with a
 *     step of Delta L_0 / n_{i-1}.
 *
 * Conventions shared by every call:
 *   - every function returns a grin_status (0 = success); nothing throws;
 *   - per-ray problems (NaN or zero direction, n <= 0) are reported in the
 *     ray's exit id (GRIN_EXIT_INVALID) and do not fail the batch; reaching
 *     max_steps is an outcome (GRIN_EXIT_MAXSTEPS), not an error;
 *   - ray and output arrays of grin_trace are caller-owned DEVICE memory on
 *     the context's GPU; grin_trace_host takes HOST memory instead; media,
 *     contexts and servers are library-owned and freed by their destroy call;
 *   - grin_trace is asynchronous on the caller's CUDA stream (NULL = the
 *     legacy default stream); kernel faults surface at the next synchronising
 *     call on that stream;
 *   - a context and its media may be used from one host thread at a time,
 *     except the grin_serve_* calls, which are thread-safe.
 */
#ifndef GRIN_H
#define GRIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grin_ctx_s* grin_ctx;
typedef struct grin_medium_s* grin_medium;
typedef struct grin_server_s* grin_server;

typedef enum {
  GRIN_OK = 0,
  GRIN_ERR_INVALID_ARG = -1,   /* a NULL pointer, bad enum or size */
  GRIN_ERR_OOM = -2,           /* device or host allocation failed */
  GRIN_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  GRIN_ERR_NOT_IMPLEMENTED = -4,
  GRIN_ERR_TIMEOUT = -5,       /* a bounded wait ran out */
  GRIN_ERR_BUSY = -6,          /* admission refused (serving); context still owns objects */
  GRIN_ERR_NOT_FOUND = -7,     /* unknown job id (serving) */
  GRIN_ERR_CANCELLED = -8,     /* job cancelled (serving) */
  GRIN_ERR_CHECKED_BOUNDS = -9 /* the bounds-checked build caught an out-of-range
                                  index in a kernel (see grin_checked_status) */
} grin_status;

/* Exit ids written per ray.  Non-negative ids name the face the ray left by:
 * box faces 0..5 = -x, +x, -y, +y, -z, +z; sphere 0; cylinder side 0, the
 * z0 end 1, the z1 end 2. */
enum {
  GRIN_EXIT_MISS = -1,          /* started outside and never met the surface */
  GRIN_EXIT_ENTRY_REFLECT = -2, /* totally reflected at the entry point */
  GRIN_EXIT_MAXSTEPS = -3,      /* max_steps interior steps taken */
  GRIN_EXIT_INVALID = -4        /* non-finite or zero direction, n <= 0 */
};

enum { GRIN_MEDIUM_POLY = 0, GRIN_MEDIUM_GRID = 1, GRIN_MEDIUM_SPHERICAL = 2, GRIN_MEDIUM_N2P = 3 };
enum { GRIN_FORM_LINEAR = 0, GRIN_FORM_SQRT = 1, GRIN_FORM_RECIP = 2 };
enum { GRIN_BOUNDARY_BOX = 0, GRIN_BOUNDARY_SPHERE = 1, GRIN_BOUNDARY_CYLINDER = 2 };
enum { GRIN_F32 = 0, GRIN_F64 = 1 };
enum { GRIN_PREC_FP64 = 0, GRIN_PREC_FP32_MIXED = 1, GRIN_PREC_FP64_FAST = 2 };

#define GRIN_MAX_DEGREE 6
#define GRIN_MAX_LEVELS 65536

/*
 * Medium description (copied by grin_medium_create; the caller may free its
 * buffers afterwards).  The index field n(x, y, z) is either
 *   - GRIN_MEDIUM_POLY: a polynomial p of degree <= GRIN_MAX_DEGREE in the
 *     normalised coordinates x' = (x - norm_offset) / norm_scale (the
 *     normalisation style of the corrector lens, Sec. V), with monomials
 *     x'^i y'^j z'^k in graded-lex order (total degree ascending; within one
 *     degree i descending, then j descending), C(degree+3, 3) host doubles
 *     in `coeffs`; `form` maps p to n: n = p, n = sqrt(p) (Luneburg lens,
 *     parabolic fiber of Eq. 22) or n = form_c / p (Maxwell fish-eye);
 *   - GRIN_MEDIUM_GRID: float32 samples grid[(k * ny + j) * nx + i] at
 *     origin + (i, j, k) * spacing (host memory, or device memory if
 *     grid_on_device), read by Catmull-Rom tricubic interpolation (Keys 1981)
 *     with edge-clamped taps and its analytic gradient;
 *   - GRIN_MEDIUM_SPHERICAL: the spherical freeform field of Sec. V,
 *     p = a0 + a1 G1 + a2 G2 + a3 G3 with G1 = 0.3 (r^2 - 1),
 *     G2 = r cos(5 theta), G3 = r^2 sin^2(theta) cos(2 phi) in the normalised
 *     coordinates x' (r = |x'|, theta from +z', phi the azimuth), a0..a3 the
 *     4 host doubles in `coeffs` (degree is ignored); `form` maps p to n as
 *     for polynomials.  At r = 0 the polar angle is taken as 0.
 *     grin_trace_adjoint's gradient is with respect to a0..a3;
 *   - GRIN_MEDIUM_N2P: the N2P-GRIN cylinder lens of Sec. VI,
 *     n = [1 + ((R^2 - (rho/2)^2) / F^2)^beta]^gamma with rho the distance
 *     from the axis through (norm_offset[0], norm_offset[1]) parallel to z;
 *     `coeffs` = R > 0, F > 0, beta, gamma (4 host doubles); form must be
 *     GRIN_FORM_LINEAR; degree and norm_scale are ignored.  The z extent is
 *     the boundary's (a cylinder, z0 = -L, z1 = 0, in the paper).
 *     grin_trace_adjoint's gradient is with respect to (R, F, beta, gamma).
 * n_levels > 0 turns the field into that many isoindicial shells (the
 * discretised media of Sec. I and the abstract): level
 * k = clamp(floor(n_levels (f - level_lo) / (level_hi - level_lo)), 0,
 * n_levels - 1) has index level_lo + (k + 1/2)(level_hi - level_lo)/n_levels,
 * the gradient is zero inside a shell and grad f at a level change.
 * The enclosing surface (Sec. II (i)) is a box (lo[3], hi[3]), a sphere
 * (centre[3], R) or a z-axis cylinder (cx, cy, R, z0, z1) in `boundary`;
 * n_ext is the surround index.  Points exactly on the surface are outside.
 */
typedef struct {
  int32_t kind;
  int32_t form;
  double form_c;
  int32_t degree;
  const double* coeffs;
  double norm_offset[3];
  double norm_scale[3];
  int32_t nx, ny, nz;
  const float* grid;
  int32_t grid_on_device;
  double origin[3];
  double spacing[3];
  int32_t n_levels;
  double level_lo, level_hi;
  int32_t boundary_kind;
  double boundary[8];
  double n_ext;
} grin_medium_desc;

/* Ray batch: structure-of-arrays origins and directions (directions need not
 * be unit; they are normalised on entry), `count` rays of `dtype`
 * (GRIN_F32 or GRIN_F64). */
typedef struct {
  const void *ox, *oy, *oz;
  const void *dx, *dy, *dz;
  int64_t count;
  int32_t dtype;
} grin_rays;

/* Per-ray results, `count` entries each: the final point (the exit point on
 * the surface for a ray that left), the final direction (refracted into the
 * surround for a ray that left), the accumulated optical path length (the
 * exterior approach segment included), the exit id, the number of interior
 * steps (a step cut short at the surface counts as one), and the numbers of
 * internal and boundary total internal reflections.
 *
 * margin (optional, NULL to skip): 4 doubles a ray, ray-major
 * (margin[4 r + k]), the decision margins of the trace, each the minimum
 * over the ray's steps of a quantity whose sign decides an integer outcome,
 * so that a caller can tell which exit states are ill-conditioned:
 *   k = 0: distance of |N.I| from its critical value sqrt(1 - 1/mu^2) at a
 *          refraction test with mu > 1 (D / (mu^2 (|N.I| + critical)),
 *          Eq. 9 and Sec. II (v)); INFINITY if no test had mu > 1;
 *   k = 1: |N.I| at the gradient steps (the sign in Eq. 9; the tangential
 *          case Sec. II (iv) at zero);
 *   k = 2: distance of a step's end point to the enclosing surface, in
 *          steps (first order for curved surfaces; Sec. II (i));
 *   k = 3: distance of the level coordinate of a layered medium to the
 *          nearest shell boundary, in levels; INFINITY for continuous media.
 * GRIN_PREC_FP64 computes them in FP64 exactly as the plain tracer steps;
 * GRIN_PREC_FP32_MIXED computes them in FP32 on its own trajectory;
 * GRIN_PREC_FP64_FAST and the serving and allocation-free entry points do
 * not (GRIN_ERR_NOT_IMPLEMENTED when margin is not NULL). */
typedef struct {
  double *px, *py, *pz;
  double *dx, *dy, *dz;
  double* opl;
  int32_t* exit_id;
  int32_t* steps;
  int32_t* tir_internal;
  int32_t* tir_boundary;
  double* margin;
} grin_out;

/* grin_params.flags.
 * GRIN_TRACE_LEVEL_ROOT: for a layered medium, refract where a step meets a
 *   shell boundary instead of at the first sampled point beyond it.  The
 *   layered media are the discretised media of Sec. I, stacks of isoindicial
 *   surfaces; with this flag the first point of a step outside the current
 *   shell (found on the step, by bisection in FP64 or by safeguarded Newton
 *   iterations in the mixed tracer) ends the step (it counts as a step and
 *   adds its fraction of Delta L_0, like a crossing of the enclosing
 *   surface, Sec. II (i)), and the ray refracts there by Eq. 8-9 with the
 *   isoindicial normal grad f / |grad f| of the smooth field and
 *   mu = n_k / n_k' of the two shells, or is totally reflected (Sec. II
 *   (v)) and stays in its shell.  Inside a shell the steps are straight
 *   (Sec. II (iii)).  No effect on continuous media.  GRIN_PREC_FP64 and
 *   GRIN_PREC_FP32_MIXED (and the serving loop) support it;
 *   GRIN_PREC_FP64_FAST and grin_trace_adjoint return
 *   GRIN_ERR_NOT_IMPLEMENTED. */
enum { GRIN_TRACE_LEVEL_ROOT = 1u };

/* dopl = Delta L_0 > 0 (Eq. 3); max_steps >= 0 interior steps per ray;
 * precision:
 *   GRIN_PREC_FP64: the plain FP64 tracer, one thread per ray, every formula
 *     evaluated as written with unfused IEEE operations (polynomials as
 *     monomial sums), so results do not depend on compiler contraction;
 *   GRIN_PREC_FP64_FAST: the same steps in FP64 with Horner polynomials and
 *     fused multiply-adds (differs from GRIN_PREC_FP64 by rounding order);
 *   GRIN_PREC_FP32_MIXED: FP32 stepping with compensated position sums, the
 *     index difference n_i - n_{i-1} by the trapezoid rule on grad n (exact to
 *     O(step^3); point values for layered media), an exact step-count optical
 *     path, FP64 for the surface root, the boundary refraction and
 *     near-critical discriminants; persistent ray-pool kernel.
 * flags: 0 or GRIN_TRACE_LEVEL_ROOT (above); other bits give
 * GRIN_ERR_INVALID_ARG. */
typedef struct {
  double dopl;
  int32_t max_steps;
  int32_t precision;
  uint32_t flags;
} grin_params;

/* Context on one CUDA device (ordinal `device`); makes that device current
 * on the calling thread.  The context owns the media and servers created on
 * it: grin_ctx_destroy waits for the device, frees the context and returns
 * GRIN_OK, or returns GRIN_ERR_BUSY and frees nothing while any of them has
 * not been destroyed yet. */
int grin_ctx_create(int device, grin_ctx* out);
int grin_ctx_destroy(grin_ctx ctx);

/* Static text for a status code. */
const char* grin_status_string(int status);

/* Number of monomials of a polynomial of the given total degree. */
int grin_poly_terms(int degree);

/* Validate and copy a medium description to the device.  Errors:
 * GRIN_ERR_INVALID_ARG for a bad kind, form, degree, grid size, spacing,
 * scale, level range or boundary; GRIN_ERR_OOM / GRIN_ERR_CUDA on device
 * failures (nothing is leaked). */
int grin_medium_create(grin_ctx ctx, const grin_medium_desc* desc, grin_medium* out);
int grin_medium_destroy(grin_medium medium);
/* Device bytes the medium holds (its sample grid, if any). */
int grin_medium_device_bytes(grin_medium medium, size_t* bytes);

/* Trace rays->count rays (device SoA) into out (device SoA), asynchronously
 * on `cuda_stream`.  count == 0 is a no-op.  Errors: GRIN_ERR_INVALID_ARG
 * for NULL pointers, count < 0, dopl <= 0 or non-finite, max_steps < 0, bad
 * precision or dtype; GRIN_ERR_CUDA if the launch fails.
 * GRIN_PREC_FP32_MIXED on a GRIN_MEDIUM_GRID medium with at least 65,536
 * rays first buckets the rays by the cell of the medium's bounding box where
 * they enter it (three small kernels) and the pool claims them in that order,
 * so neighbouring rays share warps and their interpolation stencils; each
 * ray's result is bitwise the same in any order.  Its scratch
 * (6 bytes a ray) comes from a stream-ordered memory pool the context owns,
 * allocated and freed on `cuda_stream`; if that allocation fails the rays
 * are claimed in index order. */
int grin_trace(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
               const grin_params* params, const grin_out* out, void* cuda_stream);

/* Same as grin_trace with rays and out in HOST memory: the library copies the
 * rays to context-owned device buffers, traces, copies the results back and
 * synchronises before returning (no copy is in flight on return).  A batch
 * of at least 262,144 rays is split into up to 8 chunks of at least 131,072
 * rays, pipelined on four streams the context owns (created on first use):
 * the upload of the next chunk and the download of the previous one overlap
 * the trace of the current one, and the work starts after what is already
 * queued on `cuda_stream`.  Each ray's result is bitwise the same as one
 * grin_trace over the whole batch.  Pinned host buffers let the copies run
 * asynchronously; pageable ones work but serialise them.  Errors: as
 * grin_trace, plus GRIN_ERR_OOM if the staging buffers cannot grow. */
int grin_trace_host(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                    const grin_params* params, const grin_out* out, void* cuda_stream);

/* Trajectory tap: the plain FP64 trace (params->precision must be
 * GRIN_PREC_FP64) that also records each ray's points, for plots and
 * debugging of a few rays (one thread per ray).  The paper draws the whole
 * polyline of each ray (Sec. IV-V); these are its vertices P_i (Eq. 2): the
 * first point inside the medium (the start point, or the entry point on the
 * surface), then every step's end point, full steps and steps cut at the
 * surface (Sec. II (i)) alike.  Exterior segments are not sampled.
 *   path:     caller-owned device array of rays->count * cap * 3 doubles,
 *             ray-major: point i of ray r is path[3 (cap r + i) + 0..2];
 *   cap:      points stored per ray (>= 1); later points are not stored, the
 *             trace itself runs to its end as in grin_trace;
 *   path_len: caller-owned device array of rays->count int64: the number of
 *             points the ray produced, which may exceed cap.
 * out receives exactly what grin_trace (GRIN_PREC_FP64) writes.  Errors as
 * grin_trace, and GRIN_ERR_INVALID_ARG for another precision, cap < 1, a
 * NULL path or path_len, or a path size beyond int64. */
int grin_trace_path(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                    const grin_params* params, const grin_out* out, double* path, int64_t cap,
                    int64_t* path_len, void* cuda_stream);

/* Kernel launches made by the last grin_trace / grin_trace_host /
 * grin_trace_path call on this context (for accounting). */
int grin_ctx_last_launches(grin_ctx ctx, int32_t* launches);

/* Summary of a trace's results, for logging and monitoring.  `out` holds
 * the results of `count` rays (device arrays, as grin_trace wrote them);
 * they are reduced on the device on cuda_stream and the totals copied back,
 * so the call synchronises that stream.
 *   rays, ray_steps: count and the sum of the step counts;
 *   exit_face[f]: rays that left through face f (exit id 0..5), and the
 *     rays of each other exit id;
 *   tir_internal, tir_boundary: sums of the TIR counts;
 *   flagged: rays with any of the four decision margins (grin_out.margin,
 *     which must then be set) below the matching entry of margin_min (four
 *     thresholds), or -1 when margin_min is NULL;
 *   elapsed_ms: device time of the most recent grin_trace call on this
 *     context (for grin_trace_host, the trace of its last chunk), from CUDA
 *     events recorded on its stream around its kernels (-1 if it recorded
 *     none: a capturing stream, or no call yet).
 * Errors: GRIN_ERR_INVALID_ARG for a null pointer among the arrays it
 * reads, a negative count, or margin_min without out->margin. */
typedef struct {
  int64_t rays, ray_steps;
  int64_t exit_face[6];
  int64_t exit_miss, exit_entry_reflect, exit_max_steps, exit_invalid;
  int64_t tir_internal, tir_boundary;
  int64_t flagged;
  double elapsed_ms;
} grin_trace_stats;
int grin_trace_stats_compute(grin_ctx ctx, const grin_out* out, int64_t count,
                             const double* margin_min, grin_trace_stats* stats,
                             void* cuda_stream);

/* ------------------------------------------------------------ adjoint
 *
 * Gradient of a loss of the exit states with respect to the medium
 * parameters, for direct design (the design use of VRT, Sec. VI): reverse
 * mode through the discrete VRT map of the plain FP64 tracer with its
 * branch decisions held fixed (refraction or TIR at each point, surface
 * crossings, exit).  The forward sweep saves the ray state every
 * checkpoint_every steps in `workspace` (104 bytes a checkpoint); the
 * backward sweep recomputes each segment from its checkpoint and carries the
 * adjoint back through it.  checkpoint_every = 1 stores every step with its
 * case and the field at its end point, so the backward sweep recomputes
 * nothing, for 104 bytes a ray-step of workspace (55 GB for 262,144 rays of
 * up to 2,000 steps).  The gradient is the same for every checkpoint_every.
 * Supported media: a box, sphere or cylinder boundary, and either a
 * polynomial with n = p, sqrt(p) or form_c / p (gradient w.r.t. its
 * C(degree+3,3) graded-lex coefficients), the spherical freeform (a0..a3,
 * with the same forms), the N2P lens (gradient w.r.t. R, F, beta, gamma: 4
 * entries) or a grid (gradient w.r.t. its nx*ny*nz samples, x fastest);
 * continuous or in point-sampled shells (n_levels > 0: a shell's index is a
 * constant, the parameters act through the refraction normal of the smooth
 * field).  GRIN_TRACE_LEVEL_ROOT (exact shell crossings) and a margin output
 * give GRIN_ERR_NOT_IMPLEMENTED.  Tangential incidence (N.I == 0, Sec. II (iv))
 * is differentiated through its arc, including the extra index sample. */

/* dL/d(exit state): device FP64 arrays of `count` entries each (the same
 * fields as grin_out; any may be NULL for zero). */
typedef struct {
  const double *px, *py, *pz;
  const double *dx, *dy, *dz;
  const double* opl;
} grin_out_grad;

/* Device bytes of workspace grin_trace_adjoint needs. */
int grin_trace_adjoint_workspace_size(grin_medium medium, int64_t ray_count,
                                      const grin_params* params, int32_t checkpoint_every,
                                      size_t* bytes);

/* The checkpoint interval for a workspace of at most budget_bytes: 1 (every
 * step stored, so the backward sweep recomputes nothing: the fastest) when
 * its workspace fits, else the smallest K <= 64 whose workspace fits (every
 * K >= 2 recomputes each step once).  GRIN_ERR_OOM if not even K = 64 fits;
 * GRIN_ERR_NOT_IMPLEMENTED for media the adjoint does not support.  Host
 * arithmetic only; no device memory is touched. */
int grin_trace_adjoint_interval(grin_medium medium, int64_t ray_count, const grin_params* params,
                                size_t budget_bytes, int32_t* checkpoint_every);

/* Forward sweep (writes `out`, bitwise the results of grin_trace with
 * GRIN_PREC_FP64) then backward sweep, adding dL/d(parameters) into the
 * device FP64 array dL_dmedium (the caller zeroes it).  params->precision
 * must be GRIN_PREC_FP64; 1 <= checkpoint_every <= 64; rays, out, dL_dout
 * and workspace are device memory; asynchronous on cuda_stream.  Rays that
 * miss, reflect at entry or are invalid contribute nothing. */
int grin_trace_adjoint(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                       const grin_params* params, const grin_out* out,
                       const grin_out_grad* dL_dout, double* dL_dmedium,
                       int32_t checkpoint_every, void* workspace, size_t workspace_bytes,
                       void* cuda_stream);

/* The two sweeps of grin_trace_adjoint as separate calls, for a caller that
 * needs the exit states before it knows dL/dout (an autograd forward and
 * backward): together they do what one grin_trace_adjoint call does, with
 * the forward trace done once.
 *   grin_trace_adjoint_forward writes `out` (bitwise grin_trace with
 *   GRIN_PREC_FP64) and leaves the checkpoints and each ray's exit id and step
 *   count in `workspace`;
 *   grin_trace_adjoint_backward runs the backward sweep from that workspace
 *   and adds dL/d(parameters) into dL_dmedium.  It must get the same
 *   medium, rays, params and checkpoint_every as the forward call, and the
 *   workspace unchanged in between (nothing checks this: other contents give
 *   a meaningless gradient).  Both are asynchronous on cuda_stream; argument
 *   errors and unsupported media as for grin_trace_adjoint. */
int grin_trace_adjoint_forward(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                               const grin_params* params, const grin_out* out,
                               int32_t checkpoint_every, void* workspace, size_t workspace_bytes,
                               void* cuda_stream);
int grin_trace_adjoint_backward(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                                const grin_params* params, const grin_out_grad* dL_dout,
                                double* dL_dmedium, int32_t checkpoint_every, void* workspace,
                                size_t workspace_bytes, void* cuda_stream);

/* ------------------------------------------------------------ serving
 *
 * A server batches trace jobs continuously on one GPU.  A job is a batch of
 * rays through one medium (host buffers, like grin_trace_host) traced by the
 * mixed-precision tracer.  A scheduler thread owns the GPU work:
 *   - admission: queued jobs are admitted first come, first served, when
 *     their device footprint (rays in, results out, resident ray state and,
 *     for gridded media with at least 65,536 rays, 6 bytes a ray of claim
 *     order as in grin_trace) fits in what is left of the server's device
 *     arena (hbm_budget_bytes, taken once at creation) and resident ray slots
 *     are free;
 *   - ticks: every tick advances each running job's slots by step_quantum
 *     steps; a slot whose ray ends takes the job's next ray; the ray state
 *     stays on the device between ticks, so a small job submitted while a
 *     large one runs finishes after a few ticks instead of after it;
 *   - completion: when all of a job's rays have ended its results are copied
 *     to the caller's host buffers and the job becomes GRIN_JOB_DONE.
 * Per-ray results do not depend on the other jobs in flight (bitwise equal
 * to grin_trace_host with the mixed tracer).  The caller keeps its host
 * buffers alive until the job is DONE, FAILED or CANCELLED.  All grin_serve_*
 * calls are thread-safe. */
enum { GRIN_JOB_QUEUED = 0, GRIN_JOB_RUNNING = 1, GRIN_JOB_DONE = 2, GRIN_JOB_FAILED = 3,
       GRIN_JOB_CANCELLED = 4 };

typedef struct {
  size_t hbm_budget_bytes;   /* device arena for job data (> 0) */
  int32_t step_quantum;      /* steps per slot per tick; 0 = 1024 */
  int32_t max_slots_per_job; /* resident slots one job may hold; 0 = a quarter of the GPU's */
} grin_serve_config;

typedef struct {
  uint64_t submitted, done, failed, cancelled;
  uint64_t ticks;
  double ray_steps;          /* summed over finished jobs */
  size_t arena_bytes, arena_in_use;
  int32_t slots_total, slots_in_use, jobs_queued, jobs_running;
} grin_serve_counters;

/* Create a server on the context's device.  Errors: GRIN_ERR_INVALID_ARG,
 * GRIN_ERR_OOM if the arena cannot be allocated. */
int grin_serve_create(grin_ctx ctx, const grin_serve_config* config, grin_server* out);
/* Stop the scheduler; queued and running jobs end as CANCELLED. */
int grin_serve_destroy(grin_server server);
/* Queue a job (precision must be GRIN_PREC_FP32_MIXED; medium from the
 * server's context; rays and out are host buffers).  GRIN_ERR_BUSY if the
 * job could never fit the arena. */
int grin_serve_submit(grin_server server, grin_medium medium, const grin_rays* rays,
                      const grin_params* params, const grin_out* out, uint64_t* job_id);
/* State of a job and its latency: submit to completion once DONE, else the
 * time since submission.  GRIN_ERR_NOT_FOUND for an unknown id. */
int grin_serve_poll(grin_server server, uint64_t job_id, int32_t* state, double* latency_s);
/* Where a job's latency went: *queued_s from submission to admission (to
 * now while it is still queued, to its end if it ended unadmitted), *run_s
 * from admission to completion (to now while it runs).
 * GRIN_ERR_NOT_FOUND for an unknown id. */
int grin_serve_timing(grin_server server, uint64_t job_id, double* queued_s, double* run_s);
/* Wait up to timeout_s seconds for the job to end (DONE, FAILED or
 * CANCELLED); GRIN_ERR_TIMEOUT if it has not. */
int grin_serve_wait(grin_server server, uint64_t job_id, double timeout_s, int32_t* state);
/* Cancel a queued or running job (takes effect at the next tick). */
int grin_serve_cancel(grin_server server, uint64_t job_id);
int grin_serve_stats(grin_server server, grin_serve_counters* stats);

/* ------------------------------------------------- bounds-checked build
 *
 * The library is also built with every device array index of its kernels
 * range-checked (lib/libgrin_vrt_checked.so, same ABI; a stand-in for a
 * memory checker): the grid samples of every gather, the slots of the mixed
 * tracer's tap cache in shared memory, the claim order and the ray indices,
 * the adjoint's samples and gradient entries.  An index out of range is
 * replaced by 0, so the access stays in bounds and the kernel runs on, and
 * the site of the first one is recorded per device.  The paper has no
 * counterpart.
 * grin_build_checked: 1 in the checked build, 0 in the ordinary one.
 * grin_checked_status: the recorded site on `device` (0 if none; 1 a ray
 *   index, 2 a grid sample of the mixed tracer, 3 a tap-cache slot, 4 a grid
 *   sample of the FP64 tracers, 5 the adjoint), read after synchronising the
 *   device and cleared; returns GRIN_ERR_CHECKED_BOUNDS when a site was
 *   recorded, else GRIN_OK (always GRIN_OK with 0 in the ordinary build).
 * grin_checked_selftest: in the checked build, runs a one-thread kernel that
 *   forms an out-of-range grid index on purpose (the check redirects it, no
 *   memory outside the array is touched) and leaves site 4 to be read;
 *   GRIN_ERR_NOT_IMPLEMENTED in the ordinary build, which runs nothing. */
int grin_build_checked(void);
int grin_checked_status(int device, int32_t* site);
int grin_checked_selftest(int device);

/* Largest batch grin_trace_host_static accepts. */
#define GRIN_STATIC_MAX_RAYS 65536

/* Trace without allocating anything, for callers that may not call
 * cudaMalloc (a plug-in whose host application owns the GPU memory budget,
 * a loop that must not allocate after start-up, a caller whose device
 * memory is all in its own pool).  The paper has no counterpart: this is a
 * deployment variant of grin_trace_host.
 *   - No context and no grin_medium: `desc` is read directly; only
 *     polynomial media (GRIN_MEDIUM_POLY) are accepted, since they live
 *     entirely in the kernel's parameters; others give GRIN_ERR_INVALID_ARG.
 *   - rays and out are HOST buffers as for grin_trace_host; at most
 *     GRIN_STATIC_MAX_RAYS rays (GRIN_ERR_INVALID_ARG beyond).
 *   - The device side uses one fixed array of about 7.5 MiB that every GPU
 *     loading the library reserves until the process exits; it holds the
 *     staged rays, the results and the ray-queue counter (cleared on the
 *     stream before each launch).  It is shared by all calls and keeps the
 *     last call's contents: calls whose GPU work overlaps (other streams or
 *     threads) race on it and must be serialised by the caller.
 *   - Runs on the calling thread's current device and context; every call
 *     looks the array's address up there (cudaGetSymbolAddress, which
 *     allocates nothing once the library's module is loaded), so a device
 *     reset or a different current context between calls is safe.
 *   - Copies into the caller's host buffers and synchronises `cuda_stream`
 *     before returning, which a stream being captured into a CUDA graph does
 *     not allow: on such a stream it returns GRIN_ERR_INVALID_ARG and queues
 *     nothing.  Otherwise the same statuses as grin_trace_host. */
int grin_trace_host_static(const grin_medium_desc* desc, const grin_rays* rays,
                           const grin_params* params, const grin_out* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GRIN_H */
