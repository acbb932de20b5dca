// grin_internal.h -- device-side medium record and launch entry points shared
// by the C ABI (grin_capi.cu) and the kernels (trace_fp64.cu, trace_mixed.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>
#include <vector>

#include "grin.h"

namespace grin {

// Bounds-checked build (-DGRIN_CHECKED, built beside the library as
// lib/libgrin_vrt_checked.so): every index a kernel forms into a device array
// of the call -- grid samples, the tap cache in shared memory, the claim
// order, the ray arrays -- goes through GRIN_IDX.  An index outside [0, n)
// records its site in the device word DevMedium::oob (the first one wins;
// grin_checked_status reads and clears it) and is replaced by 0, so the
// access stays inside the array and the kernel runs on.  The ordinary build
// compiles GRIN_IDX to the bare index.
enum CheckSite : unsigned {
  kSiteRay = 1,         // a ray index (claim order value) outside the batch
  kSiteGridMixed = 2,   // a grid sample of the mixed tracer's gathers
  kSiteTapCache = 3,    // a slot of the mixed tracer's tap cache
  kSiteGridFP64 = 4,    // a grid sample of the FP64 tracers
  kSiteGridAdjoint = 5  // a grid sample or gradient entry of the adjoint
};
#ifdef GRIN_CHECKED
__device__ __forceinline__ int64_t checked_index(unsigned int* word, int64_t i, int64_t n,
                                                 unsigned site) {
  if (i >= 0 && i < n) return i;
  if (word) atomicCAS(word, 0u, site);
  return 0;
}
#define GRIN_IDX(m, i, n, site) ::grin::checked_index((m).oob, (int64_t)(i), (int64_t)(n), ::grin::site)
#else
#define GRIN_IDX(m, i, n, site) (i)
#endif

// Largest supported polynomial: C(GRIN_MAX_DEGREE + 3, 3) coefficients.
constexpr int kMaxTerms = 84;

// Polynomial evaluators are instantiated for these total degrees; a medium
// of lower degree is zero-padded to the next class.
// Coefficient layout of an analytic medium, also the template parameter PC of
// the kernels: polynomial degree classes, the spherical freeform field, or
// the N2P cylinder lens.
enum PolyClass : int32_t { kSpherical = 1, kPoly2 = 2, kN2P = 3, kPoly4 = 4, kPoly6 = 6 };

// Everything a kernel needs to evaluate n, grad n and the boundary, passed by
// value as a kernel parameter (it lives in the constant bank, so every lane
// reads the same coefficient in one broadcast).
struct DevMedium {
  int32_t kind;      // GRIN_MEDIUM_POLY / GRIN_MEDIUM_GRID
  int32_t form;      // GRIN_FORM_*
  int32_t pclass;    // PolyClass of the coefficient layout
  int32_t n_levels;  // 0: continuous
  int32_t bkind;     // GRIN_BOUNDARY_*
  int32_t nx, ny, nz;
  int32_t rows16;  // grid rows start on 16-byte boundaries (nx % 4 == 0)
  double form_c, n_ext;
  // Index offset: the FP32 path carries nu = n - base so that the difference
  // of successive indices (which drives each refraction) keeps its bits.
  double base;
  double off[3], inv_scale[3];
  double origin[3], inv_spacing[3];
  double lvl_lo, lvl_hi, lvl_span;  // level_lo, level_hi, level_hi - level_lo
  double b[8];                    // boundary parameters (grin_medium_desc)
  const float* grid;              // device samples (x fastest)
  int64_t grid_n;                 // nx * ny * nz
  // bounds-checked build: the device word recording the first out-of-range
  // index (a CheckSite), one per device (see checked_index)
  unsigned int* oob;
  double scale[3], spacing[3];    // as given (the plain FP64 tracer divides)
  double cglex[kMaxTerms];        // coefficients in graded-lex order, zero padded
  double c64[kMaxTerms];          // coefficients in Horner layout (see hidx)
  float c32[kMaxTerms];           // same, constant term shifted for nu
  // c32 again at a stride of two floats (c32s[2 t] = c32[t], odd slots zero),
  // read by the FP32 polynomial evaluation: no two coefficients it reads are
  // adjacent, so the compiler keeps each one as the constant operand of its
  // FMA instead of merging neighbours into vector loads into registers
  // (measured: about ten fewer instructions a ray-step)
  float c32s[2 * kMaxTerms];
  float base_f, form_c_f, n_ext_f;
  float off_f[3], inv_scale_f[3], origin_f[3], inv_spacing_f[3];
  // -off / scale, so that the normalised coordinate is one FMA,
  // x = p inv_scale_f + noff_f
  float noff_f[3];
  // residuals of origin_f and inv_spacing_f: origin = origin_f + origin_lo_f and
  // 1 / spacing = inv_spacing_f + inv_spacing_lo_f to about 2^-48 relative
  float origin_lo_f[3], inv_spacing_lo_f[3];
  float lvl_lo_rel_f, lvl_scale_f, lvl_step_f;  // lo - base, L / span, span / L
  float b_f[8];
};

struct TraceArgs {
  const void *ox, *oy, *oz, *dx, *dy, *dz;
  int64_t count;
  int32_t dtype;  // GRIN_F32 / GRIN_F64
  double *px, *py, *pz, *ux, *uy, *uz, *opl;
  int32_t *exit_id, *steps, *tir_i, *tir_b;
  double dopl;
  int32_t max_steps;
  // mixed tracer: claim order (a permutation of 0..count-1), or nullptr for
  // index order
  const uint32_t* perm = nullptr;
  // grin_params.flags (GRIN_TRACE_LEVEL_ROOT) and the optional per-ray decision
  // margins (grin_out.margin: 4 doubles a ray, or nullptr)
  uint32_t flags = 0;
  double* margin = nullptr;
};

// Validated device record of a medium description (grin_capi.cu); a grid's
// samples go to *samples for the caller to upload (nullptr refuses grids).
int describe_medium(const grin_medium_desc* d, DevMedium* m, std::vector<float>* samples);
// The allocation-free entry point's own bounds word (in its static array):
// read and clear it on the current device (grin_static.cu).
int static_oob_take(unsigned int* value);

// Number of kernel launches made; negative grin_status on failure.
int launch_fp64(const DevMedium& m, const TraceArgs& a, cudaStream_t s, int sm_count);
int launch_fp64_fast(const DevMedium& m, const TraceArgs& a, cudaStream_t s, int sm_count);
// The plain FP64 trace, recording each ray's points (trace_fp64.cu).
int launch_fp64_path(const DevMedium& m, const TraceArgs& a, double* path, int64_t cap,
                     int64_t* plen, cudaStream_t s);
int launch_mixed(const DevMedium& m, const TraceArgs& a, unsigned long long* queue,
                 cudaStream_t s, int sm_count);

// Serving: bytes of one resident ray slot, and one tick over a job's slots
// (nslots a multiple of 128; counters = {next ray, finished rays}).
size_t serve_slot_bytes();
int launch_serve_tick(const DevMedium& m, const TraceArgs& a, void* slots, int nslots,
                      unsigned long long* counters, int quantum, cudaStream_t s);

constexpr int kQueueSlots = 4096;

// grin_trace_host pipelines batches of at least 2 * kHostChunkMin rays in up
// to kHostChunks chunks (each at least kHostChunkMin rays).
constexpr int kHostChunks = 8;
constexpr int64_t kHostChunkMin = 131072;

// Claim order for the mixed tracer on gridded media (ray_order.cu): rays
// bucketed by the cell of the medium's bounding box where they enter it.
// Used from this many rays.
constexpr int64_t kOrderMinRays = 65536;
size_t order_scratch_bytes(int64_t n);
// Three launches into `scratch` (order_scratch_bytes(count) bytes, 256-byte
// aligned); *perm_out points into it.  Returns the launch count or a status.
int launch_order(const DevMedium& m, const TraceArgs& a, void* scratch, int sm_count,
                 cudaStream_t s, const uint32_t** perm_out);
// The adjoint's backward order: rays by step count (meta[2 r + 1]), longest
// first; same scratch layout.  Returns the launch count or a status.
int launch_order_by_steps(const int32_t* meta, int64_t n, void* scratch, cudaStream_t s,
                          const uint32_t** perm_out);

// Launches kern<<<grid, block, 0, s>>>(args...) and returns 1, or
// GRIN_ERR_CUDA if this launch failed.  cudaLaunchKernelEx reports the
// launch's own status; the runtime's per-thread last-error slot, which any
// earlier runtime call of the process may have left set, is not consulted
// (and is cleared after a failed launch).
template <typename... P, typename... A>
inline int launch_kernel(void (*kern)(P...), unsigned grid, unsigned block, cudaStream_t s,
                         A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  if (cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...) != cudaSuccess) {
    cudaGetLastError();
    return GRIN_ERR_CUDA;
  }
  return 1;
}

// Adjoint (adjoint.cu): supported media, workspace bytes, and the forward
// (checkpointing) plus backward sweeps; gout = dL/d(px, py, pz, dx, dy, dz,
// opl) device arrays; grad accumulates dL/d(parameters).
bool adjoint_supported(const DevMedium& m);
size_t adjoint_workspace(int64_t rays, int32_t max_steps, int32_t k);
// phase: kAdjBoth, or one of the two sweeps (the backward sweep reads the
// checkpoints and step counts a forward call left in ws; it writes no
// outputs and needs no gout for the forward sweep)
enum AdjPhase : int { kAdjBoth = 0, kAdjForward = 1, kAdjBackward = 2 };
// grin_trace_stats_compute's reduction: kStatWords totals (see grin_stats.cu)
// into the zeroed device words `acc`
constexpr int kStatWords = 16;
int launch_stats(const TraceArgs& a, const double* margin_min, unsigned long long* acc,
                 cudaStream_t st);
int launch_adjoint(const DevMedium& m, const TraceArgs& a, int32_t k, void* ws,
                   const double* const* gout, double* grad, int nterms, cudaStream_t st,
                   int phase = kAdjBoth);

}  // namespace grin

struct grin_ctx_s {
  int device = 0;
  // media and servers created on this context and not yet destroyed; the
  // context cannot be destroyed while any remain
  std::atomic<int> children{0};
  int sm_count = 0;
  // One 8-byte ray-queue counter per trace call, taken round robin, so calls
  // on different streams do not share a counter while fewer than kQueueSlots
  // are in flight.
  unsigned long long* queues = nullptr;
  int next_queue = 0;
  int last_launches = 0;
  // device staging for grin_trace_host (grown on demand)
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // stream-ordered pool for the per-call claim-order scratch of the mixed
  // tracer (created on first use; keeps freed blocks for reuse)
  cudaMemPool_t pool = nullptr;
  // grin_trace_host's pipeline (created on first use): upload stream, two
  // trace streams, download stream; per chunk an upload and a trace event;
  // and an event marking the caller's stream
  cudaStream_t hs[4] = {};
  cudaEvent_t hev[2 * grin::kHostChunks + 1] = {};
  // grin_trace_stats_compute: its device totals, and the timing events of
  // the last grin_trace call (created on first use; timed = both recorded)
  unsigned long long* stats = nullptr;
  cudaEvent_t tev[2] = {};
  bool timed = false;
};

struct grin_medium_s {
  grin_ctx ctx = nullptr;
  grin::DevMedium dm{};
  float* grid_dev = nullptr;
  size_t grid_bytes = 0;
};
