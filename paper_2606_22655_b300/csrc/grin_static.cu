// grin_static.cu -- grin_trace_host_static: a trace entry point that makes
// no device (or host) allocation at all.
//
// Who needs it: code that is not allowed to call cudaMalloc -- a plug-in
// running inside a host application that owns the GPU memory budget, a
// real-time loop that must not allocate after start-up, or a caller that
// has already handed all device memory to its own pool.  Such a caller
// cannot create a grin_ctx (which allocates its ray-queue counters) or a
// grid medium (which copies the samples to the device).  This entry point
// takes the medium description itself (polynomial media only: they live
// entirely in the kernel's parameter block) and host buffers, and uses one
// file-scope __device__ array, reserved when the library is loaded on a GPU,
// for everything the trace needs on the device: the rays, the results and
// the ray-queue counter of the persistent kernel.
//
// The array is shared by every call on a device and keeps the last call's
// contents; the queue counter is cleared on the stream before each launch.
// Two calls whose work overlaps on the GPU (different streams, or different
// host threads) race on the array: callers must serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "grin_device.cuh"
#include "grin_internal.h"

namespace {

// Largest batch the static array holds, and its bytes per ray: up to six
// FP64 inputs and seven FP64 plus four int32 outputs.
constexpr int64_t kMaxRays = GRIN_STATIC_MAX_RAYS;
constexpr size_t kPerRay = 6 * 8 + 7 * 8 + 4 * 4;
constexpr size_t kHeader = 256;  // the ray-queue counter, the bounds word, padding
constexpr size_t kOobOffset = 8;  // the bounds-checked build's word (see grin_checked_status)
constexpr size_t kScratchBytes = kHeader + kPerRay * (size_t)kMaxRays;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// The device address of g_scratch in the current context, looked up on every
// call: cudaGetSymbolAddress allocates nothing once the module is loaded, and
// an address cached per device could name a module instance that a later
// cudaDeviceReset, or another context made current by the caller, no longer
// holds.
int scratch_for_current_device(unsigned char** ptr, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRIN_ERR_CUDA;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return GRIN_ERR_CUDA;
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return GRIN_ERR_CUDA;
  }
  *ptr = (unsigned char*)p;
  *sms = n;
  return GRIN_OK;
}

}  // namespace

// The bounds word in the static array: read and clear it (current device).
int grin::static_oob_take(unsigned int* value) {
  *value = 0;
  unsigned char* base = nullptr;
  int sms = 0;
  if (scratch_for_current_device(&base, &sms) != GRIN_OK) return GRIN_ERR_CUDA;
  if (cudaMemcpy(value, base + kOobOffset, sizeof(unsigned int), cudaMemcpyDeviceToHost) !=
          cudaSuccess ||
      cudaMemset(base + kOobOffset, 0, sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    return GRIN_ERR_CUDA;
  }
  return GRIN_OK;
}

extern "C" int grin_trace_host_static(const grin_medium_desc* desc, const grin_rays* rays,
                                      const grin_params* p, const grin_out* out,
                                      void* cuda_stream) {
  if (!desc || !rays || !p || !out) return GRIN_ERR_INVALID_ARG;
  if (rays->count < 0 || rays->count > kMaxRays) return GRIN_ERR_INVALID_ARG;
  if (rays->dtype != GRIN_F32 && rays->dtype != GRIN_F64) return GRIN_ERR_INVALID_ARG;
  if (!(std::isfinite(p->dopl) && p->dopl > 0.0) || p->max_steps < 0 ||
      (p->flags & ~(uint32_t)GRIN_TRACE_LEVEL_ROOT))
    return GRIN_ERR_INVALID_ARG;
  if (out->margin || (p->precision == GRIN_PREC_FP64_FAST && p->flags))
    return GRIN_ERR_NOT_IMPLEMENTED;
  if (p->precision != GRIN_PREC_FP64 && p->precision != GRIN_PREC_FP32_MIXED &&
      p->precision != GRIN_PREC_FP64_FAST)
    return GRIN_ERR_INVALID_ARG;
  // polynomial media only (they live entirely in the kernel's parameter
  // block); built exactly as grin_medium_create builds them
  if (desc->kind != GRIN_MEDIUM_POLY) return GRIN_ERR_INVALID_ARG;
  grin::DevMedium m;
  int st = grin::describe_medium(desc, &m, nullptr);
  if (st != GRIN_OK) return st;
  const int64_t n = rays->count;
  if (n == 0) return GRIN_OK;
  if (!rays->ox || !rays->oy || !rays->oz || !rays->dx || !rays->dy || !rays->dz)
    return GRIN_ERR_INVALID_ARG;
  if (!out->px || !out->py || !out->pz || !out->dx || !out->dy || !out->dz || !out->opl ||
      !out->exit_id || !out->steps || !out->tir_internal || !out->tir_boundary)
    return GRIN_ERR_INVALID_ARG;

  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the copies into pageable host memory and the final synchronisation are
  // not allowed while the stream is being captured into a graph
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return GRIN_ERR_CUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) return GRIN_ERR_INVALID_ARG;
  unsigned char* base = nullptr;
  int sms = 0;
  st = scratch_for_current_device(&base, &sms);
  if (st != GRIN_OK) return st;
  const size_t esz = rays->dtype == GRIN_F64 ? 8 : 4;
  unsigned long long* queue = (unsigned long long*)base;
  m.oob = (unsigned int*)(base + kOobOffset);
  unsigned char* in = base + kHeader;
  const void* hin[6] = {rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz};
  void* din[6];
  for (int k = 0; k < 6; ++k) {
    din[k] = in + (size_t)k * esz * (size_t)n;
    if (cudaMemcpyAsync(din[k], hin[k], esz * (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return GRIN_ERR_CUDA;
  }
  unsigned char* ob = in + 6 * esz * (size_t)n;
  double* dd[7];
  for (int k = 0; k < 7; ++k) dd[k] = (double*)(ob + (size_t)k * 8 * (size_t)n);
  int32_t* di[4];
  for (int k = 0; k < 4; ++k) di[k] = (int32_t*)(ob + 56 * (size_t)n + (size_t)k * 4 * (size_t)n);

  grin::TraceArgs a;
  a.ox = din[0];
  a.oy = din[1];
  a.oz = din[2];
  a.dx = din[3];
  a.dy = din[4];
  a.dz = din[5];
  a.count = n;
  a.dtype = rays->dtype;
  a.px = dd[0];
  a.py = dd[1];
  a.pz = dd[2];
  a.ux = dd[3];
  a.uy = dd[4];
  a.uz = dd[5];
  a.opl = dd[6];
  a.exit_id = di[0];
  a.steps = di[1];
  a.tir_i = di[2];
  a.tir_b = di[3];
  a.dopl = p->dopl;
  a.max_steps = p->max_steps;
  a.flags = p->flags;
  int rc;
  if (p->precision == GRIN_PREC_FP64) rc = grin::launch_fp64(m, a, s, sms);
  else if (p->precision == GRIN_PREC_FP64_FAST) rc = grin::launch_fp64_fast(m, a, s, sms);
  else rc = grin::launch_mixed(m, a, queue, s, sms);  // clears the queue counter first
  if (rc < 0) return rc;

  double* hd[7] = {out->px, out->py, out->pz, out->dx, out->dy, out->dz, out->opl};
  int32_t* hi[4] = {out->exit_id, out->steps, out->tir_internal, out->tir_boundary};
  for (int k = 0; k < 7; ++k)
    if (cudaMemcpyAsync(hd[k], dd[k], 8 * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return GRIN_ERR_CUDA;
  for (int k = 0; k < 4; ++k)
    if (cudaMemcpyAsync(hi[k], di[k], 4 * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return GRIN_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GRIN_ERR_CUDA;
  return GRIN_OK;
}
