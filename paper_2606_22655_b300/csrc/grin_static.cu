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
#include <mutex>

#include "grin_device.cuh"
#include "grin_internal.h"

namespace {

// Largest batch the static array holds, and its bytes per ray: up to six
// FP64 inputs and seven FP64 plus four int32 outputs.
constexpr int64_t kMaxRays = GRIN_STATIC_MAX_RAYS;
constexpr size_t kPerRay = 6 * 8 + 7 * 8 + 4 * 4;
constexpr size_t kHeader = 256;  // the ray-queue counter, padded
constexpr size_t kScratchBytes = kHeader + kPerRay * (size_t)kMaxRays;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device addresses of g_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_dev[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};
std::mutex g_setup_mutex;

int scratch_for_current_device(unsigned char** ptr, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRIN_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GRIN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_dev[dev]) {
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
    g_sm_count[dev] = n;
    g_scratch_dev[dev] = (unsigned char*)p;
  }
  *ptr = g_scratch_dev[dev];
  *sms = g_sm_count[dev];
  return GRIN_OK;
}

// The polynomial medium as grin_medium_create would hold it, built on the
// stack (the polynomial lives entirely in the kernel parameter block).
int poly_medium(const grin_medium_desc* d, grin::DevMedium* out) {
  grin::DevMedium& m = *out;
  std::memset(&m, 0, sizeof(m));
  if (d->kind != GRIN_MEDIUM_POLY || !d->coeffs) return GRIN_ERR_INVALID_ARG;
  if (d->degree < 0 || d->degree > GRIN_MAX_DEGREE) return GRIN_ERR_INVALID_ARG;
  if (d->form < GRIN_FORM_LINEAR || d->form > GRIN_FORM_RECIP) return GRIN_ERR_INVALID_ARG;
  if (d->form == GRIN_FORM_RECIP && !std::isfinite(d->form_c)) return GRIN_ERR_INVALID_ARG;
  if (!(std::isfinite(d->n_ext) && d->n_ext > 0.0)) return GRIN_ERR_INVALID_ARG;
  if (d->n_levels < 0 || d->n_levels > GRIN_MAX_LEVELS) return GRIN_ERR_INVALID_ARG;
  if (d->n_levels > 0 &&
      !(std::isfinite(d->level_lo) && std::isfinite(d->level_hi) && d->level_hi > d->level_lo))
    return GRIN_ERR_INVALID_ARG;
  const double* b = d->boundary;
  for (int k = 0; k < 8; ++k)
    if (!std::isfinite(b[k])) return GRIN_ERR_INVALID_ARG;
  if (d->boundary_kind == GRIN_BOUNDARY_BOX) {
    if (!(b[0] < b[3] && b[1] < b[4] && b[2] < b[5])) return GRIN_ERR_INVALID_ARG;
  } else if (d->boundary_kind == GRIN_BOUNDARY_SPHERE) {
    if (!(b[3] > 0.0)) return GRIN_ERR_INVALID_ARG;
  } else if (d->boundary_kind == GRIN_BOUNDARY_CYLINDER) {
    if (!(b[2] > 0.0 && b[3] < b[4])) return GRIN_ERR_INVALID_ARG;
  } else {
    return GRIN_ERR_INVALID_ARG;
  }
  m.kind = GRIN_MEDIUM_POLY;
  m.form = d->form;
  m.form_c = d->form_c;
  m.n_levels = d->n_levels;
  m.bkind = d->boundary_kind;
  m.n_ext = d->n_ext;
  std::memcpy(m.b, b, sizeof(m.b));
  for (int k = 0; k < 3; ++k) {
    if (!std::isfinite(d->norm_offset[k]) || !std::isfinite(d->norm_scale[k]) ||
        d->norm_scale[k] == 0.0)
      return GRIN_ERR_INVALID_ARG;
    m.off[k] = d->norm_offset[k];
    m.scale[k] = d->norm_scale[k];
    m.inv_scale[k] = 1.0 / d->norm_scale[k];
  }
  m.pclass = d->degree <= 2 ? grin::kPoly2 : (d->degree <= 4 ? grin::kPoly4 : grin::kPoly6);
  const int D = m.pclass;
  int idx = 0;
  for (int s = 0; s <= d->degree; ++s)
    for (int i = s; i >= 0; --i)
      for (int j = s - i; j >= 0; --j) {
        double c = d->coeffs[idx];
        if (!std::isfinite(c)) return GRIN_ERR_INVALID_ARG;
        m.cglex[idx++] = c;
        m.c64[grin::hidx(D, i, j, s - i - j)] = c;
      }
  const double c0 = m.c64[0];
  float base_f = 1.0f;
  if (d->form == GRIN_FORM_LINEAR) base_f = (float)c0;
  else if (d->form == GRIN_FORM_SQRT && c0 > 0.0) base_f = (float)std::sqrt(c0);
  else if (d->form == GRIN_FORM_RECIP && c0 != 0.0 && std::isfinite(d->form_c / c0))
    base_f = (float)(d->form_c / c0);
  if (!(std::isfinite(base_f) && base_f > 0.0f)) base_f = 1.0f;
  m.base_f = base_f;
  m.base = (double)base_f;
  for (int k = 0; k < grin::kMaxTerms; ++k) m.c32[k] = (float)m.c64[k];
  if (d->form == GRIN_FORM_LINEAR) m.c32[0] = (float)(c0 - m.base);
  else if (d->form == GRIN_FORM_SQRT) m.c32[0] = (float)(c0 - m.base * m.base);
  if (d->n_levels > 0) {
    m.lvl_lo = d->level_lo;
    m.lvl_hi = d->level_hi;
    m.lvl_span = d->level_hi - d->level_lo;
    m.lvl_lo_rel_f = (float)(d->level_lo - m.base);
    m.lvl_scale_f = (float)((double)d->n_levels / m.lvl_span);
    m.lvl_step_f = (float)(m.lvl_span / (double)d->n_levels);
  }
  m.form_c_f = (float)m.form_c;
  m.n_ext_f = (float)m.n_ext;
  for (int k = 0; k < 3; ++k) {
    m.off_f[k] = (float)m.off[k];
    m.inv_scale_f[k] = (float)m.inv_scale[k];
  }
  for (int k = 0; k < 8; ++k) m.b_f[k] = (float)m.b[k];
  return GRIN_OK;
}

}  // namespace

extern "C" int grin_trace_host_static(const grin_medium_desc* desc, const grin_rays* rays,
                                      const grin_params* p, const grin_out* out,
                                      void* cuda_stream) {
  if (!desc || !rays || !p || !out) return GRIN_ERR_INVALID_ARG;
  if (rays->count < 0 || rays->count > kMaxRays) return GRIN_ERR_INVALID_ARG;
  if (rays->dtype != GRIN_F32 && rays->dtype != GRIN_F64) return GRIN_ERR_INVALID_ARG;
  if (!(std::isfinite(p->dopl) && p->dopl > 0.0) || p->max_steps < 0 || p->flags != 0)
    return GRIN_ERR_INVALID_ARG;
  if (p->precision != GRIN_PREC_FP64 && p->precision != GRIN_PREC_FP32_MIXED &&
      p->precision != GRIN_PREC_FP64_FAST)
    return GRIN_ERR_INVALID_ARG;
  grin::DevMedium m;
  int st = poly_medium(desc, &m);
  if (st != GRIN_OK) return st;
  const int64_t n = rays->count;
  if (n == 0) return GRIN_OK;
  if (!rays->ox || !rays->oy || !rays->oz || !rays->dx || !rays->dy || !rays->dz)
    return GRIN_ERR_INVALID_ARG;
  if (!out->px || !out->py || !out->pz || !out->dx || !out->dy || !out->dz || !out->opl ||
      !out->exit_id || !out->steps || !out->tir_internal || !out->tir_boundary)
    return GRIN_ERR_INVALID_ARG;

  unsigned char* base = nullptr;
  int sms = 0;
  st = scratch_for_current_device(&base, &sms);
  if (st != GRIN_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t esz = rays->dtype == GRIN_F64 ? 8 : 4;
  unsigned long long* queue = (unsigned long long*)base;
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
