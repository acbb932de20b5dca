// grin_capi.cu -- the C ABI declared in include/grin.h: contexts, media,
// argument checking and dispatch to the tracing kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "grin_device.cuh"
#include <cstdint>

#include "grin_internal.h"

using grin::DevMedium;

using grin::kQueueSlots;

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// The device record of a medium description (validated), as every trace
// kernel takes it by value; for a grid medium the samples are copied into
// *samples (the caller uploads them and sets m->grid).  A grid medium with
// samples == nullptr is refused.
int grin::describe_medium(const grin_medium_desc* d, DevMedium* mp, std::vector<float>* samples) {
  if (!d || !mp) return GRIN_ERR_INVALID_ARG;
  DevMedium& m = *mp;
  std::memset(&m, 0, sizeof(m));
  m.kind = d->kind;
  m.form = d->form;
  m.n_levels = d->n_levels;
  m.bkind = d->boundary_kind;
  m.n_ext = d->n_ext;
  m.form_c = d->form_c;
  if (!finite_pos(d->n_ext)) return GRIN_ERR_INVALID_ARG;
  if (d->kind < GRIN_MEDIUM_POLY || d->kind > GRIN_MEDIUM_N2P) return GRIN_ERR_INVALID_ARG;
  if (d->n_levels < 0 || d->n_levels > GRIN_MAX_LEVELS) return GRIN_ERR_INVALID_ARG;
  if (d->n_levels > 0 && !(std::isfinite(d->level_lo) && std::isfinite(d->level_hi) &&
                           d->level_hi > d->level_lo))
    return GRIN_ERR_INVALID_ARG;
  for (int k = 0; k < 8; ++k)
    if (!std::isfinite(d->boundary[k])) return GRIN_ERR_INVALID_ARG;
  const double* b = d->boundary;
  switch (d->boundary_kind) {
    case GRIN_BOUNDARY_BOX:
      if (!(b[0] < b[3] && b[1] < b[4] && b[2] < b[5])) return GRIN_ERR_INVALID_ARG;
      break;
    case GRIN_BOUNDARY_SPHERE:
      if (!(b[3] > 0.0)) return GRIN_ERR_INVALID_ARG;
      break;
    case GRIN_BOUNDARY_CYLINDER:
      if (!(b[2] > 0.0 && b[3] < b[4])) return GRIN_ERR_INVALID_ARG;
      break;
    default:
      return GRIN_ERR_INVALID_ARG;
  }
  std::memcpy(m.b, b, sizeof(m.b));

  if (d->kind == GRIN_MEDIUM_N2P) {
    // R, F, beta, gamma; the axis through norm_offset[0..1]; no scaling
    if (!d->coeffs || d->form != GRIN_FORM_LINEAR) return GRIN_ERR_INVALID_ARG;
    const double* c = d->coeffs;
    if (!(finite_pos(c[0]) && finite_pos(c[1]) && std::isfinite(c[2]) && std::isfinite(c[3])))
      return GRIN_ERR_INVALID_ARG;
    if (!std::isfinite(d->norm_offset[0]) || !std::isfinite(d->norm_offset[1]))
      return GRIN_ERR_INVALID_ARG;
    m.pclass = grin::kN2P;
    for (int k = 0; k < 3; ++k) {
      m.off[k] = k < 2 ? d->norm_offset[k] : 0.0;
      m.scale[k] = m.inv_scale[k] = 1.0;
    }
    for (int k = 0; k < 4; ++k) m.cglex[k] = m.c64[k] = c[k];
    m.c64[4] = 0.0;
    // base = n on the axis; the FP32 copy returns n - base (shift in c32[4])
    const double n_axis = std::pow(1.0 + std::pow(c[0] * c[0] / (c[1] * c[1]), c[2]), c[3]);
    float base_f = (float)n_axis;
    if (!(std::isfinite(base_f) && base_f > 0.0f)) base_f = 1.0f;
    m.base_f = base_f;
    m.base = (double)base_f;
    for (int k = 0; k < 4; ++k) m.c32[k] = (float)c[k];
    m.c32[4] = base_f;
  } else if (d->kind == GRIN_MEDIUM_POLY || d->kind == GRIN_MEDIUM_SPHERICAL) {
    const bool sph = d->kind == GRIN_MEDIUM_SPHERICAL;
    if (!d->coeffs || (!sph && (d->degree < 0 || d->degree > GRIN_MAX_DEGREE)))
      return GRIN_ERR_INVALID_ARG;
    if (d->form < GRIN_FORM_LINEAR || d->form > GRIN_FORM_RECIP) return GRIN_ERR_INVALID_ARG;
    if (d->form == GRIN_FORM_RECIP && !std::isfinite(d->form_c)) return GRIN_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k) {
      if (!std::isfinite(d->norm_offset[k]) || !std::isfinite(d->norm_scale[k]) ||
          d->norm_scale[k] == 0.0)
        return GRIN_ERR_INVALID_ARG;
      m.off[k] = d->norm_offset[k];
      m.inv_scale[k] = 1.0 / d->norm_scale[k];
    }
    if (sph) {
      // a0..a3 of the spherical freeform field, the same in every layout
      m.pclass = grin::kSpherical;
      for (int k = 0; k < 4; ++k) {
        if (!std::isfinite(d->coeffs[k])) return GRIN_ERR_INVALID_ARG;
        m.cglex[k] = m.c64[k] = d->coeffs[k];
      }
    } else {
      m.pclass = d->degree <= 2 ? grin::kPoly2 : (d->degree <= 4 ? grin::kPoly4 : grin::kPoly6);
      const int D = m.pclass;
      // graded-lex input: kept as is (zero padded to class D) and scattered
      // into the Horner layout of class D
      int idx = 0;
      for (int s = 0; s <= d->degree; ++s)
        for (int i = s; i >= 0; --i)
          for (int j = s - i; j >= 0; --j) {
            double c = d->coeffs[idx];
            if (!std::isfinite(c)) return GRIN_ERR_INVALID_ARG;
            m.cglex[idx++] = c;
            m.c64[grin::hidx(D, i, j, s - i - j)] = c;
          }
    }
    for (int k = 0; k < 3; ++k) m.scale[k] = d->norm_scale[k];
    const double c0 = m.c64[0];  // hidx(D, 0, 0, 0) == 0; a0 of the spherical field
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
    for (int k = 0; k < grin::kMaxTerms; ++k) m.c32s[2 * k] = m.c32[k];
  } else {
    if (!samples) return GRIN_ERR_INVALID_ARG;
    if (!d->grid || d->nx < 1 || d->ny < 1 || d->nz < 1) return GRIN_ERR_INVALID_ARG;
    const int64_t cnt = (int64_t)d->nx * d->ny * d->nz;
    if (cnt >= (int64_t(1) << 31)) return GRIN_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k) {
      if (!finite_pos(d->spacing[k]) || !std::isfinite(d->origin[k])) return GRIN_ERR_INVALID_ARG;
      m.origin[k] = d->origin[k];
      m.spacing[k] = d->spacing[k];
      m.inv_spacing[k] = 1.0 / d->spacing[k];
    }
    m.nx = d->nx;
    m.ny = d->ny;
    m.nz = d->nz;
    m.grid_n = cnt;
    m.rows16 = d->nx % 4 == 0;  // the device copy is cudaMalloc'd (256-byte aligned)
    try {
      samples->resize((size_t)cnt);
    } catch (...) {
      return GRIN_ERR_OOM;
    }
    if (d->grid_on_device) {
      if (cudaMemcpy(samples->data(), d->grid, (size_t)cnt * sizeof(float), cudaMemcpyDeviceToHost) !=
          cudaSuccess) {
        cudaGetLastError();
        return GRIN_ERR_INVALID_ARG;
      }
    } else {
      std::memcpy(samples->data(), d->grid, (size_t)cnt * sizeof(float));
    }
    float lo = INFINITY, hi = -INFINITY;
    for (float v : *samples) {
      if (!std::isfinite(v)) return GRIN_ERR_INVALID_ARG;
      lo = std::min(lo, v);
      hi = std::max(hi, v);
    }
    // FP32 interpolation subtracts this value from every tap (exact for
    // samples within a factor two of it), the samples stay as given
    float base_f = (float)(0.5 * ((double)lo + (double)hi));
    if (!(std::isfinite(base_f) && base_f != 0.0f)) base_f = 1.0f;
    m.base_f = base_f;
    m.base = (double)base_f;
  }
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
    m.noff_f[k] = (float)(-m.off[k] * m.inv_scale[k]);
    m.origin_f[k] = (float)m.origin[k];
    m.inv_spacing_f[k] = (float)m.inv_spacing[k];
    m.origin_lo_f[k] = (float)(m.origin[k] - (double)m.origin_f[k]);
    m.inv_spacing_lo_f[k] = (float)(m.inv_spacing[k] - (double)m.inv_spacing_f[k]);
  }
  for (int k = 0; k < 8; ++k) m.b_f[k] = (float)m.b[k];
  return GRIN_OK;
}

extern "C" {

const char* grin_status_string(int status) {
  switch (status) {
    case GRIN_OK: return "ok";
    case GRIN_ERR_INVALID_ARG: return "invalid argument";
    case GRIN_ERR_OOM: return "out of memory";
    case GRIN_ERR_CUDA: return "CUDA runtime error";
    case GRIN_ERR_NOT_IMPLEMENTED: return "not implemented";
    case GRIN_ERR_TIMEOUT: return "timed out";
    case GRIN_ERR_BUSY: return "busy";
    case GRIN_ERR_NOT_FOUND: return "not found";
    case GRIN_ERR_CANCELLED: return "cancelled";
    case GRIN_ERR_CHECKED_BOUNDS: return "index out of bounds (checked build)";
    default: return "unknown status";
  }
}

int grin_poly_terms(int degree) {
  if (degree < 0 || degree > GRIN_MAX_DEGREE) return 0;
  return (degree + 1) * (degree + 2) * (degree + 3) / 6;
}

// The per-device word of the bounds-checked build (allocated with the first
// context on the device; 4 bytes, also in the ordinary build).
static unsigned int* g_oob[256] = {};
static std::mutex g_oob_mutex;

static unsigned int* oob_word(int device) {
  std::lock_guard<std::mutex> lock(g_oob_mutex);
  if (device < 0 || device >= 256) return nullptr;
  if (!g_oob[device]) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(p, 0, sizeof(unsigned int)) != cudaSuccess) {
      cudaGetLastError();
      if (p) cudaFree(p);
      return nullptr;
    }
    g_oob[device] = (unsigned int*)p;
  }
  return g_oob[device];
}

int grin_build_checked(void) {
#ifdef GRIN_CHECKED
  return 1;
#else
  return 0;
#endif
}

int grin_checked_status(int device, int32_t* site) {
  if (!site) return GRIN_ERR_INVALID_ARG;
  *site = 0;
  unsigned int* w = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_oob_mutex);
    if (device < 0 || device >= 256) return GRIN_ERR_INVALID_ARG;
    w = g_oob[device];
  }
  int dev_prev = 0;
  if (cudaGetDevice(&dev_prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GRIN_ERR_CUDA;
  }
  int st = GRIN_OK;
  unsigned int v = 0;
  if (w) {
    if (cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(w, 0, sizeof(unsigned int)) != cudaSuccess)
      st = GRIN_ERR_CUDA;
  }
  unsigned int vs = 0;
  if (st == GRIN_OK && grin::static_oob_take(&vs) != GRIN_OK) st = GRIN_ERR_CUDA;
  cudaSetDevice(dev_prev);
  if (st != GRIN_OK) {
    cudaGetLastError();
    return st;
  }
  *site = (int32_t)(v ? v : vs);
  return *site ? GRIN_ERR_CHECKED_BOUNDS : GRIN_OK;
}

namespace {
// Forms the index one past the end of a one-sample grid; the check records
// site kSiteGridFP64 and redirects it to 0 (nothing is read or written).
__global__ void k_checked_selftest(grin::DevMedium m, int64_t* sink) {
  const int64_t i = GRIN_IDX(m, m.grid_n + (int64_t)threadIdx.x, m.grid_n, kSiteGridFP64);
  if (i != 0) *sink = i;  // never taken; keeps the index computed
}
}  // namespace

int grin_checked_selftest(int device) {
#ifdef GRIN_CHECKED
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return GRIN_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) return GRIN_ERR_CUDA;
  grin::DevMedium m;
  std::memset(&m, 0, sizeof(m));
  m.grid_n = 1;
  m.oob = oob_word(device);
  if (!m.oob) return GRIN_ERR_OOM;
  if (grin::launch_kernel(k_checked_selftest, 1, 1, nullptr, m, (int64_t*)nullptr) < 0)
    return GRIN_ERR_CUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? GRIN_OK : GRIN_ERR_CUDA;
#else
  (void)device;
  return GRIN_ERR_NOT_IMPLEMENTED;
#endif
}

int grin_ctx_create(int device, grin_ctx* out) {
  if (!out) return GRIN_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) return GRIN_ERR_CUDA;
  if (device < 0 || device >= n) return GRIN_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return GRIN_ERR_CUDA;
  grin_ctx c = new (std::nothrow) grin_ctx_s;
  if (!c) return GRIN_ERR_OOM;
  c->device = device;
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return GRIN_ERR_CUDA;
  }
  if (cudaMalloc(&c->queues, kQueueSlots * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return GRIN_ERR_OOM;
  }
  *out = c;
  return GRIN_OK;
}

// The context's stream-ordered pool, created on first use with no release
// threshold, so blocks freed by one call are reused by the next.
static bool order_pool(grin_ctx ctx) {
  if (ctx->pool) return true;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = ctx->device;
  if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) {
    cudaGetLastError();
    ctx->pool = nullptr;
    return false;
  }
  uint64_t keep = UINT64_MAX;
  cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  return true;
}

int grin_ctx_destroy(grin_ctx ctx) {
  if (!ctx) return GRIN_ERR_INVALID_ARG;
  if (ctx->children.load() != 0) return GRIN_ERR_BUSY;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(ctx->queues);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  for (cudaStream_t h : ctx->hs)
    if (h) cudaStreamDestroy(h);
  for (cudaEvent_t e : ctx->hev)
    if (e) cudaEventDestroy(e);
  if (ctx->stats) cudaFree(ctx->stats);
  for (cudaEvent_t e : ctx->tev)
    if (e) cudaEventDestroy(e);
  delete ctx;
  return GRIN_OK;
}

int grin_ctx_last_launches(grin_ctx ctx, int32_t* launches) {
  if (!ctx || !launches) return GRIN_ERR_INVALID_ARG;
  *launches = ctx->last_launches;
  return GRIN_OK;
}

int grin_medium_create(grin_ctx ctx, const grin_medium_desc* d, grin_medium* out) {
  if (!ctx || !d || !out) return GRIN_ERR_INVALID_ARG;
  *out = nullptr;
  DevMedium m;
  std::vector<float> samples;
  const int st = grin::describe_medium(d, &m, &samples);
  if (st != GRIN_OK) return st;

  m.oob = oob_word(ctx->device);
  if (!m.oob) return GRIN_ERR_OOM;
  grin_medium med = new (std::nothrow) grin_medium_s;
  if (!med) return GRIN_ERR_OOM;
  med->ctx = ctx;
  if (d->kind == GRIN_MEDIUM_GRID) {
    cudaSetDevice(ctx->device);
    med->grid_bytes = samples.size() * sizeof(float);
    if (cudaMalloc(&med->grid_dev, med->grid_bytes) != cudaSuccess) {
      cudaGetLastError();
      delete med;
      return GRIN_ERR_OOM;
    }
    if (cudaMemcpy(med->grid_dev, samples.data(), med->grid_bytes, cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      cudaFree(med->grid_dev);
      delete med;
      return GRIN_ERR_CUDA;
    }
    m.grid = med->grid_dev;
  }
  med->dm = m;
  ++ctx->children;
  *out = med;
  return GRIN_OK;
}

int grin_medium_destroy(grin_medium medium) {
  if (!medium) return GRIN_ERR_INVALID_ARG;
  if (medium->grid_dev) {
    cudaSetDevice(medium->ctx->device);
    cudaDeviceSynchronize();
    cudaFree(medium->grid_dev);
  }
  --medium->ctx->children;
  delete medium;
  return GRIN_OK;
}

int grin_medium_device_bytes(grin_medium medium, size_t* bytes) {
  if (!medium || !bytes) return GRIN_ERR_INVALID_ARG;
  *bytes = medium->grid_bytes;
  return GRIN_OK;
}

// out == nullptr: a call that writes no results (the adjoint's backward sweep)
static int check_trace_args(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                            const grin_params* p, const grin_out* out, bool need_out = true) {
  static const grin_out kNoOut = {};
  if (!need_out && !out) out = &kNoOut;
  if (!ctx || !medium || !rays || !p || !out) return GRIN_ERR_INVALID_ARG;
  if (medium->ctx != ctx) return GRIN_ERR_INVALID_ARG;
  if (rays->count < 0) return GRIN_ERR_INVALID_ARG;
  if (rays->dtype != GRIN_F32 && rays->dtype != GRIN_F64) return GRIN_ERR_INVALID_ARG;
  if (!finite_pos(p->dopl) || p->max_steps < 0 || (p->flags & ~(uint32_t)GRIN_TRACE_LEVEL_ROOT))
    return GRIN_ERR_INVALID_ARG;
  if (p->precision != GRIN_PREC_FP64 && p->precision != GRIN_PREC_FP32_MIXED &&
      p->precision != GRIN_PREC_FP64_FAST)
    return GRIN_ERR_INVALID_ARG;
  // the fast FP64 tracer keeps neither margins nor the shell-crossing variant
  if (p->precision == GRIN_PREC_FP64_FAST && (p->flags || out->margin))
    return GRIN_ERR_NOT_IMPLEMENTED;
  if (rays->count == 0) return GRIN_OK;
  if (!rays->ox || !rays->oy || !rays->oz || !rays->dx || !rays->dy || !rays->dz)
    return GRIN_ERR_INVALID_ARG;
  if (!need_out) return GRIN_OK;
  if (!out->px || !out->py || !out->pz || !out->dx || !out->dy || !out->dz || !out->opl ||
      !out->exit_id || !out->steps || !out->tir_internal || !out->tir_boundary)
    return GRIN_ERR_INVALID_ARG;
  return GRIN_OK;
}

int grin_trace_path(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                    const grin_params* p, const grin_out* out, double* path, int64_t cap,
                    int64_t* path_len, void* cuda_stream) {
  int st = check_trace_args(ctx, medium, rays, p, out);
  if (st != GRIN_OK) return st;
  if (p->precision != GRIN_PREC_FP64 || cap < 1 || !path || !path_len)
    return GRIN_ERR_INVALID_ARG;
  if (rays->count > 0 && cap > INT64_MAX / 3 / rays->count) return GRIN_ERR_INVALID_ARG;
  ctx->last_launches = 0;
  if (rays->count == 0) return GRIN_OK;
  grin::TraceArgs a;
  a.ox = rays->ox;
  a.oy = rays->oy;
  a.oz = rays->oz;
  a.dx = rays->dx;
  a.dy = rays->dy;
  a.dz = rays->dz;
  a.count = rays->count;
  a.dtype = rays->dtype;
  a.px = out->px;
  a.py = out->py;
  a.pz = out->pz;
  a.ux = out->dx;
  a.uy = out->dy;
  a.uz = out->dz;
  a.opl = out->opl;
  a.exit_id = out->exit_id;
  a.steps = out->steps;
  a.tir_i = out->tir_internal;
  a.tir_b = out->tir_boundary;
  a.dopl = p->dopl;
  a.max_steps = p->max_steps;
  a.flags = p->flags;
  a.margin = out->margin;
  int rc = grin::launch_fp64_path(medium->dm, a, path, cap, path_len, (cudaStream_t)cuda_stream);
  if (rc < 0) return rc;
  ctx->last_launches = rc;
  return GRIN_OK;
}

// The timing events of grin_trace (created once); false if unavailable.
static bool trace_events(grin_ctx ctx) {
  if (ctx->tev[0]) return true;
  if (cudaEventCreate(&ctx->tev[0]) == cudaSuccess && cudaEventCreate(&ctx->tev[1]) == cudaSuccess)
    return true;
  cudaGetLastError();
  for (cudaEvent_t& e : ctx->tev)
    if (e) cudaEventDestroy(e), e = nullptr;
  return false;
}

static int trace_launches(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                          const grin_params* p, const grin_out* out, cudaStream_t s);

int grin_trace(grin_ctx ctx, grin_medium medium, const grin_rays* rays, const grin_params* p,
               const grin_out* out, void* cuda_stream) {
  int st = check_trace_args(ctx, medium, rays, p, out);
  if (st != GRIN_OK) return st;
  ctx->last_launches = 0;
  ctx->timed = false;
  if (rays->count == 0) return GRIN_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // device time of the call, from events around its kernels (not on a
  // capturing stream, where a recorded event would become part of a graph)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool timed = cudaStreamIsCapturing(s, &cap) == cudaSuccess &&
                     cap == cudaStreamCaptureStatusNone && trace_events(ctx) &&
                     cudaEventRecord(ctx->tev[0], s) == cudaSuccess;
  cudaGetLastError();
  const int rc = trace_launches(ctx, medium, rays, p, out, s);
  if (rc < 0) return rc;
  ctx->timed = timed && cudaEventRecord(ctx->tev[1], s) == cudaSuccess;
  ctx->last_launches = rc;
  return GRIN_OK;
}

// grin_trace's kernels: the number launched, or a negative grin_status.
static int trace_launches(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                          const grin_params* p, const grin_out* out, cudaStream_t s) {
  grin::TraceArgs a;
  a.ox = rays->ox;
  a.oy = rays->oy;
  a.oz = rays->oz;
  a.dx = rays->dx;
  a.dy = rays->dy;
  a.dz = rays->dz;
  a.count = rays->count;
  a.dtype = rays->dtype;
  a.px = out->px;
  a.py = out->py;
  a.pz = out->pz;
  a.ux = out->dx;
  a.uy = out->dy;
  a.uz = out->dz;
  a.opl = out->opl;
  a.exit_id = out->exit_id;
  a.steps = out->steps;
  a.tir_i = out->tir_internal;
  a.tir_b = out->tir_boundary;
  a.dopl = p->dopl;
  a.max_steps = p->max_steps;
  a.flags = p->flags;
  a.margin = out->margin;
  int rc;
  if (p->precision == GRIN_PREC_FP64) {
    rc = grin::launch_fp64(medium->dm, a, s, ctx->sm_count);
  } else if (p->precision == GRIN_PREC_FP64_FAST) {
    rc = grin::launch_fp64_fast(medium->dm, a, s, ctx->sm_count);
  } else {
    unsigned long long* q = ctx->queues + ctx->next_queue;
    ctx->next_queue = (ctx->next_queue + 1) % kQueueSlots;
    // large batches in a gridded medium: claim rays in the order of where
    // they enter it (ray_order.cu), so a warp's stencils overlap, from scratch
    // allocated and freed on this call's stream.  Analytic media are ALU-bound
    // and keep index order, whose ray reads and result writes coalesce.
    void* order = nullptr;
    int lo = 0;
    if (medium->dm.kind == GRIN_MEDIUM_GRID && a.count >= grin::kOrderMinRays &&
        a.count < (int64_t(1) << 31) && order_pool(ctx) &&
        cudaMallocFromPoolAsync(&order, grin::order_scratch_bytes(a.count), ctx->pool, s) ==
            cudaSuccess) {
      lo = grin::launch_order(medium->dm, a, order, ctx->sm_count, s, &a.perm);
      if (lo < 0) {
        a.perm = nullptr;
        lo = 0;
      }
    } else {
      cudaGetLastError();
      order = nullptr;
    }
    rc = grin::launch_mixed(medium->dm, a, q, s, ctx->sm_count);
    if (order) cudaFreeAsync(order, s);
    if (rc >= 0) rc += lo;
  }
  return rc;
}

int grin_trace_stats_compute(grin_ctx ctx, const grin_out* out, int64_t count,
                             const double* margin_min, grin_trace_stats* stats,
                             void* cuda_stream) {
  if (!ctx || !out || !stats || count < 0) return GRIN_ERR_INVALID_ARG;
  if (count > 0 && (!out->exit_id || !out->steps || !out->tir_internal || !out->tir_boundary))
    return GRIN_ERR_INVALID_ARG;
  if (margin_min && !out->margin) return GRIN_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  if (!ctx->stats &&
      cudaMalloc(&ctx->stats, grin::kStatWords * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    ctx->stats = nullptr;
    return GRIN_ERR_OOM;
  }
  grin::TraceArgs a{};
  a.count = count;
  a.exit_id = out->exit_id;
  a.steps = out->steps;
  a.tir_i = out->tir_internal;
  a.tir_b = out->tir_boundary;
  a.margin = out->margin;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (grin::launch_stats(a, margin_min, ctx->stats, s) < 0) return GRIN_ERR_CUDA;
  unsigned long long w[grin::kStatWords];
  if (cudaMemcpyAsync(w, ctx->stats, sizeof(w), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return GRIN_ERR_CUDA;
  stats->rays = (int64_t)w[0];
  stats->ray_steps = (int64_t)w[1];
  for (int f = 0; f < 6; ++f) stats->exit_face[f] = (int64_t)w[2 + f];
  stats->exit_miss = (int64_t)w[8];
  stats->exit_entry_reflect = (int64_t)w[9];
  stats->exit_max_steps = (int64_t)w[10];
  stats->exit_invalid = (int64_t)w[11];
  stats->tir_internal = (int64_t)w[12];
  stats->tir_boundary = (int64_t)w[13];
  stats->flagged = margin_min ? (int64_t)w[14] : -1;
  stats->elapsed_ms = -1.0;
  float ms = 0.0f;
  if (ctx->timed && cudaEventSynchronize(ctx->tev[1]) == cudaSuccess &&
      cudaEventElapsedTime(&ms, ctx->tev[0], ctx->tev[1]) == cudaSuccess)
    stats->elapsed_ms = ms;
  cudaGetLastError();
  return GRIN_OK;
}

// The streams and events of grin_trace_host's pipeline, created once.
static bool host_pipeline(grin_ctx ctx) {
  if (ctx->hs[0]) return true;
  bool ok = true;
  for (cudaStream_t& h : ctx->hs)
    ok = ok && cudaStreamCreateWithFlags(&h, cudaStreamNonBlocking) == cudaSuccess;
  for (cudaEvent_t& e : ctx->hev)
    ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  if (ok) return true;
  cudaGetLastError();
  for (cudaStream_t& h : ctx->hs)
    if (h) cudaStreamDestroy(h), h = nullptr;
  for (cudaEvent_t& e : ctx->hev)
    if (e) cudaEventDestroy(e), e = nullptr;
  return false;
}

static grin_rays rays_at(const grin_rays& r, const void* const* base, int64_t off, int64_t cnt,
                         size_t esz) {
  grin_rays c = r;
  const void** f[6] = {&c.ox, &c.oy, &c.oz, &c.dx, &c.dy, &c.dz};
  for (int k = 0; k < 6; ++k) *f[k] = (const char*)base[k] + off * esz;
  c.count = cnt;
  return c;
}

int grin_trace_host(grin_ctx ctx, grin_medium medium, const grin_rays* rays, const grin_params* p,
                    const grin_out* out, void* cuda_stream) {
  int st = check_trace_args(ctx, medium, rays, p, out);
  if (st != GRIN_OK) return st;
  ctx->last_launches = 0;
  const int64_t n = rays->count;
  if (n == 0) return GRIN_OK;
  const size_t esz = rays->dtype == GRIN_F64 ? 8 : 4;
  const size_t in_bytes = 6 * esz * (size_t)n;
  const bool with_margin = out->margin != nullptr;
  const size_t out_bytes = (7 * 8 + 4 * 4 + (with_margin ? 32 : 0)) * (size_t)n;
  const size_t need = in_bytes + out_bytes + 256;
  if (ctx->stage_bytes < need) {
    if (ctx->stage) {
      cudaDeviceSynchronize();
      cudaFree(ctx->stage);
      ctx->stage = nullptr;
      ctx->stage_bytes = 0;
    }
    if (cudaMalloc(&ctx->stage, need) != cudaSuccess) {
      cudaGetLastError();
      return GRIN_ERR_OOM;
    }
    ctx->stage_bytes = need;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  char* base = (char*)ctx->stage;
  const void* hin[6] = {rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz};
  const void* din[6];
  for (int k = 0; k < 6; ++k) din[k] = base + k * esz * (size_t)n;
  char* ob = base + in_bytes;
  double* dd[7];
  for (int k = 0; k < 7; ++k) dd[k] = (double*)(ob + k * 8 * (size_t)n);
  int32_t* di[4];
  for (int k = 0; k < 4; ++k) di[k] = (int32_t*)(ob + 56 * (size_t)n + k * 4 * (size_t)n);
  double* dm = with_margin ? (double*)(ob + 72 * (size_t)n) : nullptr;  // 4 a ray
  double* hd[7] = {out->px, out->py, out->pz, out->dx, out->dy, out->dz, out->opl};
  int32_t* hi[4] = {out->exit_id, out->steps, out->tir_internal, out->tir_boundary};

  // Chunks of at least kHostChunkMin rays (a multiple of 1024), at most
  // kHostChunks of them; a batch below two chunks runs as one.
  int64_t chunk = n;
  if (n >= 2 * grin::kHostChunkMin) {
    chunk = (n + grin::kHostChunks - 1) / grin::kHostChunks;
    chunk = std::max<int64_t>(grin::kHostChunkMin, (chunk + 1023) / 1024 * 1024);
  }
  const int nchunks = (int)((n + chunk - 1) / chunk);
  const bool piped = nchunks > 1 && host_pipeline(ctx);
  // Upload, trace, download of chunk i are ordered by events; chunk i + 1's
  // upload and chunk i - 1's download overlap chunk i's trace, and the traces
  // alternate between two streams so that the next chunk's kernel takes over
  // the SMs the previous one frees.  A single chunk runs on the caller's
  // stream.
  cudaStream_t up = piped ? ctx->hs[0] : s, down = piped ? ctx->hs[3] : s;
  if (piped) {
    cudaEvent_t start = ctx->hev[2 * grin::kHostChunks];
    bool ok = cudaEventRecord(start, s) == cudaSuccess;
    for (cudaStream_t h : ctx->hs) ok = ok && cudaStreamWaitEvent(h, start, 0) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return GRIN_ERR_CUDA;
    }
  }
  int launches = 0;
  for (int i = 0; i < (piped ? nchunks : 1) && st == GRIN_OK; ++i) {
    const int64_t off = piped ? (int64_t)i * chunk : 0;
    const int64_t cnt = piped ? std::min<int64_t>(chunk, n - off) : n;
    cudaStream_t ts = piped ? ctx->hs[1 + (i & 1)] : s;
    for (int k = 0; k < 6 && st == GRIN_OK; ++k)
      if (cudaMemcpyAsync((char*)din[k] + off * esz, (const char*)hin[k] + off * esz,
                          esz * (size_t)cnt, cudaMemcpyHostToDevice, up) != cudaSuccess)
        st = GRIN_ERR_CUDA;
    if (st == GRIN_OK && piped &&
        (cudaEventRecord(ctx->hev[2 * i], up) != cudaSuccess ||
         cudaStreamWaitEvent(ts, ctx->hev[2 * i], 0) != cudaSuccess))
      st = GRIN_ERR_CUDA;
    if (st != GRIN_OK) break;
    grin_rays dr = rays_at(*rays, din, off, cnt, esz);
    grin_out dout = {dd[0] + off, dd[1] + off, dd[2] + off, dd[3] + off, dd[4] + off, dd[5] + off,
                     dd[6] + off, di[0] + off, di[1] + off, di[2] + off, di[3] + off,
                     with_margin ? dm + 4 * off : nullptr};
    st = grin_trace(ctx, medium, &dr, p, &dout, ts);
    if (st != GRIN_OK) break;
    launches += ctx->last_launches;
    if (piped && (cudaEventRecord(ctx->hev[2 * i + 1], ts) != cudaSuccess ||
                  cudaStreamWaitEvent(down, ctx->hev[2 * i + 1], 0) != cudaSuccess)) {
      st = GRIN_ERR_CUDA;
      break;
    }
    for (int k = 0; k < 7 && st == GRIN_OK; ++k)
      if (cudaMemcpyAsync(hd[k] + off, dd[k] + off, 8 * (size_t)cnt, cudaMemcpyDeviceToHost,
                          down) != cudaSuccess)
        st = GRIN_ERR_CUDA;
    for (int k = 0; k < 4 && st == GRIN_OK; ++k)
      if (cudaMemcpyAsync(hi[k] + off, di[k] + off, 4 * (size_t)cnt, cudaMemcpyDeviceToHost,
                          down) != cudaSuccess)
        st = GRIN_ERR_CUDA;
    if (with_margin && st == GRIN_OK &&
        cudaMemcpyAsync(out->margin + 4 * off, dm + 4 * off, 32 * (size_t)cnt,
                        cudaMemcpyDeviceToHost, down) != cudaSuccess)
      st = GRIN_ERR_CUDA;
  }
  // Nothing may still read or write the caller's buffers when this returns.
  bool synced = true;
  if (piped)
    for (cudaStream_t h : ctx->hs) synced = cudaStreamSynchronize(h) == cudaSuccess && synced;
  synced = cudaStreamSynchronize(s) == cudaSuccess && synced;
  if (st != GRIN_OK) {
    cudaGetLastError();
    return st;
  }
  ctx->last_launches = launches;
  return synced ? GRIN_OK : GRIN_ERR_CUDA;
}

int grin_trace_adjoint_workspace_size(grin_medium medium, int64_t ray_count, const grin_params* p,
                                      int32_t k, size_t* bytes) {
  if (!medium || !p || !bytes || ray_count < 0 || k < 1 || k > 64 || p->max_steps < 0)
    return GRIN_ERR_INVALID_ARG;
  if (!grin::adjoint_supported(medium->dm)) return GRIN_ERR_NOT_IMPLEMENTED;
  *bytes = grin::adjoint_workspace(ray_count, p->max_steps, k);
  return GRIN_OK;
}

int grin_trace_adjoint_interval(grin_medium medium, int64_t ray_count, const grin_params* p,
                                size_t budget_bytes, int32_t* k_out) {
  if (!medium || !p || !k_out || ray_count < 0 || p->max_steps < 0) return GRIN_ERR_INVALID_ARG;
  if (!grin::adjoint_supported(medium->dm)) return GRIN_ERR_NOT_IMPLEMENTED;
  // every step stored: the backward sweep recomputes nothing
  if (grin::adjoint_workspace(ray_count, p->max_steps, 1) <= budget_bytes) {
    *k_out = 1;
    return GRIN_OK;
  }
  // otherwise every step is recomputed once whatever K is; the smallest K
  // that fits keeps the thread's segment records shortest
  for (int32_t k = 2; k <= 64; ++k)
    if (grin::adjoint_workspace(ray_count, p->max_steps, k) <= budget_bytes) {
      *k_out = k;
      return GRIN_OK;
    }
  return GRIN_ERR_OOM;
}

// The forward sweep, the backward sweep or both (grin::AdjPhase); out and g
// as the phase needs them.
static int trace_adjoint_phase(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                               const grin_params* p, const grin_out* out, const grin_out_grad* g,
                               double* grad, int32_t k, void* ws, size_t ws_bytes, void* cuda_stream,
                               int phase) {
  static const grin_out kNoOut = {};
  const bool backward_only = phase == grin::kAdjBackward;
  int st = check_trace_args(ctx, medium, rays, p, backward_only ? nullptr : out, !backward_only);
  if (st != GRIN_OK) return st;
  if (backward_only) out = &kNoOut;  // the backward sweep writes no results
  if (!ws || k < 1 || k > 64 || p->precision != GRIN_PREC_FP64) return GRIN_ERR_INVALID_ARG;
  if (phase != grin::kAdjForward && (!g || !grad)) return GRIN_ERR_INVALID_ARG;
  if (p->flags || out->margin) return GRIN_ERR_NOT_IMPLEMENTED;
  if (!grin::adjoint_supported(medium->dm)) return GRIN_ERR_NOT_IMPLEMENTED;
  ctx->last_launches = 0;
  if (rays->count == 0) return GRIN_OK;
  if (ws_bytes < grin::adjoint_workspace(rays->count, p->max_steps, k)) return GRIN_ERR_INVALID_ARG;
  const double* gout[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (phase != grin::kAdjForward) {
    const double* gg[7] = {g->px, g->py, g->pz, g->dx, g->dy, g->dz, g->opl};
    for (int q = 0; q < 7; ++q) {
      if (!gg[q]) return GRIN_ERR_INVALID_ARG;
      gout[q] = gg[q];
    }
  }
  grin::TraceArgs a;
  a.ox = rays->ox;
  a.oy = rays->oy;
  a.oz = rays->oz;
  a.dx = rays->dx;
  a.dy = rays->dy;
  a.dz = rays->dz;
  a.count = rays->count;
  a.dtype = rays->dtype;
  a.px = out->px;
  a.py = out->py;
  a.pz = out->pz;
  a.ux = out->dx;
  a.uy = out->dy;
  a.uz = out->dz;
  a.opl = out->opl;
  a.exit_id = out->exit_id;
  a.steps = out->steps;
  a.tir_i = out->tir_internal;
  a.tir_b = out->tir_boundary;
  a.dopl = p->dopl;
  a.max_steps = p->max_steps;
  a.flags = p->flags;
  a.margin = out->margin;
  const grin::DevMedium& m = medium->dm;
  // polynomial: its coefficients; N2P lens: R, F, beta, gamma; spherical freeform: a0 .. a3
  int nterms = m.kind == GRIN_MEDIUM_POLY ? grin_poly_terms(m.pclass)
               : (m.kind == GRIN_MEDIUM_N2P || m.kind == GRIN_MEDIUM_SPHERICAL) ? 4 : 0;
  int rc = grin::launch_adjoint(m, a, k, ws, phase == grin::kAdjForward ? nullptr : gout, grad, nterms,
                                (cudaStream_t)cuda_stream, phase);
  if (rc < 0) return rc;
  ctx->last_launches = rc;
  return GRIN_OK;
}

int grin_trace_adjoint(grin_ctx ctx, grin_medium medium, const grin_rays* rays, const grin_params* p,
                       const grin_out* out, const grin_out_grad* g, double* grad, int32_t k,
                       void* ws, size_t ws_bytes, void* cuda_stream) {
  if (!g || !grad) return GRIN_ERR_INVALID_ARG;
  return trace_adjoint_phase(ctx, medium, rays, p, out, g, grad, k, ws, ws_bytes, cuda_stream,
                             grin::kAdjBoth);
}

int grin_trace_adjoint_forward(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                               const grin_params* p, const grin_out* out, int32_t k, void* ws,
                               size_t ws_bytes, void* cuda_stream) {
  return trace_adjoint_phase(ctx, medium, rays, p, out, nullptr, nullptr, k, ws, ws_bytes,
                             cuda_stream, grin::kAdjForward);
}

int grin_trace_adjoint_backward(grin_ctx ctx, grin_medium medium, const grin_rays* rays,
                                const grin_params* p, const grin_out_grad* g, double* grad,
                                int32_t k, void* ws, size_t ws_bytes, void* cuda_stream) {
  return trace_adjoint_phase(ctx, medium, rays, p, nullptr, g, grad, k, ws, ws_bytes, cuda_stream,
                             grin::kAdjBackward);
}

}  // extern "C"
