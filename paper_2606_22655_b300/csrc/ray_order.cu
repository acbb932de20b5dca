// ray_order.cu -- the order in which the persistent ray pool claims rays.
//
// Rays that start near each other follow similar paths for a while, so lanes
// of one warp that hold neighbouring rays read overlapping samples of a
// gridded medium (the 64-tap Catmull-Rom stencil) and meet the surface and
// the rare cases at similar steps.  Before a large mixed-precision trace the
// rays are therefore bucketed by where they first meet the medium's bounding
// box: that point is quantised to 32 cells per axis and the three 5-bit cell
// indices are interleaved into a 15-bit Morton key; a counting sort over the
// 32,768 keys gives a permutation, which the pool follows when it claims
// rays.  Each ray's arithmetic does not depend on its lane or on when it is
// claimed, so results are bitwise those of the unsorted order; only the
// order within one key is left to the atomics.
#include "grin_device.cuh"

namespace grin {

constexpr int kCellBits = 5;
constexpr int kKeys = 1 << (3 * kCellBits);  // 32768
constexpr int kScanThreads = 1024;

// Spreads the low 5 bits of v to every third bit.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  uint32_t r = 0;
#pragma unroll
  for (int b = 0; b < kCellBits; ++b) r |= ((v >> b) & 1u) << (3 * b);
  return r;
}

// Axis-aligned bounding box of the enclosing surface.
__device__ __forceinline__ void surface_bbox(const DevMedium& m, double* lo, double* hi) {
  const double* b = m.b;
  if (m.bkind == GRIN_BOUNDARY_BOX) {
    for (int k = 0; k < 3; ++k) {
      lo[k] = b[k];
      hi[k] = b[3 + k];
    }
  } else if (m.bkind == GRIN_BOUNDARY_SPHERE) {
    for (int k = 0; k < 3; ++k) {
      lo[k] = b[k] - b[3];
      hi[k] = b[k] + b[3];
    }
  } else {
    lo[0] = b[0] - b[2];
    hi[0] = b[0] + b[2];
    lo[1] = b[1] - b[2];
    hi[1] = b[1] + b[2];
    lo[2] = b[3];
    hi[2] = b[4];
  }
}

__global__ void k_order_keys(DevMedium m, TraceArgs a, uint16_t* keys, uint32_t* hist) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double lo[3], hi[3];
  surface_bbox(m, lo, hi);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.count; r += stride) {
    double p[3] = {ld(a.ox, r, a.dtype), ld(a.oy, r, a.dtype), ld(a.oz, r, a.dtype)};
    const double d[3] = {ld(a.dx, r, a.dtype), ld(a.dy, r, a.dtype), ld(a.dz, r, a.dtype)};
    // slab entry into the box when the origin is outside it
    double tn = 0.0, tf = INFINITY;
    for (int k = 0; k < 3; ++k) {
      if (d[k] != 0.0) {
        double t1 = (lo[k] - p[k]) / d[k], t2 = (hi[k] - p[k]) / d[k];
        tn = fmax(tn, fmin(t1, t2));
        tf = fmin(tf, fmax(t1, t2));
      }
    }
    if (tn <= tf && isfinite(tn))
      for (int k = 0; k < 3; ++k) p[k] += tn * d[k];
    uint32_t key = 0;
    for (int k = 0; k < 3; ++k) {
      double u = (p[k] - lo[k]) / (hi[k] - lo[k]) * (double)(1 << kCellBits);
      int c = isfinite(u) ? (int)fmin(fmax(u, 0.0), (double)((1 << kCellBits) - 1)) : 0;
      key |= spread3((uint32_t)c) << k;
    }
    keys[r] = (uint16_t)key;
    atomicAdd(hist + key, 1u);
  }
}

// Exclusive prefix sum of the kKeys counts, in place, by one block: each
// thread sums its run of kKeys / kScanThreads counts, the run totals are
// scanned in shared memory, then each thread writes its run's offsets.
__global__ void __launch_bounds__(kScanThreads) k_order_scan(uint32_t* hist) {
  constexpr int kRun = kKeys / kScanThreads;
  __shared__ uint32_t tot[kScanThreads];
  const int t = threadIdx.x;
  uint32_t s = 0;
  for (int i = 0; i < kRun; ++i) s += hist[t * kRun + i];
  tot[t] = s;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {
    uint32_t v = t >= off ? tot[t - off] : 0u;
    __syncthreads();
    tot[t] += v;
    __syncthreads();
  }
  uint32_t run = tot[t] - s;  // exclusive start of this thread's run
  for (int i = 0; i < kRun; ++i) {
    const uint32_t c = hist[t * kRun + i];
    hist[t * kRun + i] = run;
    run += c;
  }
}

__global__ void k_order_scatter(int64_t n, const uint16_t* keys, uint32_t* next, uint32_t* perm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride)
    perm[atomicAdd(next + keys[r], 1u)] = (uint32_t)r;
}

// perm (n uint32), keys (n uint16) and the counts, each 256-byte aligned.
size_t order_scratch_bytes(int64_t n) {
  const size_t perm = ((size_t)n * sizeof(uint32_t) + 255) & ~size_t(255);
  const size_t keys = ((size_t)n * sizeof(uint16_t) + 255) & ~size_t(255);
  return perm + keys + (size_t)kKeys * sizeof(uint32_t);
}

// Key of the adjoint's backward sweep: rays by step count, longest first,
// so a warp's threads walk back through similar numbers of steps.
__global__ void k_order_steps(int64_t n, const int32_t* meta, uint16_t* keys, uint32_t* hist) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    const int st = min(max(meta[2 * r + 1], 0), kKeys - 1);
    const uint32_t key = (uint32_t)(kKeys - 1 - st);
    keys[r] = (uint16_t)key;
    atomicAdd(hist + key, 1u);
  }
}

struct OrderBufs {
  uint32_t* perm;
  uint16_t* keys;
  uint32_t* hist;
};

static OrderBufs order_bufs(void* scratch, int64_t n) {
  char* p = (char*)scratch;
  OrderBufs b;
  b.perm = (uint32_t*)p;
  p += ((size_t)n * sizeof(uint32_t) + 255) & ~size_t(255);
  b.keys = (uint16_t*)p;
  p += ((size_t)n * sizeof(uint16_t) + 255) & ~size_t(255);
  b.hist = (uint32_t*)p;
  return b;
}

// The scan and the scatter, after a key kernel has filled keys and hist.
static int finish_order(const OrderBufs& b, int64_t n, unsigned blocks, cudaStream_t s,
                        const uint32_t** perm_out) {
  if (launch_kernel(k_order_scan, 1, kScanThreads, s, b.hist) < 0) return GRIN_ERR_CUDA;
  if (launch_kernel(k_order_scatter, blocks, 256, s, n, (const uint16_t*)b.keys, b.hist, b.perm) < 0)
    return GRIN_ERR_CUDA;
  *perm_out = b.perm;
  return 2;
}

static bool clear_hist(const OrderBufs& b, cudaStream_t s) {
  if (cudaMemsetAsync(b.hist, 0, kKeys * sizeof(uint32_t), s) == cudaSuccess) return true;
  cudaGetLastError();
  return false;
}

int launch_order(const DevMedium& m, const TraceArgs& a, void* scratch, int sm_count,
                 cudaStream_t s, const uint32_t** perm_out) {
  if (a.count <= 0 || a.count >= (int64_t(1) << 31)) return GRIN_ERR_INVALID_ARG;
  const OrderBufs b = order_bufs(scratch, a.count);
  if (!clear_hist(b, s)) return GRIN_ERR_CUDA;
  const unsigned blocks = (unsigned)sm_count * 8;
  if (launch_kernel(k_order_keys, blocks, 256, s, m, a, b.keys, b.hist) < 0) return GRIN_ERR_CUDA;
  const int rc = finish_order(b, a.count, blocks, s, perm_out);
  return rc < 0 ? rc : rc + 1;
}

int launch_order_by_steps(const int32_t* meta, int64_t n, void* scratch, cudaStream_t s,
                          const uint32_t** perm_out) {
  if (n <= 0 || n >= (int64_t(1) << 31)) return GRIN_ERR_INVALID_ARG;
  const OrderBufs b = order_bufs(scratch, n);
  if (!clear_hist(b, s)) return GRIN_ERR_CUDA;
  const int64_t want = (n + 255) / 256;
  const unsigned blocks = (unsigned)(want < 4096 ? want : 4096);
  if (launch_kernel(k_order_steps, blocks, 256, s, n, meta, b.keys, b.hist) < 0) return GRIN_ERR_CUDA;
  const int rc = finish_order(b, n, blocks, s, perm_out);
  return rc < 0 ? rc : rc + 1;
}

}  // namespace grin
