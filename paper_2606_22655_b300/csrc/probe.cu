// probe.cu -- measurement probes for the roofline denominators of the
// tracers' kernels: the FP32 fused-multiply-add rate of the CUDA cores and
// the read bandwidth of an L2-resident buffer, each timed with CUDA events
// on the device that is current.  The paper has no counterpart; bench.py
// reports the tracers against these measured peaks.
#include <cuda_runtime.h>

#include "grin_internal.h"
#include "grin_probe.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

// Each thread runs kChains independent FMA chains for `iters` rounds; the
// result is stored only if it matches an impossible value, so the chains
// are not removed and nothing is written.
__global__ void __launch_bounds__(256) k_fma(int64_t iters, float a, float b, float* sink) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == 1.2345e-30f) *sink = s;
}

// Sums n float4 of `src` (strided over the grid) `rounds` times.
__global__ void __launch_bounds__(256) k_read(const float4* __restrict__ src, int64_t n, int rounds,
                                              float* sink) {
  float acc = 0.0f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int r = 0; r < rounds; ++r)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const float4 v = __ldcg(src + i);
      acc += v.x + v.y + v.z + v.w;
    }
  if (acc == 1.2345e-30f) *sink = acc;
}

int sm_count(int* n) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRIN_ERR_CUDA;
  if (cudaDeviceGetAttribute(n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GRIN_ERR_CUDA;
  return GRIN_OK;
}

}  // namespace

extern "C" int grin_probe_fp32_fma(int64_t iters, double* flops_per_s, double* seconds) {
  if (!flops_per_s || iters < 1) return GRIN_ERR_INVALID_ARG;
  int sms = 0;
  if (sm_count(&sms) != GRIN_OK) return GRIN_ERR_CUDA;
  const unsigned blocks = (unsigned)sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GRIN_ERR_CUDA;
  int st = GRIN_OK;
  // one warm-up launch, then the timed one
  for (int rep = 0; rep < 2 && st == GRIN_OK; ++rep) {
    if (rep == 1 && cudaEventRecord(e0, nullptr) != cudaSuccess) st = GRIN_ERR_CUDA;
    if (st == GRIN_OK && grin::launch_kernel(k_fma, blocks, threads, nullptr, rep ? iters : iters / 8 + 1,
                                             1.0000001f, 1e-7f, (float*)nullptr) < 0)
      st = GRIN_ERR_CUDA;
  }
  float ms = 0.0f;
  if (st == GRIN_OK && (cudaEventRecord(e1, nullptr) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    st = GRIN_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GRIN_OK) return st;
  const double flops = 2.0 * kChains * (double)iters * blocks * threads;
  *flops_per_s = flops / (1e-3 * ms);
  if (seconds) *seconds = 1e-3 * ms;
  return GRIN_OK;
}

extern "C" int grin_probe_l2_read(size_t bytes, int rounds, double* bytes_per_s) {
  if (!bytes_per_s || bytes < 16 * 1024 || rounds < 1) return GRIN_ERR_INVALID_ARG;
  int sms = 0;
  if (sm_count(&sms) != GRIN_OK) return GRIN_ERR_CUDA;
  void* buf = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return GRIN_ERR_OOM;
  }
  int st = cudaMemset(buf, 0, bytes) == cudaSuccess ? GRIN_OK : GRIN_ERR_CUDA;
  const int64_t n = (int64_t)(bytes / 16);
  const unsigned blocks = (unsigned)sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = GRIN_ERR_CUDA;
  // one warm-up round brings the buffer into L2
  if (st == GRIN_OK && grin::launch_kernel(k_read, blocks, threads, nullptr, (const float4*)buf, n, 1,
                                           (float*)nullptr) < 0)
    st = GRIN_ERR_CUDA;
  float ms = 0.0f;
  if (st == GRIN_OK &&
      (cudaEventRecord(e0, nullptr) != cudaSuccess ||
       grin::launch_kernel(k_read, blocks, threads, nullptr, (const float4*)buf, n, rounds,
                           (float*)nullptr) < 0 ||
       cudaEventRecord(e1, nullptr) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
       cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    st = GRIN_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (st != GRIN_OK) {
    cudaGetLastError();
    return st;
  }
  *bytes_per_s = (double)n * 16.0 * rounds / (1e-3 * ms);
  return GRIN_OK;
}
