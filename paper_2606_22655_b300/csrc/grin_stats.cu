// grin_stats.cu -- totals of a trace's results on the device
// (grin_trace_stats_compute): a grid-stride pass over the rays, per-thread
// counters summed across the warp by shuffles, one atomic add per warp and
// counter.
#include "grin_device.cuh"

namespace grin {

// acc words: 0 rays, 1 ray-steps, 2..7 exits by face 0..5, 8 miss, 9 entry
// reflection, 10 step limit, 11 invalid, 12 internal TIRs, 13 boundary TIRs,
// 14 flagged rays
__global__ void k_stats(TraceArgs a, double m0, double m1, double m2, double m3, int use_margin,
                        unsigned long long* acc) {
  unsigned long long c[15] = {};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.count; r += stride) {
    const int e = a.exit_id[r];
    c[0] += 1;
    c[1] += (unsigned long long)max(a.steps[r], 0);
    if (e >= 0 && e < 6) c[2 + e] += 1;
    else if (e == GRIN_EXIT_MISS) c[8] += 1;
    else if (e == GRIN_EXIT_ENTRY_REFLECT) c[9] += 1;
    else if (e == GRIN_EXIT_MAXSTEPS) c[10] += 1;
    else c[11] += 1;
    c[12] += (unsigned long long)max(a.tir_i[r], 0);
    c[13] += (unsigned long long)max(a.tir_b[r], 0);
    if (use_margin) {
      const double* g = a.margin + 4 * r;
      c[14] += (g[0] < m0 || g[1] < m1 || g[2] < m2 || g[3] < m3) ? 1 : 0;
    }
  }
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    unsigned long long v = c[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31u) == 0 && v) atomicAdd(acc + k, v);
  }
}

int launch_stats(const TraceArgs& a, const double* mm, unsigned long long* acc, cudaStream_t st) {
  if (cudaMemsetAsync(acc, 0, kStatWords * sizeof(unsigned long long), st) != cudaSuccess)
    return GRIN_ERR_CUDA;
  if (a.count == 0) return 0;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (a.count + 255) / 256;
  const unsigned blocks = (unsigned)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
  return launch_kernel(k_stats, blocks, 256, st, a, mm ? mm[0] : 0.0, mm ? mm[1] : 0.0,
                       mm ? mm[2] : 0.0, mm ? mm[3] : 0.0, mm ? 1 : 0, acc);
}

}  // namespace grin
