/*
 * grin_probe.h -- measurement probes of the B300 VRT library, for the
 * roofline denominators its benchmark reports the tracers against.  The
 * paper has no counterpart.  Both run on the calling thread's current device
 * on the legacy default stream, synchronise, and return a grin_status.
 */
#ifndef GRIN_PROBE_H
#define GRIN_PROBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* FP32 FMA rate of the CUDA cores: every SM runs 8 blocks of 256 threads,
 * each thread 8 independent fused-multiply-add chains for `iters` rounds
 * (>= 1; one shorter warm-up launch first).  *flops_per_s counts an FMA as
 * 2 FLOPs; *seconds (may be NULL) is the timed launch's duration. */
int grin_probe_fp32_fma(int64_t iters, double* flops_per_s, double* seconds);

/* Read bandwidth of an L2-resident buffer: `bytes` (>= 16 KiB; take it well
 * below the L2's 126 MB) allocated and zeroed on the device, read once to
 * warm L2, then read `rounds` times (16-byte cached-in-L2 loads) in one timed
 * launch; the buffer is freed before return.  GRIN_ERR_OOM if it cannot be
 * allocated. */
int grin_probe_l2_read(size_t bytes, int rounds, double* bytes_per_s);

#ifdef __cplusplus
}
#endif
#endif /* GRIN_PROBE_H */
