/*
 * bsm_probe.h -- peak-rate probes of libbsm.so (GB300, sm_103a).
 *
 * The paper has no counterpart: these calls measure, on the device they run
 * on, the rates that bound the library's kernels, so that a roofline fraction
 * can be stated against a measured denominator.  Each call runs one launch on
 * every SM of the current device, times it with CUDA events on `stream`
 * (cudaStream_t as void*, NULL = legacy default stream), synchronises, and
 * returns the work done and the time.  The clock the device ran at is not
 * controlled or reported here; sample it alongside (nvidia-smi) to compare
 * runs.  Every mbarrier wait inside is bounded (TIMEOUT instead of a hang).
 * Return codes are bsm_status values (bsm.h).
 */
#ifndef BSM_PROBE_H
#define BSM_PROBE_H

#include <stdint.h>

#include "bsm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* FP64 probe kinds: mma.sync f64 tensor-core shapes, and scalar DFMA. */
enum {
  BSM_PROBE_DMMA_M8N8K4 = 0, /* the shape of the library's FP64 kernel */
  BSM_PROBE_DMMA_M16N8K4 = 1,
  BSM_PROBE_DMMA_M16N8K8 = 2,
  BSM_PROBE_DMMA_M16N8K16 = 3,
  BSM_PROBE_DFMA = 4,
  BSM_PROBE_MIXED = 5 /* half the warps DMMA m8n8k4, half DFMA (8 rounds per DMMA round):
                         whether the two share one FP64 pipe */
};

/*
 * bsm_probe_fp64 -- FP64 rate with register operands: blocks of 256 threads
 * at full occupancy on every SM, eight independent accumulator chains per
 * thread, `iters` rounds of eight instructions each.
 *   kind    a BSM_PROBE_* value above
 *   iters   >= 1 (about 2e4 rounds per 0.1 s at GB300's FP64 rate for m8n8k4)
 *   flops   receives the flops executed (2 per multiply-add)
 *   ms      receives the launch's duration (CUDA events)
 * Errors: INVALID_ARG, OOM, CUDA.
 */
bsm_status bsm_probe_fp64(int kind, int64_t iters, double *flops, float *ms, void *stream);

/*
 * bsm_probe_tcgen05 -- tcgen05.mma issue rate at M = 128 and a given N, as
 * the split kernel issues them: operands in shared memory (K-major core
 * matrices, no swizzle; an A tile is 4 KiB, a B tile n * 32 bytes), FP32
 * accumulators in TMEM, one CTA per SM, `iters` rounds of four instructions
 * per issuing thread alternating between two accumulators.
 *   fmt     0: kind::f16 BF16 x BF16 (K = 16 per instruction);
 *           1: kind::f8f6f4 E4M3 x E4M3 (K = 32)
 *   n       16..256, a multiple of 16
 *   tiles   1..8: consecutive instructions cycle through this many distinct
 *           (A, B) tile pairs (1: every instruction reads the same pair)
 *   issuers 1..4 threads (lane 0 of warps 0..issuers-1) each issue `iters`
 *           rounds into their own two accumulators (2 issuers n <= 512)
 *   flops   receives 2 * 128 * n * K * instructions
 *   ms      receives the launch's duration
 * Errors: INVALID_ARG, OOM, TIMEOUT, CUDA.
 */
bsm_status bsm_probe_tcgen05(int fmt, int n, int tiles, int issuers, int64_t iters, double *flops,
                             float *ms, void *stream);

/*
 * bsm_probe_bulk_copy -- HBM read rate of 1-D bulk copies (cp.async.bulk)
 * into shared memory: a device buffer of `bytes` (allocated and freed by the
 * call) is streamed in chunks of `stage_bytes` through a ring of `stages`
 * shared-memory stages per SM, one CTA per SM.
 *   stage_bytes  >= 1024, a multiple of 16; stages 2..8, their product
 *                <= 200 KiB
 *   bytes_moved  receives the bytes copied (bytes rounded down to stages)
 *   ms           receives the launch's duration
 * Errors: INVALID_ARG, OOM, TIMEOUT, CUDA.
 */
bsm_status bsm_probe_bulk_copy(int64_t bytes, int stage_bytes, int stages, double *bytes_moved,
                               float *ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BSM_PROBE_H */
