/*
 * mrcm_testing.h — test hooks of the GB300 MRCM library (not part of the
 * solve).  They expose single internal kernels so that tests can compare
 * them with references directly.
 */
#ifndef MRCM_TESTING_H
#define MRCM_TESTING_H

#include <stdint.h>
#include "mrcm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One n x n FP32 GEMM of the large-slab interface factor:
 *   C = alpha (A1 B1 + A2 B2) (+ C if acc),  row-major, device pointers,
 * A2/B2 may be NULL.  impl 0: the SIMT kernel; impl 1: the tcgen05 kernel
 * (3 x TF32 split products, FP32 accumulation in tensor memory).  d_status
 * (device int) receives MRCM_FLAG_TIMEOUT if a bounded wait of the tensor-core
 * kernel ran out.  Synchronises the stream. */
mrcm_status mrcm_test_gemm(int32_t impl, int32_t n, const float *d_a1, const float *d_b1,
                           const float *d_a2, const float *d_b2, float *d_c, double alpha,
                           int32_t acc, int32_t *d_status, void *cuda_stream);

/* Failure detection without a fault: runs the tensor-core kernels' bounded
 * mbarrier wait (the one behind MRCM_ETIMEOUT, include/mrcm.h) on a barrier
 * that nothing completes, giving up after limit tries (1 .. 2^26); the probe
 * kernel then raises MRCM_FLAG_TIMEOUT in d_status (device int) and returns,
 * leaving the context usable.  MRCM_EINVAL for a NULL d_status or a limit out
 * of range.  Synchronises the stream.  (No counterpart in the paper.) */
mrcm_status mrcm_test_wait_timeout(uint32_t limit, int32_t *d_status, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MRCM_TESTING_H */
