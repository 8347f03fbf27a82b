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

/* Fault injection on the host side of the refinement: rounds the stored
 * FP32 inverse Schur blocks of subdomain `sub` (the context's order:
 * realisations in turn, each row-major by subdomain row then column) to
 * `mantissa_bits` explicit mantissa bits, ties to even (7: bfloat16), so that
 * the subdomain's FP32 refinement in the next mrcm_build_basis stalls on a
 * high-contrast field as a low-precision factor would.  Call it between
 * mrcm_factor_local and mrcm_build_basis.  MRCM_EINVAL: NULL context, an FP64
 * context, sub out of range, mantissa_bits outside 1..22, or a 16 x 16
 * subdomain whose FP32 factor the basis kernel forms itself (not stored).
 * Asynchronous on the context's stream.  (No counterpart in the paper.) */
mrcm_status mrcm_test_degrade_factor(mrcm_ctx *ctx, int32_t sub, int32_t mantissa_bits);

/* The integer-pipe conversions between binary32 and binary64 that the FP32
 * refinement loops of the local solves use (IEEE 754 encodings, round to
 * nearest, ties to even), against the hardware conversions.  For every i in
 * [start, start + count): the float with bit pattern i mod 2^32 is converted
 * to double; four doubles derived from i are converted to float: a hashed
 * 64-bit pattern, the value of float pattern i times (1 + k 2^-24) for
 * k = i/8 mod 4 (rounding ties and near-ties), and that float scaled by
 * 2^-(40 + i mod 128) and by 2^(i mod 128) (subnormal, zero and overflow
 * results).  Results must agree bit for bit; a NaN input must give a NaN.
 * d_mismatch (device, two uint64) accumulates the float->double and the
 * double->float mismatch counts.  count at most 2^32; synchronises the
 * stream.  MRCM_EINVAL: NULL d_mismatch or count out of range.  (No
 * counterpart in the paper.) */
mrcm_status mrcm_test_fp_convert(uint64_t start, uint64_t count, uint64_t *d_mismatch,
                                 void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MRCM_TESTING_H */
