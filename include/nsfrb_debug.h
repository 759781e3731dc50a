/*
 * nsfrb_debug.h -- test hooks of libnsfrb (not part of the search API).
 * They expose internal building blocks so that tests can check them against
 * library routines; the paper has no counterpart.
 */
#ifndef NSFRB_DEBUG_H
#define NSFRB_DEBUG_H

#include "nsfrb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The classifier's BF16 tensor-core GEMM with FP32 accumulation, on device
 * buffers, asynchronous on `stream`:
 *   tn == 0:  C[M][N]  = A[M][K] * B[N][K]^T   (A, B K-contiguous)
 *   tn != 0:  C[M][N]  = A[K][M]^T * B[K][N]    (split-K, C zeroed first)
 * A, B: BF16; C: FP32.  K, and M and N for tn != 0, must be multiples of 8.
 * EINVAL for other shapes. */
nsfrb_status nsfrb_dbg_gemm(int32_t tn, int32_t M, int32_t N, int32_t K, const void *d_a, const void *d_b,
                            float *d_c, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NSFRB_DEBUG_H */
