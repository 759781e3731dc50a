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

/* One 3x3x3 convolution of the classifier (Sec. 2.3; zero padding 1) on device buffers,
 * asynchronous on `stream`:
 *   y[b][z][y][x][co] = sum over taps (dz, dy, dx) and ci of
 *                       w[co][(dz * 3 + dy) * 3 + dx][ci] * x[b][z + dz - 1][y + dy - 1][x + dx - 1][ci]
 * x: BF16 [B][D][H][W][CI] (channels last), w: BF16 [CO][27][CI], y: FP32 [B][D][H][W][CO].
 * d_part (may be NULL): per 128-voxel brick of the kernel that ran, the column sums of y and
 * of y^2 ([brick][2][CO], FP32); d_err: device int32 that a kernel ORs error bits into.
 * path 0: the library's choice (tcgen05 kernel, else the mma.sync halo kernel);
 * path 1: the mma.sync halo kernel only; path 2: the tcgen05 kernel only;
 * path 3: the tcgen05 kernel with its halo producers stalled, so that its bounded waits run
 *         out (after about 2 s): it then ORs 4 into *d_err, frees its tensor memory and returns
 *         without touching y (failure-path test).
 * EINVAL when the requested path has no kernel for the shape, channels or shared memory.
 * *h_used (host int32, may be NULL) receives 1 (halo kernel) or 2 (tcgen05 kernel). */
nsfrb_status nsfrb_dbg_conv3(int32_t path, int32_t B, int32_t D, int32_t H, int32_t W, int32_t CI, int32_t CO,
                             const void *d_x, const void *d_w, float *d_y, float *d_part, int32_t *d_err,
                             int32_t *h_used, void *stream);

/* The library's bounded device wait, on its own: a kernel waits on an mbarrier that nothing
 * arrives at, gives up after limit_ms (1..5000) and latches an error bit, which the host reads.
 * Returns NSFRB_ETIMEOUT when the wait ran out as it must (the device stays usable), NSFRB_OK
 * if it did not, EINVAL for a bad limit.  Synchronous. */
nsfrb_status nsfrb_dbg_wait_timeout(int32_t limit_ms);

/* The MAD normalisation pass of the search (Sec. 2.2, robust reading) on its own, asynchronous on
 * `stream`: for each of the n_rows rows of n_t samples of d_in (`dtype` storage, row-major),
 *   m = median, MAD = median |x - m| (exact order statistics; for even n_t the mean of the two
 *   middle values, formed in FP32), y = (x - m) * (1 / (1.4826 MAD)) in FP32,
 * into d_out [n_rows][n_t] FP32; a row with MAD 0 is written as zeros and sets d_bad[row] = 1
 * (d_bad: n_rows bytes, zeroed here first).  n_t in [1, 1247].  EINVAL for other sizes. */
nsfrb_status nsfrb_dbg_mad_normalise(const void *d_in, int32_t dtype, int64_t n_rows, int32_t n_t, float *d_out,
                                     uint8_t *d_bad, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NSFRB_DEBUG_H */
