// Candidate compaction (Fig. 1 / Sec. 2.2: candidates are the pixels whose
// maximum S/N is above the threshold) and selection of the pixels that are
// re-scored from FP32 data when the cube is stored in 16-bit form.
#include "nsfrb_internal.h"

namespace nsfrb {
namespace {

// Count of candidate pixels per block of kCompactBlock pixels.
__global__ void __launch_bounds__(kCompactBlock) count_kernel(const PixRec *rec, int64_t n, float thr,
                                                             int32_t *counts) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kCompactBlock + threadIdx.x;
    const int flag = (i < n) && (rec[i].snr > thr);
    const int total = __syncthreads_count(flag);
    if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// Deterministic scatter: block offset = sum of earlier block counts, in-block
// order by pixel index (warp ballots + warp-count prefix).
__global__ void __launch_bounds__(kCompactBlock) scatter_kernel(const PixRec *rec, int64_t n, int32_t nx,
                                                               float thr, const int32_t *counts,
                                                               int32_t n_blocks, CandRec *out,
                                                               int32_t *n_out) {
    __shared__ int32_t s_warp[kCompactBlock / 32];
    __shared__ int32_t s_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        int32_t acc = 0;
        for (int b = lane; b < static_cast<int>(blockIdx.x); b += 32) acc += counts[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_off = acc;
    }
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kCompactBlock + threadIdx.x;
    const bool flag = (i < n) && (rec[i].snr > thr);
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    int32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    const int32_t pos = s_off + before + __popc(bal & ((1u << lane) - 1u));
    if (flag) {
        const PixRec r = rec[i];
        out[pos] = CandRec{static_cast<int32_t>(i / nx), static_cast<int32_t>(i % nx), r.dm_idx, r.w_idx,
                           r.t_idx, r.snr};
    }
    if (blockIdx.x == n_blocks - 1 && threadIdx.x == 0) {
        int32_t tot = 0;
        for (int w = 0; w < kCompactBlock / 32; ++w) tot += s_warp[w];
        *n_out = s_off + tot;
    }
}

__global__ void rescore_select_kernel(const PixRec *rec, int64_t n, float thr, float eps, int32_t *list,
                                      int32_t *n_list) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = rec[i].snr;
    if (s >= thr - eps && s <= thr + eps) {
        const int32_t at = atomicAdd(n_list, 1);
        list[at] = static_cast<int32_t>(i);
    }
}

}  // namespace

cudaError_t launch_compact(const PixRec *rec, int64_t n_pix, int32_t nx, float thr, int32_t *block_counts,
                           int32_t n_blocks, CandRec *out, int32_t *n_out, cudaStream_t s) {
    count_kernel<<<n_blocks, kCompactBlock, 0, s>>>(rec, n_pix, thr, block_counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scatter_kernel<<<n_blocks, kCompactBlock, 0, s>>>(rec, n_pix, nx, thr, block_counts, n_blocks, out, n_out);
    return cudaGetLastError();
}

cudaError_t launch_rescore_select(const PixRec *rec, int64_t n_pix, float thr, float eps, int32_t *list,
                                  int32_t *n_list, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(n_list, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int bs = 256;
    const int64_t nb = (n_pix + bs - 1) / bs;
    rescore_select_kernel<<<static_cast<unsigned>(nb), bs, 0, s>>>(rec, n_pix, thr, eps, list, n_list);
    return cudaGetLastError();
}

}  // namespace nsfrb
