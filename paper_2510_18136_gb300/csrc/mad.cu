// Robust noise normalisation of arXiv 2510.18136 Sec. 2.2 ("median subtracted in each pixel ...
// normalized by the running standard deviation"; read here as per (pixel, subband) median and
// 1.4826 MAD over the window) as a pass of its own ahead of the search: every (pixel, subband) row
// of a slab of pixels is normalised once, x <- (x - median) / (1.4826 MAD), into an FP32 slab that
// the barrier-free search then reads like any FP32 cube with unit noise per sample.
//
// One warp per row: the row goes to shared memory, the median and the MAD come from the radix
// selection of the search kernel's own MAD path (the same selected values, the same FP32
// operations, so the normalised rows are bit-identical to those the search kernel forms in place).
// A zero MAD marks the pixel invalid (bad[pixel] = 1, its rows are written as zeros).
#include <algorithm>

#include "nsfrb.h"
#include "search_impl.cuh"

namespace nsfrb {
namespace {

constexpr int kMadWarps = 8;

__global__ void __launch_bounds__(kMadWarps * 32) mad_normalise_kernel(const void *__restrict__ cube, int dtype,
                                                                     int64_t pix0, int64_t n_pix, int n_sub, int n_t,
                                                                     float *__restrict__ out,
                                                                     uint8_t *__restrict__ bad) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t row_bytes = align_up(sizeof(float) * static_cast<size_t>(n_t), 16);
    float *row = reinterpret_cast<float *>(smem + warp * (2 * row_bytes + sizeof(uint32_t) * kHistBins));
    float *dev = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(row) + row_bytes);
    uint32_t *hist = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(row) + 2 * row_bytes);
    const int64_t n_rows = n_pix * n_sub;
    for (int64_t r = static_cast<int64_t>(blockIdx.x) * kMadWarps + warp; r < n_rows;
         r += static_cast<int64_t>(gridDim.x) * kMadWarps) {
        const int64_t src = (pix0 * n_sub + r) * n_t;
        for (int t = lane; t < n_t; t += 32) row[t] = dev::load_elem(cube, src + t, dtype);
        __syncwarp();
        const float med = dev::warp_median(row, n_t, hist, dtype == NSFRB_BF16);
        for (int t = lane; t < n_t; t += 32) dev[t] = fabsf(row[t] - med);
        __syncwarp();
        const float mad = dev::warp_median(dev, n_t, hist, false);
        float *dst = out + r * n_t;
        if (mad == 0.0f) {
            for (int t = lane; t < n_t; t += 32) dst[t] = 0.0f;
            if (lane == 0) bad[pix0 + r / n_sub] = 1;
        } else {
            const float inv = 1.0f / (1.4826f * mad);
            for (int t = lane; t < n_t; t += 32) dst[t] = (row[t] - med) * inv;
        }
        __syncwarp();
    }
}

}  // namespace

size_t mad_smem_bytes(int n_t) {
    return kMadWarps * (2 * align_up(sizeof(float) * static_cast<size_t>(n_t), 16) + sizeof(uint32_t) * kHistBins);
}

cudaError_t launch_mad_normalise(const void *cube, int dtype, int64_t pix0, int64_t n_pix, int n_sub, int n_t,
                                 float *out, uint8_t *bad, int n_sm, cudaStream_t s) {
    const size_t smem = mad_smem_bytes(n_t);
    const cudaError_t e = cudaFuncSetAttribute(mad_normalise_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int64_t rows = n_pix * n_sub;
    const int64_t blocks = std::min<int64_t>((rows + kMadWarps - 1) / kMadWarps, static_cast<int64_t>(n_sm) * 4);
    mad_normalise_kernel<<<static_cast<unsigned>(std::max<int64_t>(1, blocks)), kMadWarps * 32, smem, s>>>(
        cube, dtype, pix0, n_pix, n_sub, n_t, out, bad);
    return cudaGetLastError();
}

}  // namespace nsfrb
