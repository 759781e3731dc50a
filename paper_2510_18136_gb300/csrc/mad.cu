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
constexpr int kPerLane = (kMaxT + 31) / 32;   // samples of a row per lane

// The values a selection runs over: v[t], or |v[t] - c| (the deviations from the median,
// formed when read rather than stored).
struct RowView {
    const float *v;
    float c;
    bool dev;
    __device__ __forceinline__ float at(int t) const { return dev ? fabsf(v[t] - c) : v[t]; }
};

// Exact order statistic of rank `rank` (0-based) of the view's n values by one warp: 8-bit radix
// passes over the order-preserving key from the top byte down, as the search kernel's MAD path
// selects (with key16 the low 16 key bits are fixed by the sign: two passes).  Returns the key.
__device__ uint32_t select_key(const RowView &f, int n, int rank, uint32_t *hist, bool key16) {
    const int lane = threadIdx.x & 31;
    uint32_t prefix = 0, pmask = 0;
    const int last = key16 ? 16 : 0;
#pragma unroll 1
    for (int shift = 24; shift >= last; shift -= 8) {
#pragma unroll
        for (int j = 0; j < dev::kHistBinsPerLane; ++j) hist[32 * j + lane] = 0;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
            const int t = 32 * j + lane;
            if (t < n) {
                const uint32_t key = dev::f2key(f.at(t));
                if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
            }
        }
        __syncwarp();
        uint32_t cnt[8];
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            cnt[j] = hist[8 * lane + j];
            s += cnt[j];
        }
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(dev::kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - s;
        const bool mine = (static_cast<uint32_t>(rank) >= excl) && (static_cast<uint32_t>(rank) < incl);
        const unsigned bal = __ballot_sync(dev::kFull, mine);
        const int src = __ffs(bal) - 1;
        int digit = 0;
        uint32_t before = 0;
        if (mine) {
            uint32_t acc = excl;
            bool done = false;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (!done && static_cast<uint32_t>(rank) < acc + cnt[j]) {
                    digit = 8 * lane + j;
                    before = acc;
                    done = true;
                }
                acc += cnt[j];
            }
        }
        digit = __shfl_sync(dev::kFull, digit, src);
        before = __shfl_sync(dev::kFull, before, src);
        rank -= static_cast<int>(before);
        prefix |= static_cast<uint32_t>(digit) << shift;
        pmask |= 255u << shift;
        __syncwarp();
    }
    if (key16) prefix |= (prefix & 0x80000000u) ? 0u : 0xffffu;
    return prefix;
}

// Median of the view's values: the middle order statistic, or for even n the mean of the two
// middle ones, the upper from the lower (it equals the lower when more than n / 2 keys are at
// most the lower's, else it is the smallest key above it).
__device__ float median_view(const RowView &f, int n, uint32_t *hist, bool key16) {
    const uint32_t ka = select_key(f, n, (n - 1) / 2, hist, key16);
    const float a = dev::key2f(ka);
    if (n & 1) return a;
    const int lane = threadIdx.x & 31;
    uint32_t le = 0, above = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < kPerLane; ++j) {
        const int t = 32 * j + lane;
        if (t < n) {
            const uint32_t key = dev::f2key(f.at(t));
            if (key <= ka)
                ++le;
            else
                above = min(above, key);
        }
    }
    le = __reduce_add_sync(dev::kFull, le);
    above = __reduce_min_sync(dev::kFull, above);
    const float b = (le >= static_cast<uint32_t>(n / 2) + 1) ? a : dev::key2f(above);
    return 0.5f * (a + b);
}

__global__ void __launch_bounds__(kMadWarps * 32, 4) mad_normalise_kernel(const void *__restrict__ cube, int dtype,
                                                                     int64_t pix0, int64_t n_pix, int n_sub, int n_t,
                                                                     float *__restrict__ out,
                                                                     uint8_t *__restrict__ bad, int vec) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t row_bytes = align_up(sizeof(float) * static_cast<size_t>(n_t), 16);
    float *row = reinterpret_cast<float *>(smem + warp * (row_bytes + sizeof(uint32_t) * kHistBins));
    uint32_t *hist = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(row) + row_bytes);
    const int64_t n_rows = n_pix * n_sub;
    for (int64_t r = static_cast<int64_t>(blockIdx.x) * kMadWarps + warp; r < n_rows;
         r += static_cast<int64_t>(gridDim.x) * kMadWarps) {
        const int64_t src = (pix0 * n_sub + r) * n_t;
        if (vec) {
            // 16-byte loads, a lane's all in flight together: 8 16-bit or 4 FP32 samples each
            if (dtype == NSFRB_F32) {
                const float4 *g = reinterpret_cast<const float4 *>(static_cast<const float *>(cube) + src);
#pragma unroll
                for (int j = 0; j < (kPerLane * 32 + 127) / 128; ++j) {
                    const int q = 32 * j + lane;
                    if (q < n_t / 4) reinterpret_cast<float4 *>(row)[q] = __ldg(g + q);
                }
            } else {
                const uint4 *g = reinterpret_cast<const uint4 *>(static_cast<const unsigned short *>(cube) + src);
#pragma unroll
                for (int j = 0; j < (kPerLane * 32 + 255) / 256; ++j) {
                    const int q = 32 * j + lane;
                    if (q < n_t / 8) {
                        const uint4 u = __ldg(g + q);
                        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
                        float4 a, b;
                        float *o = &a.x;
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            float *oo = h < 2 ? &a.x + 2 * h : &b.x + 2 * (h - 2);
                            oo[0] = dev::widen16(static_cast<unsigned short>(w[h] & 0xffffu), dtype);
                            oo[1] = dev::widen16(static_cast<unsigned short>(w[h] >> 16), dtype);
                        }
                        (void)o;
                        reinterpret_cast<float4 *>(row)[2 * q] = a;
                        reinterpret_cast<float4 *>(row)[2 * q + 1] = b;
                    }
                }
            }
        } else {
            for (int t = lane; t < n_t; t += 32) row[t] = dev::load_elem(cube, src + t, dtype);
        }
        __syncwarp();
        const float med = median_view(RowView{row, 0.0f, false}, n_t, hist, dtype == NSFRB_BF16);
        const float mad = median_view(RowView{row, med, true}, n_t, hist, false);
        float *dst = out + r * n_t;
        if (mad == 0.0f) {
            for (int t = lane; t < n_t; t += 32) dst[t] = 0.0f;
            if (lane == 0) bad[pix0 + r / n_sub] = 1;
        } else {
            const float inv = 1.0f / (1.4826f * mad);
#pragma unroll
            for (int j = 0; j < kPerLane; ++j) {
                const int t = 32 * j + lane;
                if (t < n_t) dst[t] = (row[t] - med) * inv;
            }
        }
        __syncwarp();
    }
}

}  // namespace

size_t mad_smem_bytes(int n_t) {
    return kMadWarps * (align_up(sizeof(float) * static_cast<size_t>(n_t), 16) + sizeof(uint32_t) * kHistBins);
}

cudaError_t launch_mad_normalise(const void *cube, int dtype, int64_t pix0, int64_t n_pix, int n_sub, int n_t,
                                 float *out, uint8_t *bad, int n_sm, cudaStream_t s) {
    const size_t smem = mad_smem_bytes(n_t);
    cudaError_t e = cudaFuncSetAttribute(mad_normalise_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mad_normalise_kernel, kMadWarps * 32, smem);
    if (e != cudaSuccess) return e;
    // 16-byte loads need 16-byte aligned rows (a 16-byte aligned cube, rows a multiple of 16 bytes)
    const size_t es = dtype == NSFRB_F32 ? 4 : 2;
    const int vec = (reinterpret_cast<uintptr_t>(cube) % 16 == 0 && (es * n_t) % 16 == 0) ? 1 : 0;
    const int64_t rows = n_pix * n_sub;
    const int64_t blocks = std::min<int64_t>((rows + kMadWarps - 1) / kMadWarps,
                                             static_cast<int64_t>(n_sm) * std::max(1, per_sm));
    mad_normalise_kernel<<<static_cast<unsigned>(std::max<int64_t>(1, blocks)), kMadWarps * 32, smem, s>>>(
        cube, dtype, pix0, n_pix, n_sub, n_t, out, bad, vec);
    return cudaGetLastError();
}

}  // namespace nsfrb
