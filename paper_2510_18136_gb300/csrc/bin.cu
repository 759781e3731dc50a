// Time binning for the longer search timescales of arXiv 2510.18136 Sec. 2.2
// (0.67 s = 5 samples and 10.05 s = 75 samples of 134 ms): each (pixel,
// subband) row of n_t samples becomes n_t / factor sums of `factor`
// consecutive samples (a trailing remainder is dropped).  FP32 output.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "plan_internal.h"

namespace nsfrb {
namespace {

template <typename T>
__device__ __forceinline__ float widen(T v);
template <>
__device__ __forceinline__ float widen<float>(float v) { return v; }
template <>
__device__ __forceinline__ float widen<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float widen<__half>(__half v) { return __half2float(v); }

// One thread per output sample; consecutive threads read consecutive input runs.
template <typename T>
__global__ void bin_kernel(const T *__restrict__ in, int64_t n_rows, int n_t, int factor, float *__restrict__ out) {
    const int n_out = n_t / factor;
    const int64_t total = n_rows * n_out;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = i / n_out;
        const int j = static_cast<int>(i - r * n_out);
        const T *src = in + r * n_t + static_cast<int64_t>(j) * factor;
        float acc = 0.0f;
        for (int q = 0; q < factor; ++q) acc += widen<T>(src[q]);
        out[i] = acc;
    }
}

}  // namespace
}  // namespace nsfrb

using namespace nsfrb;

extern "C" nsfrb_status nsfrb_bin_time(const void *d_in, int32_t dtype, int64_t n_rows, int32_t n_t, int32_t factor,
                                       float *d_out, void *stream) {
    if (!d_in || !d_out || n_rows < 0 || n_t < 1 || factor < 1 || factor > n_t || dtype < NSFRB_F32 ||
        dtype > NSFRB_F16)
        return fail(nullptr, NSFRB_EINVAL, "bad argument");
    const int64_t total = n_rows * (n_t / factor);
    if (total == 0) return NSFRB_OK;
    const int bs = 256;
    const int grid = static_cast<int>(std::min<int64_t>((total + bs - 1) / bs, 152 * 64));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == NSFRB_F32)
        bin_kernel<float><<<grid, bs, 0, s>>>(static_cast<const float *>(d_in), n_rows, n_t, factor, d_out);
    else if (dtype == NSFRB_BF16)
        bin_kernel<__nv_bfloat16><<<grid, bs, 0, s>>>(static_cast<const __nv_bfloat16 *>(d_in), n_rows, n_t, factor,
                                                     d_out);
    else
        bin_kernel<__half><<<grid, bs, 0, s>>>(static_cast<const __half *>(d_in), n_rows, n_t, factor, d_out);
    return cuda_check(nullptr, cudaGetLastError(), "bin launch");
}
