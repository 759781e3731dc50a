// Test hook for the kernels' bounded waits: a kernel waits on an mbarrier that no thread ever
// arrives at, gives up after the limit like every wait in the library, latches the error bit
// and returns; the host reads the bit and reports NSFRB_ETIMEOUT.  Nothing traps or hangs.
#include <cuda_runtime.h>

#include "async_copy.cuh"
#include "nsfrb_debug.h"
#include "nsfrb_internal.h"
#include "plan_internal.h"

namespace nsfrb {
namespace {

__global__ void stalled_wait_kernel(int32_t *err, unsigned long long limit_ns) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // phase 0 never completes: nothing arrives
    if (!dev::mbar_wait_for(&bar, 0, limit_ns) && threadIdx.x == 0) atomicOr(err, ERR_WAIT_TIMEOUT);
}

}  // namespace
}  // namespace nsfrb

extern "C" nsfrb_status nsfrb_dbg_wait_timeout(int32_t limit_ms) {
    using namespace nsfrb;
    if (limit_ms < 1 || limit_ms > 5000) return NSFRB_EINVAL;
    int32_t *d_err = nullptr;
    if (cudaMalloc(&d_err, sizeof(int32_t)) != cudaSuccess) return NSFRB_ENOMEM;
    int32_t h_err = 0;
    cudaError_t e = cudaMemset(d_err, 0, sizeof(int32_t));
    if (e == cudaSuccess) {
        stalled_wait_kernel<<<1, 32>>>(d_err, static_cast<unsigned long long>(limit_ms) * 1000000ull);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h_err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaFree(d_err);
    if (e != cudaSuccess) return NSFRB_ECUDA;
    return (h_err & ERR_WAIT_TIMEOUT) ? NSFRB_ETIMEOUT : NSFRB_OK;
}

extern "C" nsfrb_status nsfrb_dbg_mad_normalise(const void *d_in, int32_t dtype, int64_t n_rows, int32_t n_t,
                                                float *d_out, uint8_t *d_bad, void *stream) {
    using namespace nsfrb;
    if (!d_in || !d_out || !d_bad || n_rows < 1 || n_t < 1 || n_t > kMaxT || dtype < NSFRB_F32 || dtype > NSFRB_F16)
        return NSFRB_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return NSFRB_ECUDA;
    // rows as pixels of one subband: bad[] is then per row
    if (cudaMemsetAsync(d_bad, 0, static_cast<size_t>(n_rows), s) != cudaSuccess) return NSFRB_ECUDA;
    if (launch_mad_normalise(d_in, dtype, 0, n_rows, 1, n_t, d_out, d_bad, n_sm, s) != cudaSuccess) return NSFRB_ECUDA;
    return NSFRB_OK;
}
