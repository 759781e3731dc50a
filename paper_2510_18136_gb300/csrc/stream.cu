// Real-time serving of arXiv 2510.18136 Sec. 2.2: blocks of n_blk samples
// (25 x 134 ms = 3.35 s in the paper) arrive per field and are searched as
// they come, with a 3.35 s timeout for missing subband images.  Here a plan
// keeps a rolling window of the last n_t samples on the device; each pushed
// block is transposed into the window and only the trials that end inside
// the new block are searched.  The per-block device work (transpose, masked
// search, compaction, window advance) is one captured CUDA graph.
//
// Ring layout: [n_pix][n_sub][ring_len] in the plan's storage type with
// ring_len >= 2 n_t + 8.  Sample a (absolute index) is stored at a mod n_t
// and again at a mod n_t + n_t, so the current window is always the
// contiguous slice [start, start + n_t) with start = (samples so far) mod n_t.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <thread>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "plan_internal.h"

namespace nsfrb {
namespace {

template <typename T>
__device__ __forceinline__ T narrow(float v);
template <>
__device__ __forceinline__ float narrow<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half narrow<__half>(float v) { return __float2half_rn(v); }

constexpr int kTrPix = 32;   // pixels per transpose tile

// blk [n_blk][n_sub][n_pix] FP32 -> ring rows, both copies; subbands whose
// bit is clear in *mask are written as zero.  One CTA per (32-pixel tile,
// subband); the tile is staged through shared memory so that both the reads
// (along pixels) and the writes (along samples) are contiguous.  With fring
// (re-score of 16-bit windows) the FP32 values also go to the FP32 window
// [n_t][n_sub][n_pix] (device or pinned host memory), a ring of n_t sample planes in the block's own
// layout, so that those writes are contiguous along pixels too.
template <typename T>
__global__ void ingest_kernel(const float *__restrict__ blk, T *__restrict__ ring, int64_t n_pix, int n_sub,
                              int n_blk, int n_t, int64_t ring_len, const int32_t *__restrict__ state,
                              const uint32_t *__restrict__ mask, float *__restrict__ fring) {
    extern __shared__ float tile[];   // [n_blk][kTrPix + 1]
    const int k = blockIdx.y;
    const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kTrPix;
    const bool present = (*mask >> k) & 1u;
    const int wpos = state[1];   // ring position of the block's first sample
    for (int i = threadIdx.x; i < n_blk * kTrPix; i += blockDim.x) {
        const int t = i / kTrPix, j = i % kTrPix;
        const int64_t p = p0 + j;
        float v = 0.0f;
        if (present && p < n_pix) v = blk[(static_cast<int64_t>(t) * n_sub + k) * n_pix + p];
        tile[t * (kTrPix + 1) + j] = v;
        if (fring && p < n_pix) {
            int pos = wpos + t;
            if (pos >= n_t) pos -= n_t;
            fring[(static_cast<int64_t>(pos) * n_sub + k) * n_pix + p] = v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_blk * kTrPix; i += blockDim.x) {
        const int j = i / n_blk, t = i % n_blk;
        const int64_t p = p0 + j;
        if (p >= n_pix) continue;
        int pos = wpos + t;
        if (pos >= n_t) pos -= n_t;
        const float f = tile[t * (kTrPix + 1) + j];
        const T v = narrow<T>(f);
        T *row = ring + (p * n_sub + k) * ring_len;
        row[pos] = v;
        row[pos + n_t] = v;
    }
}

// Advance the window after a block: window start = write position = samples mod n_t.
__global__ void advance_kernel(int32_t *state, int n_blk, int n_t) {
    int w = state[1] + n_blk;
    w %= n_t;
    state[1] = w;
    state[0] = w;
}

}  // namespace

void destroy_stream_state(nsfrb_plan_s *pl) {
    if (!pl->streaming) return;
    if (pl->s_stream) cudaStreamSynchronize(pl->s_stream);
    if (pl->s_graph) cudaGraphExecDestroy(pl->s_graph);
    if (pl->s_ev_push) cudaEventDestroy(pl->s_ev_push);
    if (pl->s_ev_done) cudaEventDestroy(pl->s_ev_done);
    if (pl->s_stream) cudaStreamDestroy(pl->s_stream);
    cudaFree(pl->d_ring);
    cudaFree(pl->d_blk);
    cudaFree(pl->d_sstate);
    if (pl->h_fring) cudaFreeHost(pl->h_fring);
    if (pl->fring_dev) cudaFree(pl->d_fring);
    pl->h_fring = nullptr;
    pl->d_fring = nullptr;
    pl->fring_dev = false;
    pl->streaming = false;
    cudaGetLastError();
}

static size_t ring_len_for(int n_t, int dtype) {
    const size_t a = dtype == NSFRB_F32 ? 4 : 8;
    return align_up(static_cast<size_t>(2 * n_t + 8), a);
}

}  // namespace nsfrb

using namespace nsfrb;

extern "C" {

nsfrb_status nsfrb_stream_bytes(nsfrb_plan_t plan, int32_t n_blk, size_t *bytes) {
    if (!plan || !bytes || n_blk < 1 || n_blk > plan->cfg.n_t) return fail(plan, NSFRB_EINVAL, "bad argument");
    const nsfrb_config &c = plan->cfg;
    const size_t n_pix = static_cast<size_t>(c.ny) * c.nx;
    const size_t ring = n_pix * c.n_sub * ring_len_for(c.n_t, c.dtype) * elem_size(c.dtype);
    const size_t blk = static_cast<size_t>(n_blk) * c.n_sub * n_pix * sizeof(float);
    const size_t work = n_pix * (sizeof(PixRec) + sizeof(CandRec) + sizeof(int32_t));
    *bytes = ring + blk + work + 4096;
    return NSFRB_OK;
}

nsfrb_status nsfrb_stream_window_info(nsfrb_plan_t plan, int32_t *fp32_window) {
    if (!plan || !fp32_window) return fail(plan, NSFRB_EINVAL, "null argument");
    if (!plan->streaming) return fail(plan, NSFRB_ENOTREADY, "no open stream");
    *fp32_window = plan->fring_dev ? 1 : (plan->h_fring ? 2 : 0);
    return NSFRB_OK;
}

nsfrb_status nsfrb_stream_open(nsfrb_plan_t plan, int32_t n_blk, size_t hbm_reserve) {
    if (!plan || n_blk < 1 || n_blk > plan->cfg.n_t) return fail(plan, NSFRB_EINVAL, "bad argument");
    if (plan->streaming) return fail(plan, NSFRB_EINVAL, "stream already open");
    if (plan->cfg.out_mode != NSFRB_OUT_CANDIDATES)
        return fail(plan, NSFRB_EINVAL, "streaming supports candidate output only");
    nsfrb_status st = ensure_device(plan);
    if (st != NSFRB_OK) return st;
    size_t need = 0;
    nsfrb_stream_bytes(plan, n_blk, &need);
    size_t free_b = 0, total_b = 0;
    if ((st = cuda_check(plan, cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo")) != NSFRB_OK) return st;
    if (free_b < need + hbm_reserve)
        return fail(plan, NSFRB_ENOMEM, "admission: not enough free device memory for this stream");
    const nsfrb_config &c = plan->cfg;
    const int64_t n_pix = static_cast<int64_t>(c.ny) * c.nx;
    plan->n_blk = n_blk;
    plan->ring_len = static_cast<int64_t>(ring_len_for(c.n_t, c.dtype));
    const size_t ring_bytes = static_cast<size_t>(n_pix) * c.n_sub * plan->ring_len * elem_size(c.dtype);
    if (cudaMalloc(&plan->d_ring, ring_bytes) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&plan->d_blk), sizeof(float) * n_blk * c.n_sub * n_pix) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&plan->d_sstate), 64) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(plan->d_ring);
        cudaFree(plan->d_blk);
        plan->d_ring = nullptr;
        plan->d_blk = nullptr;
        return fail(plan, NSFRB_ENOMEM, "stream buffers");
    }
    plan->streaming = true;
    plan->d_mask = reinterpret_cast<uint32_t *>(plan->d_sstate + 4);
    // re-score of 16-bit windows: the FP32 window, written by the ingest kernel and read back only
    // for the pixels near the threshold; in device memory if the free memory measured for the
    // admission also covers it beyond hbm_reserve (the ingest then writes it at HBM speed), else
    // in pinned host memory over the host link
    const bool rescore = c.dtype != NSFRB_F32 && c.rescore_eps > 0.0f;
    if (rescore) {
        const size_t fbytes = static_cast<size_t>(n_pix) * c.n_sub * c.n_t * sizeof(float);
        if (free_b >= need + fbytes + hbm_reserve &&
            cudaMalloc(reinterpret_cast<void **>(&plan->d_fring), fbytes) == cudaSuccess) {
            plan->fring_dev = true;
            if ((st = cuda_check(plan, cudaMemset(plan->d_fring, 0, fbytes), "FP32 window clear"))) {
                destroy_stream_state(plan);
                return st;
            }
        }
        cudaGetLastError();
    }
    if (rescore && !plan->fring_dev) {
        const size_t fbytes = static_cast<size_t>(n_pix) * c.n_sub * c.n_t * sizeof(float);
        if (cudaHostAlloc(reinterpret_cast<void **>(&plan->h_fring), fbytes, cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            plan->h_fring = nullptr;
            destroy_stream_state(plan);
            return fail(plan, NSFRB_ENOMEM, "pinned host FP32 window for re-scoring");
        }
        std::memset(plan->h_fring, 0, fbytes);
        if ((st = cuda_check(plan, cudaHostGetDevicePointer(reinterpret_cast<void **>(&plan->d_fring), plan->h_fring, 0),
                             "host window address"))) {
            destroy_stream_state(plan);
            return st;
        }
    }
    if ((st = cuda_check(plan, cudaMemset(plan->d_ring, 0, ring_bytes), "ring clear")) ||
        (st = cuda_check(plan, cudaMemset(plan->d_sstate, 0, 64), "state clear")) ||
        (st = cuda_check(plan, cudaStreamCreateWithFlags(&plan->s_stream, cudaStreamNonBlocking), "stream")) ||
        (st = cuda_check(plan, cudaEventCreate(&plan->s_ev_push), "event")) ||
        (st = cuda_check(plan, cudaEventCreate(&plan->s_ev_done), "event"))) {
        destroy_stream_state(plan);
        return st;
    }

    // Capture the per-block device work once.
    cudaStream_t s = plan->s_stream;
    cudaGraph_t graph = nullptr;
    if ((st = cuda_check(plan, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture"))) {
        destroy_stream_state(plan);
        return st;
    }
    const dim3 tr_grid(static_cast<unsigned>((n_pix + kTrPix - 1) / kTrPix), c.n_sub);
    const size_t tr_smem = sizeof(float) * n_blk * (kTrPix + 1);
    bool ok = true;
    if (tr_smem > 48 * 1024)
        ok = false;
    else if (c.dtype == NSFRB_F32)
        ingest_kernel<float><<<tr_grid, 256, tr_smem, s>>>(plan->d_blk, static_cast<float *>(plan->d_ring), n_pix,
                                                           c.n_sub, n_blk, c.n_t, plan->ring_len, plan->d_sstate,
                                                           plan->d_mask, nullptr);
    else if (c.dtype == NSFRB_BF16)
        ingest_kernel<__nv_bfloat16><<<tr_grid, 256, tr_smem, s>>>(
            plan->d_blk, static_cast<__nv_bfloat16 *>(plan->d_ring), n_pix, c.n_sub, n_blk, c.n_t, plan->ring_len,
            plan->d_sstate, plan->d_mask, plan->d_fring);
    else
        ingest_kernel<__half><<<tr_grid, 256, tr_smem, s>>>(plan->d_blk, static_cast<__half *>(plan->d_ring), n_pix,
                                                            c.n_sub, n_blk, c.n_t, plan->ring_len, plan->d_sstate,
                                                            plan->d_mask, plan->d_fring);
    advance_kernel<<<1, 1, 0, s>>>(plan->d_sstate, n_blk, c.n_t);
    cudaMemsetAsync(plan->d_err, 0, sizeof(int32_t), s);
    nsfrb_status qs = NSFRB_OK;
    if (ok)
        qs = queue_search(plan, plan->d_ring, 0, c.dtype, plan->ring_len, 0, nullptr, 0, n_pix, nullptr, nullptr,
                          n_blk, s, plan->d_sstate);
    if (ok && qs == NSFRB_OK && rescore) {
        // pixels whose best over the new trials lies within +-rescore_eps of the threshold:
        // the same masked search again on their FP32 window rows (device or host memory)
        qs = cuda_check(plan,
                        launch_rescore_select(plan->d_rec, n_pix, c.threshold, c.rescore_eps, plan->d_list,
                                              plan->d_nlist, s),
                        "re-score select");
        if (qs == NSFRB_OK)
            qs = queue_search(plan, plan->d_fring, 0, NSFRB_F32, c.n_t, 0, nullptr, 0, n_pix, plan->d_list,
                              plan->d_nlist, n_blk, s, plan->d_sstate, c.n_t, n_pix);
    }
    if (ok && qs == NSFRB_OK)
        qs = cuda_check(plan,
                        launch_compact(plan->d_rec, n_pix, c.nx, c.threshold, plan->d_counts, plan->n_blocks,
                                       plan->d_cand, plan->d_ncand, s),
                        "compaction");
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (!ok || qs != NSFRB_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        destroy_stream_state(plan);
        cudaGetLastError();
        if (!ok) return fail(plan, NSFRB_EINVAL, "block too long for the ingest tile");
        return qs != NSFRB_OK ? qs : cuda_check(plan, ce, "end capture");
    }
    ce = cudaGraphInstantiate(&plan->s_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        destroy_stream_state(plan);
        return cuda_check(plan, ce, "graph instantiate");
    }
    plan->n_pushed = 0;
    plan->pending = false;
    return NSFRB_OK;
}

nsfrb_status nsfrb_stream_push(nsfrb_plan_t plan, const float *h_block, uint32_t present_mask) {
    if (!plan || !h_block) return fail(plan, NSFRB_EINVAL, "null argument");
    if (!plan->streaming) return fail(plan, NSFRB_EINVAL, "stream not open");
    if (plan->pending) return fail(plan, NSFRB_ENOTREADY, "previous block not polled");
    const nsfrb_config &c = plan->cfg;
    const size_t bytes = sizeof(float) * plan->n_blk * c.n_sub * static_cast<size_t>(c.ny) * c.nx;
    cudaStream_t s = plan->s_stream;
    nsfrb_status st;
    // pageable source: the copy has consumed the value when cudaMemcpyAsync returns
    const uint32_t m = present_mask;
    if ((st = cuda_check(plan, cudaEventRecord(plan->s_ev_push, s), "event")) ||
        (st = cuda_check(plan, cudaMemcpyAsync(plan->d_blk, h_block, bytes, cudaMemcpyHostToDevice, s), "block copy")) ||
        (st = cuda_check(plan, cudaMemcpyAsync(plan->d_mask, &m, sizeof(m), cudaMemcpyHostToDevice, s), "mask")) ||
        (st = cuda_check(plan, cudaGraphLaunch(plan->s_graph, s), "graph launch")) ||
        (st = cuda_check(plan, cudaEventRecord(plan->s_ev_done, s), "event")))
        return st;
    plan->pending = true;
    ++plan->n_pushed;
    return NSFRB_OK;
}

nsfrb_status nsfrb_stream_block(nsfrb_plan_t plan, float **d_block) {
    if (!plan || !d_block) return fail(plan, NSFRB_EINVAL, "null argument");
    if (!plan->streaming) return fail(plan, NSFRB_EINVAL, "stream not open");
    *d_block = plan->d_blk;
    return NSFRB_OK;
}

nsfrb_status nsfrb_stream_push_device(nsfrb_plan_t plan, uint32_t present_mask, void *stream) {
    if (!plan) return fail(plan, NSFRB_EINVAL, "null argument");
    if (!plan->streaming) return fail(plan, NSFRB_EINVAL, "stream not open");
    if (plan->pending) return fail(plan, NSFRB_ENOTREADY, "previous block not polled");
    cudaStream_t s = plan->s_stream;
    const uint32_t m = present_mask;
    nsfrb_status st;
    // the producer's work on `stream` (the block written into d_blk) comes first
    if ((st = cuda_check(plan, cudaEventRecord(plan->s_ev_push, static_cast<cudaStream_t>(stream)), "event")) ||
        (st = cuda_check(plan, cudaStreamWaitEvent(s, plan->s_ev_push, 0), "wait")) ||
        (st = cuda_check(plan, cudaMemcpyAsync(plan->d_mask, &m, sizeof(m), cudaMemcpyHostToDevice, s), "mask")) ||
        (st = cuda_check(plan, cudaGraphLaunch(plan->s_graph, s), "graph launch")) ||
        (st = cuda_check(plan, cudaEventRecord(plan->s_ev_done, s), "event")))
        return st;
    plan->pending = true;
    ++plan->n_pushed;
    return NSFRB_OK;
}

nsfrb_status nsfrb_stream_poll(nsfrb_plan_t plan, int32_t timeout_ms, nsfrb_candidate *h_out, int32_t cap,
                               int32_t *n_total, float *latency_ms) {
    if (!plan || !n_total || cap < 0 || (cap > 0 && !h_out)) return fail(plan, NSFRB_EINVAL, "bad argument");
    if (!plan->streaming) return fail(plan, NSFRB_EINVAL, "stream not open");
    if (!plan->pending) return fail(plan, NSFRB_ENOTREADY, "no block pending");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaEventQuery(plan->s_ev_done);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_check(plan, q, "event query");
        const auto el = std::chrono::steady_clock::now() - t0;
        if (std::chrono::duration_cast<std::chrono::milliseconds>(el).count() >= timeout_ms)
            return fail(plan, NSFRB_ETIMEOUT, "block not finished within the timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    plan->pending = false;
    nsfrb_status st;
    if (latency_ms &&
        (st = cuda_check(plan, cudaEventElapsedTime(latency_ms, plan->s_ev_push, plan->s_ev_done), "elapsed")))
        return st;
    int32_t hdr[2] = {0, 0};
    if ((st = cuda_check(plan, cudaMemcpy(hdr, plan->d_err, sizeof(hdr), cudaMemcpyDeviceToHost), "copy"))) return st;
    *n_total = hdr[1];
    const int32_t n = std::min(hdr[1], cap);
    if (n > 0 && (st = cuda_check(plan, cudaMemcpy(h_out, plan->d_cand, sizeof(CandRec) * n, cudaMemcpyDeviceToHost),
                                  "copy candidates")))
        return st;
    if (hdr[0] & ERR_WAIT_TIMEOUT) return fail(plan, NSFRB_ETIMEOUT, "a bulk copy into shared memory timed out");
    if (hdr[0] & ERR_ZERO_MAD) return fail(plan, NSFRB_EINVAL, "zero MAD in at least one (pixel, subband) row");
    if (hdr[1] > cap) return fail(plan, NSFRB_ETRUNC, "more candidates than capacity");
    return NSFRB_OK;
}

nsfrb_status nsfrb_stream_blocks(nsfrb_plan_t plan, int64_t *n_blocks) {
    if (!plan || !n_blocks) return fail(plan, NSFRB_EINVAL, "null argument");
    *n_blocks = plan->n_pushed;
    return NSFRB_OK;
}

}  // extern "C"
