// nsfrb_search_static: the search of nsfrb_search for callers that cannot
// allocate device memory.  All scratch (the plan's tables, per-pixel best
// records, compaction counters) lives in one file-scope __device__ array of
// fixed size; the caller passes the cube, the noise levels and the output
// buffers.  The paper has no counterpart: this is an interface for hosts
// that run the search where cudaMalloc is not allowed.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "plan_internal.h"

namespace nsfrb {
namespace {

constexpr int64_t kStaticMaxPix = NSFRB_STATIC_MAX_PIX;
constexpr int64_t kStaticTableWords = NSFRB_STATIC_MAX_TABLE_WORDS;
constexpr int kStaticBlocks = static_cast<int>((kStaticMaxPix + kCompactBlock - 1) / kCompactBlock);
constexpr size_t kOffRec = 0;
constexpr size_t kOffTable = kOffRec + sizeof(PixRec) * kStaticMaxPix;
constexpr size_t kOffCounts = kOffTable + sizeof(int32_t) * kStaticTableWords;
constexpr size_t kStaticBytes = kOffCounts + sizeof(int32_t) * (kStaticBlocks + 4);
constexpr int kMaxDevices = 64;

// The scratch itself.  Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

std::mutex g_setup_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};
int g_n_sm[kMaxDevices] = {};
int g_max_smem[kMaxDevices] = {};

__global__ void __launch_bounds__(kCompactBlock) static_count_kernel(const PixRec *rec, int64_t n, float thr,
                                                                    int32_t *counts) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kCompactBlock + threadIdx.x;
    const int flag = (i < n) && (rec[i].snr > thr);
    const int total = __syncthreads_count(flag);
    if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// Candidates in pixel order, written only below the caller's capacity; the
// count (or a negative error code) goes to *n_out.
__global__ void __launch_bounds__(kCompactBlock) static_scatter_kernel(const PixRec *rec, int64_t n, int32_t nx,
                                                                      float thr, const int32_t *counts,
                                                                      int32_t n_blocks, const int32_t *err,
                                                                      CandRec *out, int32_t cap, int32_t *n_out) {
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
    if (flag && pos < cap) {
        const PixRec r = rec[i];
        out[pos] = CandRec{static_cast<int32_t>(i / nx), static_cast<int32_t>(i % nx), r.dm_idx, r.w_idx,
                           r.t_idx, r.snr};
    }
    if (blockIdx.x == n_blocks - 1 && threadIdx.x == 0) {
        int32_t tot = 0;
        for (int w = 0; w < kCompactBlock / 32; ++w) tot += s_warp[w];
        const int32_t e = *err;
        *n_out = (e & ERR_ZERO_MAD) ? -1 : (e & ERR_WAIT_TIMEOUT) ? -2 : s_off + tot;
    }
}

// Staging scheme for a contiguous cube under this device's shared-memory limit, as nsfrb_search
// chooses it: the barrier-free kernel for cubes with known noise whose rows are 16-byte aligned
// (FP32 rows copied as they are, 16-bit rows read in place), else bulk copies with per-pixel
// barriers, else plain loads.
bool static_stage(int C, int max_smem, SearchParams &sp, size_t &smem) { return choose_stage_for(C, max_smem, sp, smem); }

// Once per device, with that device current: the device address of the
// scratch array (its host-side name is only a stand-in) and the kernel's
// shared-memory limit.
nsfrb_status static_setup(nsfrb_plan_s *pl, int dev, unsigned char **addr, int *n_sm, int *max_smem) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (dev < 0 || dev >= kMaxDevices) return fail(pl, NSFRB_EINVAL, "device index out of range");
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        nsfrb_status st = cuda_check(pl, cudaGetSymbolAddress(&p, g_scratch), "cudaGetSymbolAddress");
        if (st != NSFRB_OK) return st;
        if ((st = cuda_check(pl, cudaDeviceGetAttribute(&g_n_sm[dev], cudaDevAttrMultiProcessorCount, dev),
                             "sm count")) != NSFRB_OK)
            return st;
        if ((st = cuda_check(pl,
                             cudaDeviceGetAttribute(&g_max_smem[dev], cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
                             "smem limit")) != NSFRB_OK)
            return st;
        if ((st = cuda_check(pl, prepare_search(pl->C, g_max_smem[dev]), "smem attribute")) != NSFRB_OK) return st;
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    } else {
        // the shared-memory attribute is per kernel: make sure this plan's kernel has it
        nsfrb_status st = cuda_check(pl, prepare_search(pl->C, g_max_smem[dev]), "smem attribute");
        if (st != NSFRB_OK) return st;
    }
    *addr = g_scratch_addr[dev];
    *n_sm = g_n_sm[dev];
    *max_smem = g_max_smem[dev];
    return NSFRB_OK;
}

}  // namespace
}  // namespace nsfrb

using namespace nsfrb;

extern "C" nsfrb_status nsfrb_search_static(nsfrb_plan_t plan, const void *d_cube, const float *d_sigma,
                                            nsfrb_candidate *d_out, int32_t cap, int32_t *d_n_total,
                                            void *stream) {
    if (!plan || !d_cube || !d_n_total || cap < 0 || (cap > 0 && !d_out))
        return fail(plan, NSFRB_EINVAL, "null argument");
    const nsfrb_config &c = plan->cfg;
    const int64_t n_pix = static_cast<int64_t>(c.ny) * c.nx;
    if (n_pix > kStaticMaxPix) return fail(plan, NSFRB_EINVAL, "image larger than NSFRB_STATIC_MAX_PIX pixels");
    if (static_cast<int64_t>(plan->table.size()) > kStaticTableWords)
        return fail(plan, NSFRB_EINVAL, "delay tables larger than NSFRB_STATIC_MAX_TABLE_WORDS");
    if (c.out_mode != NSFRB_OUT_CANDIDATES) return fail(plan, NSFRB_EINVAL, "candidate output mode only");
    if (c.noise_mode == NSFRB_NOISE_MAD && d_sigma) return fail(plan, NSFRB_EINVAL, "d_sigma must be NULL in MAD mode");
    if (c.noise_mode == NSFRB_NOISE_MAD && plan->C == kLongC)
        return fail(plan, NSFRB_EINVAL, "MAD normalisation of windows over 1247 samples needs nsfrb_search's workspace");
    if (plan->latched != NSFRB_OK) return fail(plan, plan->latched, "plan has a latched CUDA error");

    int dev = 0;
    nsfrb_status st = cuda_check(plan, cudaGetDevice(&dev), "cudaGetDevice");
    if (st != NSFRB_OK) return st;
    unsigned char *base = nullptr;
    int n_sm = 0, max_smem = 0;
    if ((st = static_setup(plan, dev, &base, &n_sm, &max_smem)) != NSFRB_OK) return st;
    PixRec *rec = reinterpret_cast<PixRec *>(base + kOffRec);
    int32_t *table = reinterpret_cast<int32_t *>(base + kOffTable);
    int32_t *counts = reinterpret_cast<int32_t *>(base + kOffCounts);
    int32_t *err = counts + kStaticBlocks;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int32_t n_blocks = static_cast<int32_t>((n_pix + kCompactBlock - 1) / kCompactBlock);

    // the array keeps the previous call's contents: load this plan's tables, clear the counters
    if ((st = cuda_check(plan,
                         cudaMemcpyAsync(table, plan->table.data(), plan->table.size() * sizeof(int32_t),
                                         cudaMemcpyHostToDevice, s),
                         "table copy")) != NSFRB_OK)
        return st;
    if ((st = cuda_check(plan, cudaMemsetAsync(counts, 0, sizeof(int32_t) * (kStaticBlocks + 4), s), "memset")))
        return st;

    SearchParams sp;
    base_params(plan, sp);
    sp.table = table;
    sp.rec = rec;
    sp.err = err;
    sp.full_snr = nullptr;
    sp.full_t = nullptr;
    sp.cube = d_cube;
    sp.cube_pix0 = 0;
    sp.dtype = c.dtype;
    sp.row_len = c.n_t;
    sp.t_off = 0;
    sp.t_off_dev = nullptr;
    sp.sigma = d_sigma;
    sp.pix0 = 0;
    sp.n_items = n_pix;
    sp.pix_list = nullptr;
    sp.n_items_dev = nullptr;
    sp.new_blk = 0;
    size_t smem = 0;
    if (!static_stage(plan->C, max_smem, sp, smem))
        return fail(plan, NSFRB_EINVAL, "shared memory does not fit this plan");
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(n_pix, n_sm)));
    if ((st = cuda_check(plan, launch_search(plan->C, sp, grid, smem, s), "search launch")) != NSFRB_OK) return st;
    static_count_kernel<<<n_blocks, kCompactBlock, 0, s>>>(rec, n_pix, c.threshold, counts);
    if ((st = cuda_check(plan, cudaGetLastError(), "count launch")) != NSFRB_OK) return st;
    static_scatter_kernel<<<n_blocks, kCompactBlock, 0, s>>>(rec, n_pix, c.nx, c.threshold, counts, n_blocks, err,
                                                             reinterpret_cast<CandRec *>(d_out), cap, d_n_total);
    return cuda_check(plan, cudaGetLastError(), "scatter launch");
}
