// PSF-based candidate clustering of arXiv 2510.18136 Sec. 2.3: among the top
// candidates by S/N, each one in turn is taken as the central lobe of the
// point-spread function; the others inside the PSF mask (the PSF thresholded
// at a percentile, centred on that candidate) are its possible sidelobes; the
// weighted mean S/N of the central and sidelobe candidates scores the
// cluster, and the central candidate of the best cluster is the final one.
// One CTA does everything (the inputs are a candidate list and a small PSF).
#include <cfloat>

#include "plan_internal.h"

namespace nsfrb {
namespace {

constexpr int kClusterThreads = 1024;
constexpr int kMaxPsf = 4096;
constexpr int kMaxTop = 32;

struct ClusterOut {
    CandRec final_cand;
    float weighted_snr;
    int32_t n_top;
    int32_t final_rank;
    uint32_t members;   // bit j: top candidate j is in the final candidate's cluster
};

// larger S/N first; equal S/N: smaller pixel index first
__device__ __forceinline__ bool better(float s1, int64_t p1, float s2, int64_t p2) {
    return s1 > s2 || (s1 == s2 && p1 < p2);
}

__global__ void __launch_bounds__(kClusterThreads) cluster_kernel(const CandRec *__restrict__ cand, int n, int nx,
                                                                 const float *__restrict__ psf, int ph, int pw,
                                                                 float pct, int top_k, int score_mode,
                                                                 CandRec *__restrict__ top,
                                                                 ClusterOut *__restrict__ out) {
    __shared__ float s_sorted[kMaxPsf];
    __shared__ CandRec s_top[kMaxTop];
    __shared__ int s_red_i[kClusterThreads / 32];
    __shared__ float s_thr;
    __shared__ float s_score[kMaxTop];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- top candidates: top_k passes of a block arg-max (excluding the ones taken)
    const int k_top = min(top_k, n);
    for (int r = 0; r < k_top; ++r) {
        float bv = -FLT_MAX;
        int bi = -1;
        for (int i = tid; i < n; i += blockDim.x) {
            bool taken = false;
            for (int q = 0; q < r; ++q)
                if (s_top[q].row == cand[i].row && s_top[q].col == cand[i].col) taken = true;
            if (taken) continue;
            const int64_t pi = static_cast<int64_t>(cand[i].row) * nx + cand[i].col;
            if (bi < 0 || better(cand[i].snr, pi, bv, static_cast<int64_t>(cand[bi].row) * nx + cand[bi].col)) {
                bv = cand[i].snr;
                bi = i;
            }
        }
        // warp then block reduction of (value, index)
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oi >= 0 && (bi < 0 || better(cand[oi].snr, static_cast<int64_t>(cand[oi].row) * nx + cand[oi].col, bv,
                                             static_cast<int64_t>(cand[bi].row) * nx + cand[bi].col))) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) s_red_i[warp] = bi;
        __syncthreads();
        if (tid == 0) {
            int b = -1;
            for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) {
                const int i = s_red_i[w];
                if (i < 0) continue;
                if (b < 0 || better(cand[i].snr, static_cast<int64_t>(cand[i].row) * nx + cand[i].col, cand[b].snr,
                                    static_cast<int64_t>(cand[b].row) * nx + cand[b].col))
                    b = i;
            }
            s_top[r] = cand[b];
        }
        __syncthreads();
    }

    // ---- PSF percentile (linear interpolation between order statistics): bitonic sort
    const int np = ph * pw;
    int m = 1;
    while (m < np) m <<= 1;
    for (int i = tid; i < m; i += blockDim.x) s_sorted[i] = i < np ? psf[i] : FLT_MAX;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < m; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const float a = s_sorted[i], b = s_sorted[l];
                    if ((a > b) == up) {
                        s_sorted[i] = b;
                        s_sorted[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    if (tid == 0) {
        const float pos = pct / 100.0f * static_cast<float>(np - 1);
        const int f = static_cast<int>(floorf(pos));
        const int c = min(f + 1, np - 1);
        s_thr = s_sorted[f] + (s_sorted[c] - s_sorted[f]) * (pos - static_cast<float>(f));
    }
    __syncthreads();

    // ---- cluster score of each top candidate (one thread each)
    const int cy = ph / 2, cx = pw / 2;
    if (tid < k_top) {
        const CandRec ci = s_top[tid];
        float num = 0.0f, den = 0.0f;
        for (int j = 0; j < k_top; ++j) {
            const int dy = s_top[j].row - ci.row, dx = s_top[j].col - ci.col;
            const int y = cy + dy, x = cx + dx;
            if (y < 0 || y >= ph || x < 0 || x >= pw) continue;
            const float v = psf[y * pw + x];
            if (v < s_thr) continue;
            // NSFRB_CLUSTER_PSF_MEAN: PSF-weighted mean, sum v snr / sum v.
            // NSFRB_CLUSTER_LSQ: the members' S/N referred to the central lobe (snr_j / v)
            // with inverse-variance weights v^2, sum v snr / sum v^2.
            num += v * s_top[j].snr;
            den += (score_mode == NSFRB_CLUSTER_LSQ) ? v * v : v;
        }
        s_score[tid] = den > 0.0f ? num / den : -FLT_MAX;
    }
    __syncthreads();
    if (tid == 0) {
        int b = 0;
        for (int i = 1; i < k_top; ++i)
            if (s_score[i] > s_score[b]) b = i;
        ClusterOut o;
        o.n_top = k_top;
        o.final_rank = k_top > 0 ? b : -1;
        o.weighted_snr = k_top > 0 ? s_score[b] : -FLT_MAX;
        o.members = 0u;
        if (k_top > 0) {
            o.final_cand = s_top[b];
            for (int j = 0; j < k_top; ++j) {
                const int y = cy + s_top[j].row - s_top[b].row, x = cx + s_top[j].col - s_top[b].col;
                if (y >= 0 && y < ph && x >= 0 && x < pw && psf[y * pw + x] >= s_thr) o.members |= 1u << j;
            }
        } else {
            o.final_cand = CandRec{-1, -1, -1, -1, -1, -FLT_MAX};
        }
        *out = o;
    }
    for (int i = tid; i < k_top; i += blockDim.x) top[i] = s_top[i];
}

}  // namespace
}  // namespace nsfrb

using namespace nsfrb;

extern "C" nsfrb_status nsfrb_psf_cluster(const nsfrb_candidate *d_cand, int32_t n, int32_t nx, const float *d_psf,
                                          int32_t ph, int32_t pw, float percentile, int32_t top_k,
                                          int32_t score_mode, nsfrb_candidate *d_top, void *d_result,
                                          void *stream) {
    if (n < 0 || (n > 0 && !d_cand) || !d_psf || ph < 1 || pw < 1 || ph * pw > kMaxPsf || top_k < 1 ||
        top_k > kMaxTop || !d_top || !d_result || nx < 1 || !(percentile >= 0.0f && percentile <= 100.0f) ||
        (score_mode != NSFRB_CLUSTER_PSF_MEAN && score_mode != NSFRB_CLUSTER_LSQ))
        return fail(nullptr, NSFRB_EINVAL, "bad argument");
    cluster_kernel<<<1, kClusterThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const CandRec *>(d_cand), n, nx, d_psf, ph, pw, percentile, top_k, score_mode,
        reinterpret_cast<CandRec *>(d_top), static_cast<ClusterOut *>(d_result));
    return cuda_check(nullptr, cudaGetLastError(), "cluster launch");
}
