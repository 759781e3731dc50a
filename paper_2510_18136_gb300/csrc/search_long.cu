// The search of arXiv 2510.18136 Sec. 2.2 for windows longer than the register path holds
// (kMaxTRegs + 1 .. kMaxT samples): per pixel and distinct DM row, the de-dispersed series
// D[t] = sum_k x_k(t + s_k), its prefix P, every width's boxcars P[t + w] - P[t] normalised by
// 1 / (sigma sqrt(w)), and the maximum over time, width and DM with the same tie rules as the
// other kernels (smallest DM row, then width index, then sample).
//
// Organisation (one CTA per pixel at a time, persistent over pixels):
//  * A pixel's FP32 rows of a long window (up to 256 KB) do not fit in shared memory, so the
//    de-dispersion reads the cube where it lies (HBM, through L1/L2) in a sample-interleaved
//    lane layout: lane j of a warp takes samples t = 32 i + j, so every subband read of a step i
//    is one coalesced 128-byte line per warp; the CTA's warps work on rows of the same pixel at
//    the same time and share its lines in L1.
//  * The prefix of a step is a warp inclusive scan of the 32 de-dispersed samples plus the
//    running total, kept as a compensated pair P = hi + lo: hi the FP32 sum, lo its exact
//    rounding error (two-sum) carried along, stored in FP16.  A boxcar is then
//    (hi[t + w] - hi[t]) + (lo[t + w] - lo[t]), whose error is relative to the boxcar itself
//    rather than to the prefix: over 4096 samples, and after bright wide pulses, an FP32 prefix
//    difference alone loses about one unit of the prefix's last place, more than the 1e-5
//    relative S/N the search keeps.  Both rows go to the warp's shared memory (consecutive lanes,
//    consecutive words).
//  * Every width is then evaluated from P in shared memory (lane-strided trials), the warp's
//    arg-max over widths taken, and the earliest sample reaching it found by re-evaluating the
//    same operations.
//  * Each warp takes a contiguous group of the pixel's distinct DM rows.  It builds the group's
//    first row from every subband (all loads of a step issued before the sum) and each next row
//    from the previous one by adding and subtracting only the subbands whose shift changed, with
//    the previous row's D[t] = P[t + 1] - P[t] read back from its compensated prefix (exact to
//    the rounding of D itself).  The CTA combines the warps' bests by (S/N, row) and writes the
//    record (and, in FULL mode, every (DM, width) result).
// Samples read past the window never enter a valid trial: a trial of row u ends before
// L_u = n_t - smax_u, and D[t] for t >= L_u is not computed.
#include <climits>

#include <cuda_fp16.h>

#include "nsfrb.h"
#include "nsfrb_internal.h"
#include "plan_internal.h"
#include "search_impl.cuh"

namespace nsfrb {
namespace dev {

__host__ __device__ inline int long_ppitch(int n_t) { return static_cast<int>(align_up(static_cast<size_t>(n_t) + 33, 4)); }

// Shared memory: tables | P rows, hi [n_warps][ppitch] FP32 and lo [n_warps][ppitch] FP16 | warp
// bests | 1 / (sigma sqrt(w)).
struct LongLayout {
    size_t table, pbuf, plo, wbest, sinv, total;
};

__host__ __device__ inline LongLayout long_layout(const SearchParams &p, int n_warps) {
    LongLayout L{};
    size_t o = 0;
    L.table = o;
    o += align_up(sizeof(int32_t) * ((size_t)p.n_u * kInfo + p.n_deltas + (size_t)p.n_u * p.n_sub), 16);
    L.pbuf = o;
    o += sizeof(float) * (size_t)n_warps * long_ppitch(p.n_t);
    L.plo = o;
    o += align_up(sizeof(__half) * (size_t)n_warps * long_ppitch(p.n_t), 16);
    L.wbest = o;
    o += sizeof(PixRec) * (size_t)n_warps;
    L.sinv = o;
    o += sizeof(float) * kMaxW;
    L.total = align_up(o, 16);
    return L;
}

// Element (pixel pix, subband k, window sample t) of the cube in any of the search's layouts
// (ring rows that wrap, sample-major windows; used by the re-score of a few pixels).
__device__ __forceinline__ float long_x_any(const SearchParams &p, int64_t pix, int k, int t, int t_off) {
    int tt = t_off + t;
    if (p.t_wrap > 0 && tt >= p.t_wrap) tt -= p.t_wrap;
    const int64_t at = p.t_stride > 0 ? (static_cast<int64_t>(tt) * p.n_sub + k) * p.t_stride + pix
                                      : ((pix - p.cube_pix0) * p.n_sub + k) * p.row_len + tt;
    return load_elem(p.cube, at, p.dtype);
}

// Element i of a pixel-major pixel tile stored as ST (0 FP32, 1 BF16, 2 FP16), widened exactly.
template <int ST>
__device__ __forceinline__ float tile_x(const void *tile, int i) {
    if constexpr (ST == 0) {
        return static_cast<const float *>(tile)[i];
    } else {
        const unsigned short u = static_cast<const unsigned short *>(tile)[i];
        if constexpr (ST == 1) return __uint_as_float(static_cast<uint32_t>(u) << 16);
        return __half2float(__ushort_as_half(u));
    }
}

// Boxcar P[a] - P[b] of the compensated prefix (hi, lo).
__device__ __forceinline__ float pdiff(const float *H, const __half *Lo, int a, int b) {
    return (H[a] - H[b]) + (__half2float(Lo[a]) - __half2float(Lo[b]));
}

// Width w from the compensated prefix: the maximum over trials t in [t_lo, L - w] (lane-strided),
// and the earliest t whose boxcar times inv equals target (the same operations).
__device__ __forceinline__ float long_max(const float *H, const __half *Lo, int w, int L, int t_lo, int lane) {
    float m = neg_inf();
    for (int t = t_lo + lane; t + w <= L; t += 32) m = fmaxf(m, pdiff(H, Lo, t + w, t));
    return m;
}
__device__ __forceinline__ int long_find(const float *H, const __half *Lo, int w, int L, int t_lo, int lane,
                                         float inv, float target) {
    for (int t = t_lo + lane; t + w <= L; t += 32)
        if (pdiff(H, Lo, t + w, t) * inv == target) return t;
    return INT_MAX;
}

// ST >= 0: a pixel-major cube of rows without wrap in storage ST; ST < 0: any layout (plain loads).
template <int ST, bool FULL>
__global__ void __launch_bounds__(kThreads, 1) search_kernel_long(const __grid_constant__ SearchParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int n_warps = blockDim.x >> 5;
    const LongLayout lay = long_layout(p, n_warps);
    int32_t *s_table = reinterpret_cast<int32_t *>(smem + lay.table);
    float *s_pbuf = reinterpret_cast<float *>(smem + lay.pbuf);
    PixRec *s_wbest = reinterpret_cast<PixRec *>(smem + lay.wbest);
    float *s_inv = reinterpret_cast<float *>(smem + lay.sinv);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_sub = p.n_sub, n_t = p.n_t;
    const int t_off = p.t_off_dev ? *p.t_off_dev : p.t_off;
    const int table_words = p.n_u * kInfo + p.n_deltas + p.n_u * n_sub;
    for (int i = tid; i < table_words; i += blockDim.x) s_table[i] = p.table[i];
    const int32_t *s_info = s_table;
    const int32_t *s_shift = s_table + p.n_u * kInfo + p.n_deltas;
    float *Pw = s_pbuf + (size_t)warp * long_ppitch(n_t);
    __half *Plo = reinterpret_cast<__half *>(smem + lay.plo) + (size_t)warp * long_ppitch(n_t);
    constexpr size_t es = (ST == 0) ? 4 : 2;   // bytes per stored sample (pixel-major layouts)
    if (lane == 0) {
        Pw[0] = 0.0f;
        Plo[0] = __float2half_rn(0.0f);
    }
    __syncthreads();

    int64_t n_items = p.n_items;
    if (p.n_items_dev) n_items = *p.n_items_dev;
    const int n_ua = p.n_u_active;
    const bool masked = p.new_blk > 0;

    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int64_t pix = p.pix_list ? static_cast<int64_t>(p.pix_list[it]) : p.pix0 + it;
        if (tid < p.n_w) {
            const float sg = (p.sigma && p.noise_mode == 0) ? p.sigma[pix] : p.sigma_default;
            s_inv[tid] = 1.0f / (sg * sqrtf(static_cast<float>(p.widths[tid])));
        }
        const bool bad = p.bad_pix && p.bad_pix[pix];
        // the pixel's tile (pixel-major layouts): subband k, window sample t at element
        // k row_len + t_off + t
        const void *tile = nullptr;
        if constexpr (ST >= 0)
            tile = static_cast<const unsigned char *>(p.cube) +
                   static_cast<size_t>(pix - p.cube_pix0) * n_sub * p.row_len * es;
        __syncthreads();

        float bsnr = neg_inf();
        int bu = -1, bwi = -1, bt = -1;
        // the warp's rows: a contiguous group [u_lo, u_hi); its first row is built from every
        // subband, each next row from the previous one by the subbands whose shift changed
        const int u_lo = (warp * n_ua) / n_warps, u_hi = ((warp + 1) * n_ua) / n_warps;
        const int32_t *s_delta = s_table + p.n_u * kInfo;
        const int32_t rl = static_cast<int32_t>(p.row_len);
        // sample tt of subband k of the pixel (tt < n_t)
        auto xat = [&](int k, int tt) -> float {
            if constexpr (ST >= 0)
                return tile_x<ST>(tile, k * rl + t_off + tt);
            else
                return long_x_any(p, pix, k, tt, t_off);
        };
#pragma unroll 1
        for (int u = bad ? u_hi : u_lo; u < u_hi; ++u) {
            const int32_t *sh = s_shift + u * n_sub;
            const int32_t *info = s_info + u * kInfo;
            const int L = n_t - info[UI_SMAX];
            const bool first = u == u_lo;
            const int d0 = info[UI_DOFF], nd = info[UI_ND];
            // de-dispersion and compensated prefix, 32 samples per step.  A next row reads the
            // previous row's D[t] = P[t + 1] - P[t] from the compensated prefix it overwrites:
            // each lane reads the old pair at t + 1, takes the one at t from the lane below (lane 0
            // from lane 31 of the step before), and writes the new pair at t + 1 afterwards.
            float run = 0.0f, run_lo = 0.0f;
            float ph_prev = 0.0f, pl_prev = 0.0f;   // old pair at the step's first index
            // the first two changed subbands of a next row (k, old and new shift), decoded once
            int dk[2] = {0, 0}, dso[2] = {0, 0}, dsn[2] = {0, 0};
#pragma unroll
            for (int j = 0; j < 2; ++j)
                if (!first && j < nd) {
                    const uint32_t pk = static_cast<uint32_t>(s_delta[d0 + j]);
                    dk[j] = pk & 63u;
                    dso[j] = (pk >> 6) & 0x1fffu;
                    dsn[j] = pk >> 19;
                }
            // the global loads of a step, issued one step ahead of its sum: a first row's first 16
            // subbands, a next row's first two changed subbands (new and old sample)
            float xa[16];
            auto fetch = [&](int tt) {
#pragma unroll
                for (int j = 0; j < 16; ++j) xa[j] = 0.0f;
                if (tt < L) {
                    if (first) {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (j < n_sub) xa[j] = xat(j, tt + sh[j]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 2; ++j)
                            if (j < nd) {
                                xa[2 * j] = xat(dk[j], tt + dsn[j]);
                                xa[2 * j + 1] = xat(dk[j], tt + dso[j]);
                            }
                    }
                }
            };
            fetch(lane);
#pragma unroll 1
            for (int t0 = 0; t0 < L; t0 += 32) {
                const int t = t0 + lane;
                float xc[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) xc[j] = xa[j];
                fetch(t + 32);
                float d = 0.0f;
                if (first) {
                    if (t < L) {
                        // subbands in order: the fetched 16, then any beyond
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (j < n_sub) d += xc[j];
#pragma unroll 1
                        for (int k = 16; k < n_sub; ++k) d += xat(k, t + sh[k]);
                    }
                } else {
                    const float oh = Pw[t + 1], ol = __half2float(Plo[t + 1]);
                    float ph = __shfl_up_sync(kFull, oh, 1), pl = __shfl_up_sync(kFull, ol, 1);
                    if (lane == 0) {
                        ph = ph_prev;
                        pl = pl_prev;
                    }
                    ph_prev = __shfl_sync(kFull, oh, 31);
                    pl_prev = __shfl_sync(kFull, ol, 31);
                    d = (oh - ph) + (ol - pl);
                    if (t < L) {
#pragma unroll
                        for (int j = 0; j < 2; ++j)
                            if (j < nd) d = (d + xc[2 * j]) - xc[2 * j + 1];
#pragma unroll 1
                        for (int e = 2; e < nd; ++e) {
                            const uint32_t pk = static_cast<uint32_t>(s_delta[d0 + e]);
                            const int k = pk & 63u, so = (pk >> 6) & 0x1fffu, sn = pk >> 19;
                            d = (d + xat(k, t + sn)) - xat(k, t + so);
                        }
                    } else {
                        d = 0.0f;
                    }
                }
                float v = d;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float y = __shfl_up_sync(kFull, v, o);
                    if (lane >= o) v += y;
                }
                // hi = run + v rounded, e its exact error (two-sum), lo = run_lo + e
                const float hi = run + v;
                const float bb = hi - run;
                const float e = (run - (hi - bb)) + (v - bb);
                const float lo = run_lo + e;
                Pw[t + 1] = hi;
                Plo[t + 1] = __float2half_rn(lo);
                // the next step's running pair from lane 31, renormalised (|lo| <= half an ulp of hi)
                const float h31 = __shfl_sync(kFull, hi, 31), l31 = __shfl_sync(kFull, lo, 31);
                run = h31 + l31;
                run_lo = l31 - (run - h31);
            }
            __syncwarp();   // P of the row (and the offsets' reads) complete
            // every width from P: trials t in [t_lo, L - w]; ascending width order with a strict
            // '>' keeps the smallest width index on ties
            float ls = neg_inf();
            int lw = -1;
#pragma unroll 1
            for (int wi = 0; wi < p.n_w; ++wi) {
                const int w = p.widths[wi];
                const int tl = masked ? max(0, L - w - p.new_blk + 1) : 0;
                const float m = long_max(Pw, Plo, w, L, tl, lane);
                const float s = m * s_inv[wi];
                if (s > ls) {
                    ls = s;
                    lw = wi;
                }
                if constexpr (FULL) {
                    const float mw = warp_max(m), sw = mw * s_inv[wi];
                    int tf = INT_MAX;
                    if (mw != neg_inf()) tf = warp_min(long_find(Pw, Plo, w, L, tl, lane, s_inv[wi], sw));
                    if (lane == 0) {
                        const int fd = info[UI_FIRST_D], ndm = info[UI_N_D];
                        for (int dd = fd; dd < fd + ndm; ++dd) {
                            const int64_t o = (pix * p.n_dm + dd) * p.n_w + wi;
                            p.full_snr[o] = sw;
                            p.full_t[o] = static_cast<int16_t>(tf == INT_MAX ? -1 : tf);
                        }
                    }
                }
            }
            // warp arg-max over (S/N, width index), only when some lane beats the warp's best
            if (__any_sync(kFull, ls > bsnr)) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float os = __shfl_xor_sync(kFull, ls, o);
                    const int ow = __shfl_xor_sync(kFull, lw, o);
                    if (os > ls || (os == ls && ow < lw && ow >= 0)) {
                        ls = os;
                        lw = ow;
                    }
                }
                if (ls > bsnr) {
                    const int w = p.widths[lw];
                    const int tl = masked ? max(0, L - w - p.new_blk + 1) : 0;
                    bt = warp_min(long_find(Pw, Plo, w, L, tl, lane, s_inv[lw], ls));
                    bsnr = ls;
                    bu = u;
                    bwi = lw;
                }
            }
            __syncwarp();
        }
        // FULL mode: DM rows without any trial (all of them for a flagged pixel)
        if constexpr (FULL) {
            if (warp == 0) {
                for (int u = bad ? 0 : n_ua; u < p.n_u; ++u) {
                    const int32_t *info = s_info + u * kInfo;
                    const int fd = info[UI_FIRST_D], ndm = info[UI_N_D];
                    for (int i = lane; i < ndm * p.n_w; i += 32) {
                        const int64_t o = (pix * p.n_dm + fd) * p.n_w + i;
                        p.full_snr[o] = neg_inf();
                        p.full_t[o] = -1;
                    }
                }
            }
        }
        if (lane == 0) s_wbest[warp] = PixRec{bsnr, bu, bwi, bt};
        __syncthreads();
        if (tid == 0) {
            // warps hold rows w, w + n_warps, ...: ties of S/N go to the smaller row
            PixRec best{neg_inf(), -1, -1, -1};
            for (int w = 0; w < n_warps; ++w) {
                const PixRec r = s_wbest[w];
                if (r.snr > best.snr || (r.snr == best.snr && r.dm_idx >= 0 && (best.dm_idx < 0 || r.dm_idx < best.dm_idx)))
                    best = r;
            }
            if (best.dm_idx >= 0) best.dm_idx = s_info[best.dm_idx * kInfo + UI_FIRST_D];
            if (bad) {
                best = PixRec{neg_inf(), -1, -1, -1};
                atomicOr(p.err, ERR_ZERO_MAD);
            }
            p.rec[pix] = best;
        }
        __syncthreads();
    }
}

}  // namespace dev

// Warps per CTA of the long-window kernel.  The CTA waits for its slowest warp at every pixel, so
// of the counts whose prefix rows fit, the one that completes the most DM rows per round
// (n_rows / ceil(n_rows / warps)), the fewest warps on ties.
int long_warps(const SearchParams &p, int max_smem) {
    int fit = 0;
    for (int w = kWarps; w >= 1 && fit == 0; --w)
        if (dev::long_layout(p, w).total <= static_cast<size_t>(max_smem)) fit = w;
    if (fit == 0) return 0;
    const int n = p.n_u_active > 0 ? p.n_u_active : 1;
    int best = 1;
    double best_rate = 0.0;
    for (int w = 1; w <= fit; ++w) {
        const double rate = static_cast<double>(n) / ((n + w - 1) / w);
        if (rate > best_rate + 1e-9) {
            best_rate = rate;
            best = w;
        }
    }
    return best;
}

size_t long_smem(const SearchParams &p, int n_warps) { return dev::long_layout(p, n_warps).total; }

#define NSFRB_LONG_LAUNCH(ST)                                                                  \
    if (p.full_snr)                                                                            \
        dev::search_kernel_long<ST, true><<<grid, threads, smem, s>>>(p);                      \
    else                                                                                       \
        dev::search_kernel_long<ST, false><<<grid, threads, smem, s>>>(p);

cudaError_t launch_search_long(const SearchParams &p, int grid, size_t smem, cudaStream_t s) {
    const int n_warps = p.teams;   // the CTA's warp count for this kernel (long_warps)
    if (n_warps < 1 || n_warps > kWarps) return cudaErrorInvalidValue;
    const unsigned threads = 32u * static_cast<unsigned>(n_warps);
    if (p.t_wrap != 0 || p.t_stride != 0) {
        NSFRB_LONG_LAUNCH(-1)
    } else if (p.dtype == NSFRB_F32) {
        NSFRB_LONG_LAUNCH(0)
    } else if (p.dtype == NSFRB_BF16) {
        NSFRB_LONG_LAUNCH(1)
    } else {
        NSFRB_LONG_LAUNCH(2)
    }
    return cudaGetLastError();
}

#define NSFRB_LONG_ATTR(ST, F)                                                                 \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(dev::search_kernel_long<ST, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);

cudaError_t prepare_search_long(size_t smem) {
    const int sm = static_cast<int>(smem);
    cudaError_t e = cudaSuccess;
    NSFRB_LONG_ATTR(-1, false)
    NSFRB_LONG_ATTR(-1, true)
    NSFRB_LONG_ATTR(0, false)
    NSFRB_LONG_ATTR(0, true)
    NSFRB_LONG_ATTR(1, false)
    NSFRB_LONG_ATTR(1, true)
    NSFRB_LONG_ATTR(2, false)
    NSFRB_LONG_ATTR(2, true)
    return e;
}

}  // namespace nsfrb
