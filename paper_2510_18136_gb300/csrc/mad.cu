// Robust noise normalisation of arXiv 2510.18136 Sec. 2.2 (each pixel's median removed and the
// samples scaled by a running noise estimate; read here as the per (pixel, subband) median and
// 1.4826 MAD over the window) as a pass of its own ahead of the search: every (pixel, subband) row
// of a slab of pixels is normalised once, x <- (x - median) / (1.4826 MAD), into an FP32 slab that
// the barrier-free search then reads like any FP32 cube with unit noise per sample.
//
// One warp per row.  The row is copied once to the warp's shared-memory buffer as stored (FP32 or
// 16-bit, by 16-byte loads where the rows allow; its mean and standard deviation s are summed on the
// way) and every pass then reads it as sample pairs in short rolled loops without branches.  The
// median and the MAD are exact order statistics of the row (the same values the search kernel's
// in-place MAD path selects, so the normalised rows are bit-identical to the ones it forms), found
// by histogram levels over a bracket of values that holds the wanted rank(s).  A level bins the
// bracket into 256 bins by a monotone map (linear in value; linear in the order-preserving integer
// key after a value level that failed to halve the bracket's count, which bounds the levels for any
// dynamic range); the bin of the rank becomes the next bracket, its ends set to its own smallest and
// largest value (runs of ties end the search at once).  The first level spans mean +- 3 s for the
// samples and [0, 3 s] for the deviations |x - median|, values outside clamped into the end bins:
// the median lies within s of the mean and the MAD is at most (1 + sqrt 2) s for any sample
// (Chebyshev), so for noise rows the rank's bin holds a few values and the search ends after one
// level with the at most 32 values of the rank's bin(s) gathered and ranked directly.  Signed zeros
// compare equal (the chosen zero's sign changes no normalised value).
// A zero MAD marks the pixel invalid (bad[pixel] = 1, its rows are written as zeros).
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "nsfrb.h"
#include "search_impl.cuh"

namespace nsfrb {
namespace {

constexpr int kMadWarps = 8;
constexpr int kBins = 256;                    // bins of a level; bin kBins takes the values outside
constexpr int kCap = 8;                       // values one lane gathers directly
constexpr int kColPitch = kCap + 1;           // words between lanes' gather columns (no bank conflicts)
constexpr int kMaxLevels = 32;                // bound on the histogram levels of one selection

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(dev::kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(dev::kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(dev::kFull, v, o));
    return v;
}

// Sample pair p (samples 2p, 2p + 1) of a row buffer in storage type ST, widened to FP32.
template <int ST>
__device__ __forceinline__ float2 row_pair(const void *row, int p) {
    if constexpr (ST == 0) {
        return reinterpret_cast<const float2 *>(row)[p];
    } else {
        const uint32_t u = reinterpret_cast<const uint32_t *>(row)[p];
        if constexpr (ST == 1) return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
        return __half22float2(*reinterpret_cast<const __half2 *>(&u));
    }
}

// The bin map of one level.  Value bins: floor(max(x - lo, 0) * scale) from one FMA rounded toward
// zero onto the integers of [2^23, 2^24) (no conversion instruction), clamped to the last bin.  Key
// bins: the offset of x's key from klo, converted and scaled (keys below klo in bin 0).  Both are
// monotone non-decreasing in x.
// With `check` (levels past the first) only values in [lo, hi] have a bin; the others, and a missing
// second sample of an odd row, go to the spare bin kBins.
struct BinMap {
    float lo, hi, scale;
    uint32_t klo;
    bool key, check;
    template <bool KEY, bool CHECK>
    __device__ __forceinline__ int of(float x, bool valid) const {
        int q;
        if constexpr (!KEY) {
            q = min(kBins - 1, __float_as_int(__fmaf_rz(fmaxf(x - lo, 0.0f), scale, 8388608.0f)) - 0x4b000000);
        } else {
            const uint32_t k = dev::f2key(x);
            q = k < klo ? 0 : min(kBins - 1, __float2int_rz(__uint2float_rz(k - klo) * scale));
        }
        bool in = valid;
        if constexpr (CHECK) in = in && x >= lo && x <= hi;
        return in ? q : kBins;
    }
};

// Bins b_r, b_w that hold ranks tr <= tw of a histogram (lane l holds bins 8 l .. 8 l + 7), the
// number of values before b_r, and the number in bins b_r .. b_w.  False if a rank is beyond the
// histogram's count.
__device__ __forceinline__ bool find_bins(const uint32_t *hist, uint32_t tr, uint32_t tw, int &br, int &bw,
                                          uint32_t &before_r, uint32_t &in_range) {
    const int lane = threadIdx.x & 31;
    const uint4 h0 = reinterpret_cast<const uint4 *>(hist)[2 * lane];
    const uint4 h1 = reinterpret_cast<const uint4 *>(hist)[2 * lane + 1];
    const uint32_t c[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) sum += c[j];
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(dev::kFull, incl, o);
        if (lane >= o) incl += y;
    }
    int lr = -1, lw = -1;
    uint32_t br_before = 0, bw_end = 0, acc = incl - sum;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (tr >= acc && tr < acc + c[j]) {
            lr = 8 * lane + j;
            br_before = acc;
        }
        if (tw >= acc && tw < acc + c[j]) {
            lw = 8 * lane + j;
            bw_end = acc + c[j];
        }
        acc += c[j];
    }
    const unsigned has_r = __ballot_sync(dev::kFull, lr >= 0), has_w = __ballot_sync(dev::kFull, lw >= 0);
    if (has_r == 0u || has_w == 0u) return false;
    const int sr = __ffs(has_r) - 1, sw = __ffs(has_w) - 1;
    br = __shfl_sync(dev::kFull, lr, sr);
    before_r = __shfl_sync(dev::kFull, br_before, sr);
    bw = __shfl_sync(dev::kFull, lw, sw);
    in_range = __shfl_sync(dev::kFull, bw_end, sw) - before_r;
    return true;
}

// The values of row view V (pairs of FP32 values) and the warp's shared scratch.
struct Scratch {
    uint32_t *hist;   // [kBins + 1]
    float *cols;      // [32][kColPitch]: each lane's directly gathered values
    float *list;      // [32]: the gathered values in order
};

// One level over the bracket of bin map bm: the histogram, then either the at most 32 values of the
// bins of ranks tr, tr + w gathered and ranked (returns 1 with a, b set), or the ends of the rank's
// bin and the smallest value of rank tr + w's bin (returns 0).  -1: counts inconsistent with n.
template <bool KEY, bool CHECK, typename View>
__device__ __forceinline__ int run_level(const View vw, const BinMap bm, int n_pairs, int last_full, int tr, int w,
                                      const Scratch sc, int &br, int &bw, uint32_t &before_r, uint32_t &m,
                                      float &bmn, float &bmx, float &wmn, float &a, float &b) {
    const int lane = threadIdx.x & 31;
    const float kInf = __int_as_float(0x7f800000);
    // histogram: every value counted, those outside the bracket into the spare bin
#pragma unroll
    for (int j = 0; j < kBins / 32; ++j) sc.hist[32 * j + lane] = 0u;
    if (lane == 0) sc.hist[kBins] = 0u;
    __syncwarp();
#pragma unroll 2
    for (int p = lane; p < n_pairs; p += 32) {
        const float2 x = vw.get(p);
        atomicAdd(&sc.hist[bm.template of<KEY, CHECK>(x.x, true)], 1u);
        atomicAdd(&sc.hist[bm.template of<KEY, CHECK>(x.y, p < last_full)], 1u);
    }
    __syncwarp();
    if (!find_bins(sc.hist, static_cast<uint32_t>(tr), static_cast<uint32_t>(tr + w), br, bw, before_r, m)) return -1;
    const uint32_t span_b = static_cast<uint32_t>(bw - br);
    const int qa = tr - static_cast<int>(before_r);
    if (m <= 32) {
        // the bins of both ranks: each lane keeps its values in its own column, then the columns are
        // packed in lane order and the values ranked (ties broken by position)
        float *col = sc.cols + lane * kColPitch;
        int k = 0;
#pragma unroll 2
        for (int p = lane; p < n_pairs; p += 32) {
            const float2 x = vw.get(p);
            const bool i0 = static_cast<uint32_t>(bm.template of<KEY, CHECK>(x.x, true) - br) <= span_b;
            const bool i1 = static_cast<uint32_t>(bm.template of<KEY, CHECK>(x.y, p < last_full) - br) <= span_b;
            if (i0 && k < kCap) col[k] = x.x;
            k += i0;
            if (i1 && k < kCap) col[k] = x.y;
            k += i1;
        }
        if (__any_sync(dev::kFull, k > kCap)) {
            // a lane met more than kCap: gather again with positions from ballots
            int base = 0;
            const unsigned below = (1u << lane) - 1u;
            for (int p0 = 0; p0 < n_pairs; p0 += 32) {
                const int p = p0 + lane;
                float2 x = make_float2(0.0f, 0.0f);
                bool i0 = false, i1 = false;
                if (p < n_pairs) {
                    x = vw.get(p);
                    i0 = static_cast<uint32_t>(bm.template of<KEY, CHECK>(x.x, true) - br) <= span_b;
                    i1 = static_cast<uint32_t>(bm.template of<KEY, CHECK>(x.y, p < last_full) - br) <= span_b;
                }
                const unsigned b0 = __ballot_sync(dev::kFull, i0);
                if (i0) sc.list[base + __popc(b0 & below)] = x.x;
                base += __popc(b0);
                const unsigned b1 = __ballot_sync(dev::kFull, i1);
                if (i1) sc.list[base + __popc(b1 & below)] = x.y;
                base += __popc(b1);
            }
        } else {
            int excl = k;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(dev::kFull, excl, o);
                if (lane >= o) excl += y;
            }
            excl -= k;
            for (int j = 0; j < k; ++j) sc.list[excl + j] = col[j];
        }
        __syncwarp();
        const int mm = static_cast<int>(m);
        int rank = -1;
        float e = 0.0f;
        if (lane < mm) {
            e = sc.list[lane];
            rank = 0;
            for (int j = 0; j < mm; ++j) {
                const float x = sc.list[j];
                rank += (x < e) || (x == e && j < lane);
            }
        }
        const unsigned ba = __ballot_sync(dev::kFull, rank == qa);
        const unsigned bb = __ballot_sync(dev::kFull, rank == qa + w);
        a = __shfl_sync(dev::kFull, e, ba ? __ffs(ba) - 1 : 0);
        b = __shfl_sync(dev::kFull, e, bb ? __ffs(bb) - 1 : 0);
        __syncwarp();
        return (ba != 0u && bb != 0u) ? 1 : -1;
    }
    // more than 32: the ends of the rank's bin (and the smallest of rank tr + w's bin)
    bmn = kInf;
    bmx = -kInf;
    wmn = kInf;
#pragma unroll 2
    for (int p = lane; p < n_pairs; p += 32) {
        const float2 x = vw.get(p);
        const int q0 = bm.template of<KEY, CHECK>(x.x, true), q1 = bm.template of<KEY, CHECK>(x.y, p < last_full);
        bmn = fminf(bmn, fminf(q0 == br ? x.x : kInf, q1 == br ? x.y : kInf));
        bmx = fmaxf(bmx, fmaxf(q0 == br ? x.x : -kInf, q1 == br ? x.y : -kInf));
        wmn = fminf(wmn, fminf(q0 == bw ? x.x : kInf, q1 == bw ? x.y : kInf));
    }
    bmn = warp_min(bmn);
    bmx = warp_max(bmx);
    wmn = warp_min(wmn);
    return 0;
}

// Order statistics r and r + w of the n values of the view (get(p): pair p; pairs past n/2 have a
// missing second value when n is odd), in the first level's bracket [lo, hi] (values outside it
// clamped into the end bins).  Bracket invariant: clt values below the bracket, cnt in it, ranks r,
// r + w in [clt, clt + cnt).  A value level halves cnt or is followed by a key level, which cuts
// the bracket's key range by 128 or to single keys: at most 11 + 7 + 6 levels past the first.
template <typename View>
__device__ bool select_pair(const View &vw, int n, int r, int w, float lo, float hi, const Scratch &sc, float &a,
                            float &b) {
    const int n_pairs = (n + 1) >> 1;
    const int last_full = (n & 1) ? n_pairs - 1 : n_pairs;   // pairs below this have both values
    int clt = 0, cnt = n;
    bool by_key = false, check = false;
    for (int level = 0; level <= kMaxLevels; ++level) {
        if (level == kMaxLevels) return false;
        if (check && lo == hi) {
            a = b = lo;
            return true;
        }
        BinMap bm;
        bm.lo = lo;
        bm.hi = hi;
        bm.check = check;
        const float span = hi - lo;
        bm.scale = static_cast<float>(kBins) / span;
        bm.key = by_key || !(span > 0.0f) || !isfinite(span) || !isfinite(bm.scale);
        // key bins: signed zeros at the ends take the key that keeps every bracket value's offset
        // non-negative
        bm.klo = dev::f2key(lo == 0.0f ? -0.0f : lo);
        if (bm.key)
            bm.scale = static_cast<float>(kBins) / (static_cast<float>(dev::f2key(hi == 0.0f ? 0.0f : hi) - bm.klo) + 1.0f);
        int br, bw;
        uint32_t before_r, m;
        float bmn, bmx, wmn;
        int st;
        if (!bm.key && !bm.check)
            st = run_level<false, false>(vw, bm, n_pairs, last_full, r - clt, w, sc, br, bw, before_r, m, bmn, bmx, wmn, a, b);
        else if (!bm.key)
            st = run_level<false, true>(vw, bm, n_pairs, last_full, r - clt, w, sc, br, bw, before_r, m, bmn, bmx, wmn, a, b);
        else if (!bm.check)
            st = run_level<true, false>(vw, bm, n_pairs, last_full, r - clt, w, sc, br, bw, before_r, m, bmn, bmx, wmn, a, b);
        else
            st = run_level<true, true>(vw, bm, n_pairs, last_full, r - clt, w, sc, br, bw, before_r, m, bmn, bmx, wmn, a, b);
        if (st < 0) return false;
        if (st == 1) return true;
        if (bw != br) {   // rank r is its bin's largest value, rank r + 1 the next bin's smallest
            a = bmx;
            b = wmn;
            return true;
        }
        clt += static_cast<int>(before_r);
        by_key = !bm.key && static_cast<int>(m) * 2 > cnt;
        cnt = static_cast<int>(m);
        lo = bmn;
        hi = bmx;
        check = true;
        __syncwarp();
    }
    return false;
}

template <int ST, bool DEV>
struct RowView {
    const void *row;
    float c;
    __device__ __forceinline__ float2 get(int p) const {
        float2 x = row_pair<ST>(row, p);
        if constexpr (DEV) {
            x.x = fabsf(x.x - c);
            x.y = fabsf(x.y - c);
        }
        return x;
    }
};

// Shared memory of one warp: its row buffer (n_t + 1 samples of es bytes, as stored), histogram,
// gather space.
__host__ __device__ inline size_t row_buf_bytes(int es, int n_t) {
    return ((static_cast<size_t>(es) * static_cast<size_t>(n_t + 1) + 15) / 16) * 16;
}
__host__ __device__ inline size_t warp_smem_bytes(int es, int n_t) {
    return row_buf_bytes(es, n_t) + sizeof(uint32_t) * (kBins + 4) + sizeof(float) * (32 * kColPitch + 32);
}

// VEC: rows copied by 16-byte loads (16-byte aligned cube and output, rows of whole 16 bytes).
template <int ST, bool VEC>
__global__ void __launch_bounds__(kMadWarps * 32) mad_normalise_kernel(const void *__restrict__ cube, int64_t pix0,
                                                                     int64_t n_pix, int n_sub, int n_t,
                                                                     float *__restrict__ out,
                                                                     uint8_t *__restrict__ bad) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int kEs = ST == 0 ? 4 : 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *mine = smem + warp * warp_smem_bytes(kEs, n_t);
    void *row = mine;
    Scratch sc;
    sc.hist = reinterpret_cast<uint32_t *>(mine + row_buf_bytes(kEs, n_t));
    sc.cols = reinterpret_cast<float *>(sc.hist + kBins + 4);
    sc.list = sc.cols + 32 * kColPitch;
    const float kInf = __int_as_float(0x7f800000);
    const int64_t n_rows = n_pix * n_sub;
    const int n = n_t, r = (n_t - 1) / 2, w = (n_t & 1) ? 0 : 1;
    const int n_pairs = (n + 1) >> 1;
    for (int64_t rr = static_cast<int64_t>(blockIdx.x) * kMadWarps + warp; rr < n_rows;
         rr += static_cast<int64_t>(gridDim.x) * kMadWarps) {
        const int64_t src = (pix0 * n_sub + rr) * n_t;
        // copy the row as stored; sums of (x - x0) and its square about the row's first sample
        const float x0 = dev::load_elem(cube, src, ST);
        float s1 = 0.0f, s2 = 0.0f;
        __syncwarp();
        if constexpr (VEC) {
            const uint4 *g = reinterpret_cast<const uint4 *>(static_cast<const unsigned char *>(cube) + src * kEs);
            uint4 *d = reinterpret_cast<uint4 *>(row);
            const int n16 = n_t * kEs / 16;
            for (int i = lane; i < n16; i += 32) {
                const uint4 u = __ldg(g + i);
                d[i] = u;
                const uint32_t wv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    if constexpr (ST == 0) {
                        const float y = __uint_as_float(wv[h]) - x0;
                        s1 += y;
                        s2 = fmaf(y, y, s2);
                    } else {
                        const float2 f = row_pair<ST>(&wv[h], 0);
                        const float y0 = f.x - x0, y1 = f.y - x0;
                        s1 += y0 + y1;
                        s2 = fmaf(y0, y0, fmaf(y1, y1, s2));
                    }
                }
            }
        } else {
            for (int t = lane; t < n_t; t += 32) {
                const float x = dev::load_elem(cube, src + t, ST);
                if constexpr (ST == 0)
                    reinterpret_cast<float *>(row)[t] = x;
                else
                    reinterpret_cast<unsigned short *>(row)[t] = static_cast<const unsigned short *>(cube)[src + t];
                const float y = x - x0;
                s1 += y;
                s2 = fmaf(y, y, s2);
            }
        }
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        __syncwarp();
        const float mu = s1 / static_cast<float>(n), var = fmaxf(s2 / static_cast<float>(n) - mu * mu, 0.0f);
        const float sd = sqrtf(var), mean = x0 + mu;
        float a, b;
        bool ok;
        // samples: first bracket mean +- 3 s (a bracket of zero width or beyond the float range
        // falls back to the key bins over the row's extremes)
        {
            float lo = mean - 3.0f * sd, hi = mean + 3.0f * sd;
            if (!(hi > lo) || !isfinite(lo) || !isfinite(hi)) {
                float mn = kInf, mx = -kInf;
                for (int p = lane; p < n_pairs; p += 32) {
                    const float2 x = row_pair<ST>(row, p);
                    mn = fminf(mn, x.x);
                    mx = fmaxf(mx, x.x);
                    if (2 * p + 1 < n) {
                        mn = fminf(mn, x.y);
                        mx = fmaxf(mx, x.y);
                    }
                }
                lo = warp_min(mn);
                hi = warp_max(mx);
            }
            ok = select_pair(RowView<ST, false>{row, 0.0f}, n, r, w, lo, hi, sc, a, b);
        }
        const float med = w ? 0.5f * (a + b) : a;
        {
            // deviations: first bracket [0, 3 s] (or, for s = 0, the largest deviation)
            float hi = 3.0f * sd;
            if (!(hi > 0.0f) || !isfinite(hi)) {
                float mx = 0.0f;
                for (int p = lane; p < n_pairs; p += 32) {
                    const float2 x = row_pair<ST>(row, p);
                    mx = fmaxf(mx, fabsf(x.x - med));
                    if (2 * p + 1 < n) mx = fmaxf(mx, fabsf(x.y - med));
                }
                hi = warp_max(mx);
            }
            ok = select_pair(RowView<ST, true>{row, med}, n, r, w, 0.0f, hi, sc, a, b) && ok;
        }
        const float mad = w ? 0.5f * (a + b) : a;
        float *dst = out + rr * n_t;
        if (mad == 0.0f || !ok) {
            for (int t = lane; t < n_t; t += 32) dst[t] = 0.0f;
            if (lane == 0) bad[pix0 + rr / n_sub] = 1;
        } else {
            const float inv = 1.0f / (1.4826f * mad);
            if constexpr (VEC) {
                // four samples per lane and step: one 16-byte store
                for (int q = lane; q < n_t / 4; q += 32) {
                    const float2 y0 = row_pair<ST>(row, 2 * q), y1 = row_pair<ST>(row, 2 * q + 1);
                    reinterpret_cast<float4 *>(dst)[q] =
                        make_float4((y0.x - med) * inv, (y0.y - med) * inv, (y1.x - med) * inv, (y1.y - med) * inv);
                }
            } else {
                for (int t = lane; t < n_t; t += 32) {
                    const float x = (ST == 0) ? reinterpret_cast<const float *>(row)[t]
                                              : dev::widen16(reinterpret_cast<const unsigned short *>(row)[t], ST);
                    dst[t] = (x - med) * inv;
                }
            }
        }
    }
}

template <int ST, bool VEC>
cudaError_t launch_mad(const void *cube, int64_t pix0, int64_t n_pix, int n_sub, int n_t, float *out, uint8_t *bad,
                       int n_sm, cudaStream_t s) {
    const size_t smem = kMadWarps * warp_smem_bytes(ST == 0 ? 4 : 2, n_t);
    cudaError_t e = cudaFuncSetAttribute(mad_normalise_kernel<ST, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mad_normalise_kernel<ST, VEC>, kMadWarps * 32, smem);
    if (e != cudaSuccess) return e;
    const int64_t rows = n_pix * n_sub;
    const int64_t blocks = std::min<int64_t>((rows + kMadWarps - 1) / kMadWarps,
                                             static_cast<int64_t>(n_sm) * std::max(1, per_sm));
    mad_normalise_kernel<ST, VEC><<<static_cast<unsigned>(std::max<int64_t>(1, blocks)), kMadWarps * 32, smem, s>>>(
        cube, pix0, n_pix, n_sub, n_t, out, bad);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mad_normalise(const void *cube, int dtype, int64_t pix0, int64_t n_pix, int n_sub, int n_t,
                                 float *out, uint8_t *bad, int n_sm, cudaStream_t s) {
    // 16-byte loads and stores need 16-byte aligned rows (an aligned cube and output, rows of whole
    // 16 bytes in both)
    const size_t es = dtype == NSFRB_F32 ? 4 : 2;
    const bool vec = reinterpret_cast<uintptr_t>(cube) % 16 == 0 && (es * n_t) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(out) % 16 == 0 && (4 * static_cast<size_t>(n_t)) % 16 == 0;
    if (dtype == NSFRB_F32)
        return vec ? launch_mad<0, true>(cube, pix0, n_pix, n_sub, n_t, out, bad, n_sm, s)
                   : launch_mad<0, false>(cube, pix0, n_pix, n_sub, n_t, out, bad, n_sm, s);
    if (dtype == NSFRB_BF16)
        return vec ? launch_mad<1, true>(cube, pix0, n_pix, n_sub, n_t, out, bad, n_sm, s)
                   : launch_mad<1, false>(cube, pix0, n_pix, n_sub, n_t, out, bad, n_sm, s);
    return vec ? launch_mad<2, true>(cube, pix0, n_pix, n_sub, n_t, out, bad, n_sm, s)
               : launch_mad<2, false>(cube, pix0, n_pix, n_sub, n_t, out, bad, n_sm, s);
}

}  // namespace nsfrb
