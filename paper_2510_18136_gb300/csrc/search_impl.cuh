// Fused image-plane single-pulse search kernel (arXiv 2510.18136, Sec. 2.2):
// per pixel, de-disperse every DM trial with integer shifts, boxcar-filter
// every width with prefix sums, normalise to S/N, maximise over time, width
// and DM.  Included by one translation unit per chunk size C.
//
// Organisation (one CTA of 12 warps per pixel, persistent over pixels):
//  * The pixel's [n_sub][n_t] tile is staged in shared memory (bulk copies
//    into a double buffer for FP32, or into a 16-bit staging double buffer
//    that is widened to FP32), with -inf beyond n_t so that every time series
//    element that would read past the window is non-finite.
//  * Distinct shift rows (DM trials with identical integer tables are one
//    row) are split into 12 contiguous groups, one per warp.  A warp builds
//    the first row of its group from all subbands and each later row from
//    the previous one by adding/subtracting only the subbands whose shift
//    changed (sorted DMs change a few subbands per row).
//  * Lane j owns samples [j*C, (j+1)*C): de-dispersed values D, then the
//    in-lane prefix Lp and one warp scan of lane totals give P = sum D.
//  * Widths w <= min(C,16) are evaluated in-lane from Lp (plus a shuffled
//    halo from the next lane); widths that are multiples of 32 from P
//    re-read lane-strided (P[32 i + j]) so that P[t + w] is a register of the
//    same lane; any other width from P in shared memory.
//  * Elements beyond the valid range are -inf or NaN and are dropped by
//    fmaxf, so no per-element bounds test is needed.
#pragma once

#include <climits>
#include <cmath>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "async_copy.cuh"
#include "nsfrb_internal.h"

namespace nsfrb {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kHistBinsPerLane = kHistBins / 32;
__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }
__device__ __forceinline__ float qnan() { return __int_as_float(0x7fffffff); }

__device__ __forceinline__ float load_elem(const void *base, int64_t i, int dtype) {
    if (dtype == 0) return static_cast<const float *>(base)[i];
    const unsigned short u = static_cast<const unsigned short *>(base)[i];
    if (dtype == 1) return __uint_as_float(static_cast<uint32_t>(u) << 16);
    return __half2float(__ushort_as_half(u));
}

__device__ __forceinline__ float widen16(unsigned short u, int dtype) {
    if (dtype == 1) return __uint_as_float(static_cast<uint32_t>(u) << 16);
    return __half2float(__ushort_as_half(u));
}

// ------------------------------------------------------------------ radix select (MAD mode)

__device__ __forceinline__ uint32_t f2key(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Exact order statistic of rank `rank` (0-based) of v[0..n) by one warp: 8-bit radix passes
// over an order-preserving integer key, from the top byte down.  With key16 every key's low 16
// bits are fixed by its sign (v holds BF16 values widened to FP32: 0 for positive, 0xffff for
// negative keys), so two passes fix the key.  Returns the key.
static __device__ __noinline__ uint32_t warp_select_key(const float *v, int n, int rank, uint32_t *hist, bool key16) {
    const int lane = threadIdx.x & 31;
    uint32_t prefix = 0, pmask = 0;
    const int last = key16 ? 16 : 0;
#pragma unroll 1
    for (int shift = 24; shift >= last; shift -= 8) {
        for (int i = lane; i < kHistBins; i += 32) hist[i] = 0;
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            const uint32_t key = f2key(v[i]);
            if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
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
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - s;
        const bool mine = (static_cast<uint32_t>(rank) >= excl) && (static_cast<uint32_t>(rank) < incl);
        const unsigned bal = __ballot_sync(kFull, mine);
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
        digit = __shfl_sync(kFull, digit, src);
        before = __shfl_sync(kFull, before, src);
        rank -= static_cast<int>(before);
        prefix |= static_cast<uint32_t>(digit) << shift;
        pmask |= 255u << shift;
        __syncwarp();
    }
    if (key16) prefix |= (prefix & 0x80000000u) ? 0u : 0xffffu;
    return prefix;
}

// Median of v[0..n): the middle order statistic, or for even n the mean of the two middle
// ones, the upper found from the lower: it equals the lower when more than n / 2 keys are at
// most the lower's key, else it is the smallest key above it.
static __device__ __noinline__ float warp_median(const float *v, int n, uint32_t *hist, bool key16) {
    const uint32_t ka = warp_select_key(v, n, (n - 1) / 2, hist, key16);
    const float a = key2f(ka);
    if (n & 1) return a;
    const int lane = threadIdx.x & 31;
    uint32_t le = 0, above = 0xffffffffu;
    for (int i = lane; i < n; i += 32) {
        const uint32_t key = f2key(v[i]);
        if (key <= ka)
            ++le;
        else
            above = min(above, key);
    }
    le = __reduce_add_sync(kFull, le);
    above = __reduce_min_sync(kFull, above);
    const float b = (le >= static_cast<uint32_t>(n / 2) + 1) ? a : key2f(above);
    return 0.5f * (a + b);
}

// ------------------------------------------------------------------ boxcar building blocks

// Three-input maximum (sm_100+ form of max.f32); NaN inputs are ignored like
// the two-input form, so elements outside the valid range drop out.
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// max over f(0..N-1) with three independent accumulators of 3-input maxima (three short
// dependency chains instead of one long one), combined by one more 3-input maximum.
template <int N, typename F>
__device__ __forceinline__ float tree_max(F f) {
    float acc[3] = {neg_inf(), neg_inf(), neg_inf()};
#pragma unroll
    for (int j = 0; j + 1 < N; j += 2) acc[(j >> 1) % 3] = fmax3(acc[(j >> 1) % 3], f(j), f(j + 1));
    if constexpr (N & 1) acc[2] = fmaxf(acc[2], f(N - 1));
    return fmax3(acc[0], acc[1], acc[2]);
}

// In-lane small width W: B[c] = P[t0+c+W] - P[t0+c] from the in-lane prefix Lp
// (Lp[c] = sum of this lane's D[0..c)) and the halo H[i] = total + Lp_next[i].
template <int C, int SH, int W>
__device__ __forceinline__ float small_max_w(const float (&Lp)[C + 1], const float (&H)[SH + 1]) {
    return tree_max<C>([&](int c) { return (c + W <= C) ? Lp[c + W] - Lp[c] : H[c + W - C] - Lp[c]; });
}

template <int C, int SH, int W>
__device__ __forceinline__ int small_find_w(const float (&Lp)[C + 1], const float (&H)[SH + 1],
                                            float inv, float target, int t0) {
    int found = INT_MAX;
#pragma unroll
    for (int c = C - 1; c >= 0; --c) {
        float b;
        if (c + W <= C)
            b = Lp[c + W] - Lp[c];
        else
            b = H[c + W - C] - Lp[c];
        if (b * inv == target) found = t0 + c;
    }
    return found;
}

#define NSFRB_SMALL_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

template <int C, int SH>
__device__ __forceinline__ int small_find(int w, const float (&Lp)[C + 1], const float (&H)[SH + 1],
                                          float inv, float target, int t0) {
    switch (w) {
#define NSFRB_SC(W)                                                                  \
    case W:                                                                          \
        if constexpr (W <= SH) return small_find_w<C, SH, W>(Lp, H, inv, target, t0); \
        break;
        NSFRB_SMALL_CASES(NSFRB_SC)
#undef NSFRB_SC
        default:
            break;
    }
    return INT_MAX;
}

// Lane-strided width 32*M: Ps[i] = P[32 i + lane]; B = Ps[i+M] - Ps[i].
template <int C, int M>
__device__ __forceinline__ float large_max_m(const float (&Ps)[C]) {
    return tree_max<C - M>([&](int i) { return Ps[i + M] - Ps[i]; });
}

template <int C, int M>
__device__ __forceinline__ int large_find_m(const float (&Ps)[C], float inv, float target, int lane) {
    int found = INT_MAX;
#pragma unroll
    for (int i = C - 1 - M; i >= 0; --i)
        if ((Ps[i + M] - Ps[i]) * inv == target) found = 32 * i + lane;
    return found;
}

#define NSFRB_LARGE_CASES(X)                                                                     \
    X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) \
    X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)   \
    X(33) X(34) X(35) X(36) X(37) X(38)

template <int C>
__device__ __forceinline__ int large_find(int m, const float (&Ps)[C], float inv, float target,
                                          int lane) {
    switch (m) {
#define NSFRB_LC(M)                                                          \
    case M:                                                                  \
        if constexpr (M < C) return large_find_m<C, M>(Ps, inv, target, lane); \
        break;
        NSFRB_LARGE_CASES(NSFRB_LC)
#undef NSFRB_LC
        default:
            break;
    }
    return INT_MAX;
}

// Any width from P in shared memory; trials t in [t_lo, L - w].
__device__ __forceinline__ float generic_max(const float *Pw, int w, int L, int t_lo, int lane) {
    float m = neg_inf();
    for (int t = t_lo + lane; t + w <= L; t += 32) m = fmaxf(m, Pw[t + w] - Pw[t]);
    return m;
}

__device__ __forceinline__ int generic_find(const float *Pw, int w, int L, int t_lo, int lane,
                                            float inv, float target) {
    for (int t = t_lo + lane; t + w <= L; t += 32)
        if ((Pw[t + w] - Pw[t]) * inv == target) return t;
    return INT_MAX;
}

// Serving (at most 32 new trial ends per width, nb = new_blk <= 32): lane j takes, for every width
// w, the trial whose boxcar ends at the same prefix index e = L - nb + 1 + j (t = e - w), so P[e] is
// read once per row; lanes j >= nb, and trials with t < 0, give -inf.  The trials are those of
// t in [max(0, L - w - nb + 1), L - w], and each S/N is P[t + w] - P[t] as in every other path.
__device__ __forceinline__ int masked_end(int L, int nb, int lane) {
    const int e = L - nb + 1 + lane;
    return (lane < nb && e >= 0) ? e : -1;
}

__device__ __forceinline__ int masked_find32(const float *Pw, int w, int e, float inv, float target) {
    const int t = e - w;
    const bool ok = e >= 0 && t >= 0;
    const float b = Pw[ok ? e : 0] - Pw[ok ? t : 0];
    return (ok && b * inv == target) ? t : INT_MAX;
}

#define NSFRB_POW2(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

// In-lane prefix of this lane's chunk: Lp[c] = D[0] + ... + D[c-1]; returns the total.
// Two independent half chains (the second half is summed from its own start and
// then offset by the first half's total) halve the dependent-add latency.
template <int C>
__device__ __forceinline__ float lane_prefix(const float (&D)[C], float (&Lp)[C + 1]) {
    constexpr int H1 = (C + 1) / 2;
    Lp[0] = 0.0f;
#pragma unroll
    for (int c = 0; c < H1; ++c) Lp[c + 1] = Lp[c] + D[c];
    if constexpr (C > H1) {
        float q[C - H1];
        q[0] = D[H1];
#pragma unroll
        for (int j = 1; j < C - H1; ++j) q[j] = q[j - 1] + D[H1 + j];
#pragma unroll
        for (int j = 0; j < C - H1; ++j) Lp[H1 + 1 + j] = Lp[H1] + q[j];
    }
    return Lp[C];
}

// Halo for the in-lane small widths: H[i] = this lane's total + the next
// lane's Lp[i] (= P at the next chunk's sample i, relative to this chunk).
template <int C, int SH>
__device__ __forceinline__ void lane_halo(const float (&Lp)[C + 1], float tot, int lane, float (&H)[SH + 1]) {
    H[0] = 0.0f;
#pragma unroll
    for (int i = 1; i <= SH; ++i) {
        const float v = __shfl_down_sync(kFull, Lp[i], 1);
        H[i] = (lane == 31) ? qnan() : tot + v;
    }
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// ------------------------------------------------------------------ even chunks: sample pairs
//
// With an even C (C = 2 mod 4, so 64-bit accesses of lanes C words apart are conflict-free)
// a lane's samples are held as pairs (2m, 2m+1): shared-memory rows are read and P is written
// 64 bits at a time, and the de-dispersion sums and boxcar differences run as two-lane FP32
// instructions.  Each lane of a pair op rounds exactly like the scalar op, so every value
// equals the one-sample-at-a-time computation.

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float pget(const float2 *v, int i) { return (i & 1) ? v[i >> 1].y : v[i >> 1].x; }
__device__ __forceinline__ void pset(float2 *v, int i, float x) {
    if (i & 1)
        v[i >> 1].y = x;
    else
        v[i >> 1].x = x;
}

// D[c] += xr[c] (SUB: D[c] -= xr[c]) for c < C, xr = subband row + t0 + s.  For even s the
// row is read in aligned pairs; for odd s the aligned pairs from xr - 1 are realigned.
template <int C, bool SUB>
__device__ __forceinline__ void acc_pairs(float2 (&D)[C / 2], const float *xr, bool odd) {
    if (!odd) {
        const float2 *x = reinterpret_cast<const float2 *>(xr);
#pragma unroll
        for (int m = 0; m < C / 2; ++m) D[m] = SUB ? sub2(D[m], x[m]) : add2(D[m], x[m]);
    } else {
        const float2 *x = reinterpret_cast<const float2 *>(xr - 1);
        float lo = x[0].y;
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const float2 v = x[m + 1];
            D[m].x = SUB ? D[m].x - lo : D[m].x + lo;
            D[m].y = SUB ? D[m].y - v.x : D[m].y + v.x;
            lo = v.y;
        }
    }
}

// 16-bit storage read in place: x + y and y - x with x a BF16 (ST = 1) or FP16 (ST = 2) value and
// y FP32, by the mixed-precision add and fma of sm_100+.  x widens exactly, so each result is the
// FP32 operation on the widened value, rounded once: the same values as widening first.
template <int ST>
__device__ __forceinline__ float2 add16x2(float2 d, uint32_t u) {
    float2 r;
    if constexpr (ST == 1)
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tadd.rn.f32.bf16 %0, l, %3;\n\t"
            "add.rn.f32.bf16 %1, h, %4;\n\t}"
            : "=f"(r.x), "=f"(r.y) : "r"(u), "f"(d.x), "f"(d.y));
    else
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tadd.rn.f32.f16 %0, l, %3;\n\t"
            "add.rn.f32.f16 %1, h, %4;\n\t}"
            : "=f"(r.x), "=f"(r.y) : "r"(u), "f"(d.x), "f"(d.y));
    return r;
}
// d - x = fma(x, -1, d): the product is exact, the one rounding that of the subtraction.
template <int ST>
__device__ __forceinline__ float2 sub16x2(float2 d, uint32_t u) {
    float2 r;
    if constexpr (ST == 1)
        asm("{\n\t.reg .b16 l, h, m;\n\tmov.b32 {l, h}, %2;\n\tmov.b16 m, 0xBF80;\n\t"
            "fma.rn.f32.bf16 %0, l, m, %3;\n\tfma.rn.f32.bf16 %1, h, m, %4;\n\t}"
            : "=f"(r.x), "=f"(r.y) : "r"(u), "f"(d.x), "f"(d.y));
    else
        asm("{\n\t.reg .b16 l, h, m;\n\tmov.b32 {l, h}, %2;\n\tmov.b16 m, 0xBC00;\n\t"
            "fma.rn.f32.f16 %0, l, m, %3;\n\tfma.rn.f32.f16 %1, h, m, %4;\n\t}"
            : "=f"(r.x), "=f"(r.y) : "r"(u), "f"(d.x), "f"(d.y));
    return r;
}

// D[c] += x[e + c] (SUB: D[c] -= x[e + c]) for c < C from a 16-bit row in shared memory read as
// 32-bit words (two samples each); for odd e the pair (x[e + 2m], x[e + 2m + 1]) straddles two
// words and is reassembled by a byte permute.
template <int C, bool SUB, int ST>
__device__ __forceinline__ void acc_pairs16(float2 (&D)[C / 2], const uint16_t *row, int e) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(row + (e & ~1));
    if (!(e & 1)) {
#pragma unroll
        for (int m = 0; m < C / 2; ++m) D[m] = SUB ? sub16x2<ST>(D[m], w[m]) : add16x2<ST>(D[m], w[m]);
    } else {
        uint32_t lo = w[0];
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const uint32_t hi = w[m + 1];
            const uint32_t u = __byte_perm(lo, hi, 0x5432);
            D[m] = SUB ? sub16x2<ST>(D[m], u) : add16x2<ST>(D[m], u);
            lo = hi;
        }
    }
}

// Subband row k of a pixel tile in storage ST, its sample t + s (window offset eoff within the row).
template <int C, bool SUB, int ST>
__device__ __forceinline__ void acc_row(float2 (&D)[C / 2], const void *xs, int Tp, int k, int e) {
    if constexpr (ST == 0) {
        const float *r = static_cast<const float *>(xs) + (size_t)k * Tp + e;
        acc_pairs<C, SUB>(D, r, e & 1);
    } else {
        acc_pairs16<C, SUB, ST>(D, static_cast<const uint16_t *>(xs) + (size_t)k * Tp, e);
    }
}

// First row of a group: D = sum over subbands k of x_k(t + s_k), subbands in order.
template <int C, int ST>
__device__ __forceinline__ void dd_first(float2 (&D)[C / 2], const void *xs, int Tp, int n_sub,
                                         const int32_t *sh, int t0) {
#pragma unroll
    for (int m = 0; m < C / 2; ++m) D[m] = make_float2(0.0f, 0.0f);
#pragma unroll 1
    for (int k = 0; k < n_sub; ++k) acc_row<C, false, ST>(D, xs, Tp, k, t0 + sh[k]);
}

// D[c] += x[c + 1] - x[c] for c < C, xr = subband row + t0 + s (FP32): a subband whose shift grew
// by one sample, both terms from one read of the row.  The two differences of a pair are scalar
// (they straddle the loaded pairs), their sum with D a two-lane add.
template <int C>
__device__ __forceinline__ void acc_step1(float2 (&D)[C / 2], const float *xr, bool odd) {
    if (!odd) {
        const float2 *x = reinterpret_cast<const float2 *>(xr);     // x[m] = (xr[2m], xr[2m + 1])
        float2 v = x[0];
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const float2 nx = x[m + 1];
            D[m] = add2(D[m], make_float2(v.y - v.x, nx.x - v.y));
            v = nx;
        }
    } else {
        const float2 *x = reinterpret_cast<const float2 *>(xr - 1); // x[m] = (xr[2m - 1], xr[2m])
        float a = x[0].y;
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const float2 nx = x[m + 1];
            D[m] = add2(D[m], make_float2(nx.x - a, nx.y - nx.x));
            a = nx.y;
        }
    }
}

// acc_step1 for a 16-bit row read in place as 32-bit words: D[c] = (D[c] + x[e + c + 1]) - x[e + c]
// by the mixed-precision add and fma (the operations of acc_pairs16's add and subtract, from one
// read of the row).  u, nu: the words holding the pair's samples; OD: e odd.
template <int ST, bool OD>
__device__ __forceinline__ void step1_pair16(float2 &d, uint32_t u, uint32_t nu) {
    // even e: (x[2m], x[2m+1]) = (lo u, hi u), x[2m+2] = lo nu
    //   d.x = (d.x + hi u) - lo u,  d.y = (d.y + lo nu) - hi u
    // odd e:  x[2m] = hi u, (x[2m+1], x[2m+2]) = (lo nu, hi nu)
    //   d.x = (d.x + lo nu) - hi u, d.y = (d.y + hi nu) - lo nu
    if constexpr (ST == 1) {
        if constexpr (!OD)
            asm("{\n\t.reg .b16 ul, uh, nl, nh, m;\n\tmov.b32 {ul, uh}, %2;\n\tmov.b32 {nl, nh}, %3;\n\t"
                "mov.b16 m, 0xBF80;\n\tadd.rn.f32.bf16 %0, uh, %0;\n\tfma.rn.f32.bf16 %0, ul, m, %0;\n\t"
                "add.rn.f32.bf16 %1, nl, %1;\n\tfma.rn.f32.bf16 %1, uh, m, %1;\n\t}"
                : "+f"(d.x), "+f"(d.y) : "r"(u), "r"(nu));
        else
            asm("{\n\t.reg .b16 ul, uh, nl, nh, m;\n\tmov.b32 {ul, uh}, %2;\n\tmov.b32 {nl, nh}, %3;\n\t"
                "mov.b16 m, 0xBF80;\n\tadd.rn.f32.bf16 %0, nl, %0;\n\tfma.rn.f32.bf16 %0, uh, m, %0;\n\t"
                "add.rn.f32.bf16 %1, nh, %1;\n\tfma.rn.f32.bf16 %1, nl, m, %1;\n\t}"
                : "+f"(d.x), "+f"(d.y) : "r"(u), "r"(nu));
    } else {
        if constexpr (!OD)
            asm("{\n\t.reg .b16 ul, uh, nl, nh, m;\n\tmov.b32 {ul, uh}, %2;\n\tmov.b32 {nl, nh}, %3;\n\t"
                "mov.b16 m, 0xBC00;\n\tadd.rn.f32.f16 %0, uh, %0;\n\tfma.rn.f32.f16 %0, ul, m, %0;\n\t"
                "add.rn.f32.f16 %1, nl, %1;\n\tfma.rn.f32.f16 %1, uh, m, %1;\n\t}"
                : "+f"(d.x), "+f"(d.y) : "r"(u), "r"(nu));
        else
            asm("{\n\t.reg .b16 ul, uh, nl, nh, m;\n\tmov.b32 {ul, uh}, %2;\n\tmov.b32 {nl, nh}, %3;\n\t"
                "mov.b16 m, 0xBC00;\n\tadd.rn.f32.f16 %0, nl, %0;\n\tfma.rn.f32.f16 %0, uh, m, %0;\n\t"
                "add.rn.f32.f16 %1, nh, %1;\n\tfma.rn.f32.f16 %1, nl, m, %1;\n\t}"
                : "+f"(d.x), "+f"(d.y) : "r"(u), "r"(nu));
    }
}

template <int C, int ST>
__device__ __forceinline__ void acc_step1_16(float2 (&D)[C / 2], const uint16_t *row, int e) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(row + (e & ~1));
    uint32_t u = w[0];
    if (!(e & 1)) {
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const uint32_t nu = w[m + 1];
            step1_pair16<ST, false>(D[m], u, nu);
            u = nu;
        }
    } else {
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const uint32_t nu = w[m + 1];
            step1_pair16<ST, true>(D[m], u, nu);
            u = nu;
        }
    }
}

// Next row from the previous one: per changed subband, D = (D + x_k(t + s_new)) - x_k(t + s_old),
// both from one read of the row where the shift grew by one sample; for FP32 rows that case is
// D = D + (x_k(t + s_old + 1) - x_k(t + s_old)).  (Within a row the -inf past the window is a
// suffix, so x(t) = -inf implies x(t + 1) = -inf: the difference is never +inf, and a de-dispersed
// value past the valid range stays -inf or NaN.)
template <int C, int ST>
__device__ __forceinline__ void dd_delta(float2 (&D)[C / 2], const void *xs, int Tp, const int32_t *s_delta,
                                         int d0, int nd, int t0) {
#pragma unroll 1
    for (int e = d0; e < d0 + nd; ++e) {
        const uint32_t pk = static_cast<uint32_t>(s_delta[e]);
        const int k = pk & 63u, so = (pk >> 6) & 0x1fffu, sn = pk >> 19;
        if (sn == so + 1) {
            const int at = t0 + so;
            if constexpr (ST == 0)
                acc_step1<C>(D, static_cast<const float *>(xs) + (size_t)k * Tp + at, at & 1);
            else
                acc_step1_16<C, ST>(D, static_cast<const uint16_t *>(xs) + (size_t)k * Tp, at);
            continue;
        }
        acc_row<C, false, ST>(D, xs, Tp, k, t0 + sn);
        acc_row<C, true, ST>(D, xs, Tp, k, t0 + so);
    }
}

// In-lane prefix Lp[c] = D[0] + ... + D[c-1] for c < C as pairs; returns Lp[C] (the lane
// total).  Two chains split at an even sample, the second offset by the first's total.
template <int C>
__device__ __forceinline__ float prefix_pairs(const float2 (&D)[C / 2], float2 (&Lp)[C / 2]) {
    constexpr int H1 = 2 * ((C / 2 + 1) / 2);
    float run = 0.0f, tot = 0.0f;
    Lp[0].x = 0.0f;
#pragma unroll
    for (int c = 0; c < H1; ++c) {
        run = run + pget(D, c);
        if (c + 1 < C)
            pset(Lp, c + 1, run);
        else
            tot = run;
    }
    if constexpr (C > H1) {
        // second chain q[j] = D[H1] + ... + D[H1 + j], then Lp[H1 + 1 + j] = run + q[j]; H1 + 1 is
        // odd (C even), so the offsets of the whole pairs (Lp[H1 + 2], Lp[H1 + 3]) ... (Lp[C - 2],
        // Lp[C - 1]) are two-lane adds (each lane rounds like the scalar add: the same values)
        float q[C - H1];
        q[0] = pget(D, H1);
#pragma unroll
        for (int j = 1; j < C - H1; ++j) q[j] = q[j - 1] + pget(D, H1 + j);
        if constexpr (H1 + 1 < C) pset(Lp, H1 + 1, run + q[0]);
        const float2 rr = make_float2(run, run);
#pragma unroll
        for (int i = H1 + 2; i + 1 < C; i += 2) Lp[i >> 1] = add2(rr, make_float2(q[i - H1 - 1], q[i - H1]));
        tot = run + q[C - H1 - 1];
    }
    return tot;
}

// P[t0 + c] = carry + Lp[c] to shared memory, 64 bits at a time.
template <int C>
__device__ __forceinline__ void store_p(float *Pw, int t0, float carry, const float2 (&Lp)[C / 2]) {
    const float2 cc = make_float2(carry, carry);
    float2 *dst = reinterpret_cast<float2 *>(Pw + t0);
#pragma unroll
    for (int m = 0; m < C / 2; ++m) dst[m] = add2(cc, Lp[m]);
}

// Halo as pairs: Hh holds h[i] for i < SH, h[0] = the lane total (= Lp[C]) and
// h[i] = total + the next lane's Lp[i], so that the extended in-lane prefix
// E = (Lp[0..C), h[0..SH)) pairs up as (E[2j], E[2j+1]).  The last lane needs no mask: its chunk
// ends at sample 32 C - 1 >= n_t, whose de-dispersed value is -inf or NaN (-inf past the window,
// NaN where a row difference subtracted -inf from -inf), so its total and every h[i] are -inf or
// NaN, and each trial that reads them drops out of every maximum and never equals a target.
// (Only the unmasked search calls this; a masked search evaluates no in-lane widths.)
template <int C, int SH>
__device__ __forceinline__ void halo_pairs(const float2 (&Lp)[C / 2], float tot, float2 (&Hh)[SH / 2]) {
    Hh[0].x = tot;
#pragma unroll
    for (int i = 1; i < SH; ++i) pset(Hh, i, tot + __shfl_down_sync(kFull, pget(Lp, i), 1));
}

template <int C, int SH>
__device__ __forceinline__ float2 ext_pair(const float2 (&Lp)[C / 2], const float2 (&Hh)[SH / 2], int j) {
    return (j < C / 2) ? Lp[j] : Hh[j - C / 2];
}

// In-lane width W <= SH: W = 1 is the de-dispersed sample itself; an even W is the difference
// of extended prefix pairs W / 2 apart.
template <int C, int SH, int W>
__device__ __forceinline__ float small_max_pk(const float2 (&D)[C / 2], const float2 (&Lp)[C / 2],
                                              const float2 (&Hh)[SH / 2]) {
    static_assert(W == 1 || W % 2 == 0, "in-lane widths are 1 or even");
    float acc[3] = {neg_inf(), neg_inf(), neg_inf()};
#pragma unroll
    for (int m = 0; m < C / 2; ++m) {
        float2 b;
        if constexpr (W == 1)
            b = D[m];
        else
            b = sub2(ext_pair<C, SH>(Lp, Hh, m + W / 2), ext_pair<C, SH>(Lp, Hh, m));
        acc[m % 3] = fmax3(acc[m % 3], b.x, b.y);
    }
    return fmax3(acc[0], acc[1], acc[2]);
}

// Lane-strided P as pairs: Ps[m] = (P[64 m + lane], P[64 m + 32 + lane]).
template <int C>
__device__ __forceinline__ void load_ps(const float *Pw, int lane, float2 (&Ps)[C / 2]) {
#pragma unroll
    for (int m = 0; m < C / 2; ++m) Ps[m] = make_float2(Pw[64 * m + lane], Pw[64 * m + 32 + lane]);
}

// Width 32 M, M < C: B = Ps[i + M] - Ps[i] over i < C - M; pairs for even M.
template <int C, int M>
__device__ __forceinline__ float large_max_pk(const float2 (&Ps)[C / 2]) {
    if constexpr (M % 2 == 0) {
        float acc[3] = {neg_inf(), neg_inf(), neg_inf()};
#pragma unroll
        for (int m = 0; m < (C - M) / 2; ++m) {
            const float2 b = sub2(Ps[m + M / 2], Ps[m]);
            acc[m % 3] = fmax3(acc[m % 3], b.x, b.y);
        }
        return fmax3(acc[0], acc[1], acc[2]);
    } else {
        return tree_max<C - M>([&](int i) { return pget(Ps, i + M) - pget(Ps, i); });
    }
}

// ------------------------------------------------------------------ one warp, one pixel

// Called by a warp (all lanes) once it has read the pixel's rows for the last time: after the
// de-dispersion of its last row, or at once when its group is empty.  The barrier-free kernel
// uses it to start the next copy into the buffer early; the other callers pass this no-op.
struct NoReadDone {
    __device__ __forceinline__ void operator()() const {}
};

// FULL mode: one distinct row's results, width wi's on lane wi, written by lanes 0..n_w-1 for
// every DM of the row (a DM's widths are contiguous: one store per DM and array).
__device__ __forceinline__ void full_store_row(const SearchParams &p, const int32_t *info, int64_t pix, int lane,
                                               float fs, int ft) {
    if (lane < p.n_w) {
        const int fd = info[UI_FIRST_D], ndm = info[UI_N_D];
        const int16_t t16 = static_cast<int16_t>(ft == INT_MAX ? -1 : ft);
        for (int d = fd; d < fd + ndm; ++d) {
            const int64_t o = (pix * p.n_dm + d) * p.n_w + lane;
            p.full_snr[o] = fs;
            p.full_t[o] = t16;
        }
    }
}

// The search of one warp over the distinct DM rows [u_lo, u_hi) of one pixel whose
// subband rows are in xs (pitch Tp, -inf beyond the window): de-dispersion by row
// differences, prefix sums, the boxcars of every width class, the warp arg-max and,
// when a row improves the warp's best, the earliest sample reaching it (re-evaluated
// with the same operations).  FULL also writes every (DM, width) result of the rows.
// Returns the warp's best (snr, distinct row u, width index, t) on every lane.
template <int C, bool FULL, typename OnRead = NoReadDone>
__device__ __forceinline__ PixRec search_rows(const SearchParams &p, const float *xs, float *Pw, const float *s_inv,
                                              const int32_t *s_info, const int32_t *s_delta,
                                              const int32_t *s_shift, int u_lo, int u_hi, int64_t pix,
                                              int lane, OnRead on_read = OnRead{}) {
    constexpr int SH = (C < kSmallMax) ? C : kSmallMax;
    const int n_sub = p.n_sub, n_t = p.n_t, Tp = p.Tp;
    const int t0 = lane * C;
    float bsnr = neg_inf();
    int bu = -1, bwi = -1, bt = -1;
    float D[C];
    if (u_lo >= u_hi) on_read();
#pragma unroll 1
    for (int u = u_lo; u < u_hi; ++u) {
        const int32_t *info = s_info + u * kInfo;
        if (u == u_lo) {
#pragma unroll
            for (int c = 0; c < C; ++c) D[c] = 0.0f;
            const int32_t *sh = s_shift + u * n_sub;
#pragma unroll 1
            for (int k = 0; k < n_sub; ++k) {
                const float *xr = xs + (size_t)k * Tp + t0 + sh[k];
#pragma unroll
                for (int c = 0; c < C; ++c) D[c] += xr[c];
            }
        } else {
            const int d0 = info[UI_DOFF], nd = info[UI_ND];
#pragma unroll 1
            for (int e = d0; e < d0 + nd; ++e) {
                const uint32_t pk = static_cast<uint32_t>(s_delta[e]);
                const int k = pk & 63u, so = (pk >> 6) & 0x1fffu, sn = pk >> 19;
                const float *xo = xs + (size_t)k * Tp + t0 + so;
                const float *xn = xs + (size_t)k * Tp + t0 + sn;
#pragma unroll
                for (int c = 0; c < C; ++c) D[c] = (D[c] + xn[c]) - xo[c];
            }
        }
        if (u == u_hi - 1) on_read();
        const int L = n_t - info[UI_SMAX];

        // in-lane prefix, warp scan of lane totals, P to shared memory
        const bool masked = p.new_blk > 0;
        float ls = neg_inf();
        int lw = -1;
        auto consider = [&](int wi, float m) {
            const float s = m * s_inv[wi];
            if (s > ls || (s == ls && wi < lw)) {
                ls = s;
                lw = wi;
            }
        };
        // FULL mode: the S/N of (row u, width wi) reduced over the warp, and its TOA, kept on lane wi
        float fs = neg_inf();
        int ft = INT_MAX;
        auto write_full = [&](int wi, float s, int t) {
            if (lane == wi) {
                fs = s;
                ft = t;
            }
        };
        {
            float Lp[C + 1];
            const float tot = lane_prefix<C>(D, Lp);
            float inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float y = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc += y;
            }
            float carry = __shfl_up_sync(kFull, inc, 1);
            if (lane == 0) carry = 0.0f;
#pragma unroll
            for (int c = 0; c < C; ++c) Pw[t0 + c] = carry + Lp[c];
            if (!masked && p.has_small) {
                // power-of-two widths <= min(C, 16): in-lane, compile-time unrolled and
                // branch-free (absent widths are computed and masked); ascending width
                // order with a strict '>' keeps the smallest width index on ties
                float H[SH + 1];
                lane_halo<C, SH>(Lp, tot, lane, H);
#define NSFRB_SMALL_J(J)                                                                                   \
    if constexpr (pow2_class(C, J) == WC_SMALL) {                                                         \
const int wi = p.pow2_wi[J];                                                                       \
const float m = small_max_w<C, SH, (1 << J)>(Lp, H);                                              \
const float s = (wi >= 0) ? m * s_inv[wi < 0 ? 0 : wi] : neg_inf();                              \
if (s > ls) {                                                                                      \
    ls = s;                                                                                        \
    lw = wi;                                                                                       \
}                                                                                                  \
if constexpr (FULL) {                                                                              \
    if (wi >= 0) {                                                                                 \
        const float mw = warp_max(m), sw = mw * s_inv[wi];                                        \
        int t = INT_MAX;                                                                           \
        if (mw != neg_inf()) t = warp_min(small_find_w<C, SH, (1 << J)>(Lp, H, s_inv[wi], sw, t0)); \
        write_full(wi, sw, t);                                                                     \
    }                                                                                              \
}                                                                                                  \
    }
                NSFRB_POW2(NSFRB_SMALL_J)
#undef NSFRB_SMALL_J
            }
        }
        __syncwarp();
        if (!masked && p.has_large) {
            // power-of-two widths 32 * M with M < C: lane-strided, compile-time unrolled
            float Ps[C];
#pragma unroll
            for (int i = 0; i < C; ++i) Ps[i] = Pw[32 * i + lane];
#define NSFRB_LARGE_J(J)                                                                                   \
    if constexpr (pow2_class(C, J) == WC_LARGE) {                                                         \
const int wi = p.pow2_wi[J];                                                                       \
const float m = large_max_m<C, ((1 << J) >> 5)>(Ps);                                              \
const float s = (wi >= 0) ? m * s_inv[wi < 0 ? 0 : wi] : neg_inf();                              \
if (s > ls) {                                                                                      \
    ls = s;                                                                                        \
    lw = wi;                                                                                       \
}                                                                                                  \
if constexpr (FULL) {                                                                              \
    if (wi >= 0) {                                                                                 \
        const float mw = warp_max(m), sw = mw * s_inv[wi];                                        \
        int t = INT_MAX;                                                                           \
        if (mw != neg_inf()) t = warp_min(large_find_m<C, ((1 << J) >> 5)>(Ps, s_inv[wi], sw, lane)); \
        write_full(wi, sw, t);                                                                     \
    }                                                                                              \
}                                                                                                  \
    }
            NSFRB_POW2(NSFRB_LARGE_J)
#undef NSFRB_LARGE_J
        }
        // every other width (and every width of a masked search) from shared memory
        const int n_gen = masked ? p.n_w : p.n_gen;
#pragma unroll 1
        for (int g = 0; g < n_gen; ++g) {
            const int wi = masked ? g : p.gen_wi[g];
            const int w = p.widths[wi];
            const int tl = masked ? max(0, L - w - p.new_blk + 1) : 0;
            const float m = generic_max(Pw, w, L, tl, lane);
            consider(wi, m);
            if constexpr (FULL) {
                const float mw = warp_max(m), sw = mw * s_inv[wi];
                int t = INT_MAX;
                if (mw != neg_inf()) t = warp_min(generic_find(Pw, w, L, tl, lane, s_inv[wi], sw));
                write_full(wi, sw, t);
            }
        }
        if constexpr (FULL) full_store_row(p, info, pix, lane, fs, ft);

        // warp arg-max over (S/N, width index)
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
            // earliest sample reaching this S/N, re-evaluated exactly as above
            // (the prefix and halo are rebuilt from D: same operations, same values)
            const int w = p.widths[lw];
            const float inv = s_inv[lw];
            int t;
            if (masked || p.wclass[lw] == WC_GENERIC) {
                const int tl = masked ? max(0, L - w - p.new_blk + 1) : 0;
                t = generic_find(Pw, w, L, tl, lane, inv, ls);
            } else if (p.wclass[lw] == WC_SMALL) {
                float Lp[C + 1];
                float H[SH + 1];
                const float tot = lane_prefix<C>(D, Lp);
                lane_halo<C, SH>(Lp, tot, lane, H);
                t = small_find<C, SH>(w, Lp, H, inv, ls, t0);
            } else {
                float Ps[C];
#pragma unroll
                for (int i = 0; i < C; ++i) Ps[i] = Pw[32 * i + lane];
                t = large_find<C>(w >> 5, Ps, inv, ls, lane);
            }
            t = warp_min(t);
            bsnr = ls;
            bu = u;
            bwi = lw;
            bt = t;
        }
        __syncwarp();
    }
    return PixRec{bsnr, bu, bwi, bt};
}

// Warp sum scan of the lane totals: the prefix P at this lane's first sample.
__device__ __forceinline__ float lane_carry(float tot, int lane) {
    float inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    float carry = __shfl_up_sync(kFull, inc, 1);
    return (lane == 0) ? 0.0f : carry;
}

// Earliest-sample searches for even chunks, by the whole warp on the trials of the lanes that hold
// the target (match: their bits; found from the lanes' own maxima), with the operations of the
// maximum pass; the result is the same on every lane.

// In-lane width W (lane j's trials are samples j C .. j C + C - 1, lanes in sample order): the
// lowest matching lane's extended prefix (D for W = 1) goes to the warp's scratch, and its C trials
// are evaluated 32 at a time.
template <int C, int SH, int W>
__device__ __forceinline__ int small_find_coop(const float2 (&D)[C / 2], const float2 (&Lp)[C / 2],
                                               const float2 (&Hh)[SH / 2], float *scr, unsigned match, int lane,
                                               float inv, float target) {
    static_assert(C + SH <= kFindScr, "scratch holds a lane's extended prefix");
    const int src = __ffs(match) - 1;
    __syncwarp();
    if (lane == src) {
        float2 *s2 = reinterpret_cast<float2 *>(scr);
        if constexpr (W == 1) {
#pragma unroll
            for (int m = 0; m < C / 2; ++m) s2[m] = D[m];
        } else {
#pragma unroll
            for (int m = 0; m < C / 2; ++m) s2[m] = Lp[m];
#pragma unroll
            for (int m = 0; m < SH / 2; ++m) s2[C / 2 + m] = Hh[m];
        }
    }
    __syncwarp();
    int found = INT_MAX;
#pragma unroll
    for (int c0 = 0; c0 < C; c0 += 32) {
        const int c = c0 + lane;
        bool hit = false;
        if (c < C) {
            const float b = (W == 1) ? scr[c] : scr[c + W] - scr[c];
            hit = b * inv == target;
        }
        const unsigned bal = __ballot_sync(kFull, hit);
        if (bal && found == INT_MAX) found = src * C + c0 + __ffs(bal) - 1;
    }
    return found;
}

template <int C, int SH>
__device__ __forceinline__ int small_find_coop_w(int w, const float2 (&D)[C / 2], const float2 (&Lp)[C / 2],
                                                 const float2 (&Hh)[SH / 2], float *scr, unsigned match, int lane,
                                                 float inv, float target) {
    switch (w) {
        case 1: return small_find_coop<C, SH, 1>(D, Lp, Hh, scr, match, lane, inv, target);
        case 2: if constexpr (2 <= SH) return small_find_coop<C, SH, 2>(D, Lp, Hh, scr, match, lane, inv, target); break;
        case 4: if constexpr (4 <= SH) return small_find_coop<C, SH, 4>(D, Lp, Hh, scr, match, lane, inv, target); break;
        case 8: if constexpr (8 <= SH) return small_find_coop<C, SH, 8>(D, Lp, Hh, scr, match, lane, inv, target); break;
        case 16: if constexpr (16 <= SH) return small_find_coop<C, SH, 16>(D, Lp, Hh, scr, match, lane, inv, target); break;
        default: break;
    }
    return INT_MAX;
}

// Lane-strided width 32 M (lane j's trials are samples 32 i + j, i < C - M, from P in shared
// memory): each matching lane's trials evaluated by the warp, the earliest over the lanes kept.
template <int C>
__device__ __forceinline__ int large_find_coop(const float *Pw, int M, unsigned match, int lane, float inv,
                                               float target) {
    int best = INT_MAX;
    while (match) {
        const int j = __ffs(match) - 1;
        match &= match - 1;
        int found = INT_MAX;
#pragma unroll
        for (int k0 = 0; k0 < C; k0 += 32) {
            const int k = k0 + lane;
            const bool hit = k < C - M && (Pw[32 * (k + M) + j] - Pw[32 * k + j]) * inv == target;
            const unsigned bal = __ballot_sync(kFull, hit);
            if (bal && found == INT_MAX) found = 32 * (k0 + __ffs(bal) - 1) + j;
        }
        best = min(best, found);
    }
    return best;
}

// Even chunks: the earliest sample whose boxcar of width index wi reaches `target`, from the
// row's D (in-lane widths) or its P in shared memory (lane-strided and generic widths),
// evaluated with the operations of the maximum pass; match: the lanes whose own best is
// (target, wi).  The same on every lane.
template <int C>
__device__ __forceinline__ int find_t_even(const SearchParams &p, const float2 (&D)[C / 2], const float *Pw, int wi,
                                           float inv, float target, int L, int lane, bool masked, unsigned match,
                                           float *scr) {
    constexpr int SH = (C < kSmallMax) ? C : kSmallMax;
    const int w = p.widths[wi];
    if (masked && p.new_blk <= 32)
        return warp_min(masked_find32(Pw, w, masked_end(L, p.new_blk, lane), inv, target));
    if (masked || p.wclass[wi] == WC_GENERIC) {
        const int tl = masked ? max(0, L - w - p.new_blk + 1) : 0;
        return warp_min(generic_find(Pw, w, L, tl, lane, inv, target));
    }
    if (p.wclass[wi] == WC_SMALL) {
        float2 Lp[C / 2];
        float2 Hh[SH / 2];
        const float tot = prefix_pairs<C>(D, Lp);
        halo_pairs<C, SH>(Lp, tot, Hh);
        return small_find_coop_w<C, SH>(w, D, Lp, Hh, scr, match, lane, inv, target);
    }
    return large_find_coop<C>(Pw, w >> 5, match, lane, inv, target);
}

// search_rows for even chunks (sample pairs, see above).  The pixel's rows are in storage ST
// (0 FP32, 1 BF16, 2 FP16) with the window at element eoff of each row; with mask_tail the
// elements past the window are not -inf and the de-dispersed samples past L are set to -inf.
template <int C, bool FULL, int ST = 0, typename OnRead = NoReadDone>
__device__ __forceinline__ PixRec search_rows_even(const SearchParams &p, const void *xs, float *Pw, float *Sw,
                                                   const float *s_inv, const int32_t *s_info,
                                                   const int32_t *s_delta, const int32_t *s_shift, int u_lo,
                                                   int u_hi, int64_t pix, int lane, int eoff = 0,
                                                   bool mask_tail = false, OnRead on_read = OnRead{}) {
    static_assert(C % 2 == 0, "even chunks only");
    constexpr int SH = (C < kSmallMax) ? C : kSmallMax;
    const int n_sub = p.n_sub, n_t = p.n_t, Tp = p.Tp;
    const int t0 = lane * C;
    const int te = t0 + eoff;
    const bool masked = p.new_blk > 0;
    float bsnr = neg_inf();
    int bu = -1, bwi = -1, bt = -1;
    float2 D[C / 2];
    if (u_lo >= u_hi) on_read();
#pragma unroll 1
    for (int u = u_lo; u < u_hi; ++u) {
        const int32_t *info = s_info + u * kInfo;
        if (u == u_lo)
            dd_first<C, ST>(D, xs, Tp, n_sub, s_shift + u * n_sub, te);
        else
            dd_delta<C, ST>(D, xs, Tp, s_delta, info[UI_DOFF], info[UI_ND], te);
        if (u == u_hi - 1) on_read();
        const int L = n_t - info[UI_SMAX];
        // (a masked search reads P only up to P[L], which needs no sample past L)
        if (mask_tail && !masked) {
#pragma unroll
            for (int m = 0; m < C / 2; ++m) {
                if (t0 + 2 * m >= L) D[m].x = neg_inf();
                if (t0 + 2 * m + 1 >= L) D[m].y = neg_inf();
            }
        }

        float ls = neg_inf();
        int lw = -1;
        // FULL mode: (row u, width wi) reduced over the warp, kept on lane wi
        float fs = neg_inf();
        int ft = INT_MAX;
        auto write_full = [&](int wi, float s, int t) {
            if (lane == wi) {
                fs = s;
                ft = t;
            }
        };
        {
            float2 Lp[C / 2];
            const float tot = prefix_pairs<C>(D, Lp);
            if (!masked && p.has_small) {
                // power-of-two widths <= min(C, 16) in-lane; ascending width order with a
                // strict '>' keeps the smallest width index on ties.  The warp scan of the lane
                // totals and the store of P sit in the same block, so that the scan's shuffle
                // chain overlaps the in-lane widths, which do not need it.
                float2 Hh[SH / 2];
                halo_pairs<C, SH>(Lp, tot, Hh);
                const float carry = lane_carry(tot, lane);
#define NSFRB_SMALL_PK(J)                                                                                 \
    if constexpr (pow2_class(C, J) == WC_SMALL) {                                                        \
        const int wi = p.pow2_wi[J];                                                                      \
        const float m = small_max_pk<C, SH, (1 << J)>(D, Lp, Hh);                                        \
        const float s = (wi >= 0) ? m * s_inv[wi < 0 ? 0 : wi] : neg_inf();                             \
        if (s > ls) {                                                                                     \
            ls = s;                                                                                       \
            lw = wi;                                                                                      \
        }                                                                                                 \
        if constexpr (FULL) {                                                                             \
            if (wi >= 0) {                                                                                \
                const float mw = warp_max(m), sw = mw * s_inv[wi];                                       \
                int t = INT_MAX;                                                                          \
                if (mw != neg_inf())                                                                      \
                    t = small_find_coop<C, SH, (1 << J)>(D, Lp, Hh, Sw, __ballot_sync(kFull, m * s_inv[wi] == sw), \
                                                         lane, s_inv[wi], sw);                                   \
                write_full(wi, sw, t);                                                                    \
            }                                                                                             \
        }                                                                                                 \
    }
                NSFRB_SMALL_PK(0) NSFRB_SMALL_PK(1) NSFRB_SMALL_PK(2) NSFRB_SMALL_PK(3) NSFRB_SMALL_PK(4)
#undef NSFRB_SMALL_PK
                store_p<C>(Pw, t0, carry, Lp);
            } else {
                store_p<C>(Pw, t0, lane_carry(tot, lane), Lp);
            }
        }
        __syncwarp();
        if (!masked && p.has_large) {
            float2 Ps[C / 2];
            load_ps<C>(Pw, lane, Ps);
#define NSFRB_LARGE_PK(J)                                                                                 \
    if constexpr (pow2_class(C, J) == WC_LARGE) {                                                        \
        const int wi = p.pow2_wi[J];                                                                      \
        const float m = large_max_pk<C, ((1 << J) >> 5)>(Ps);                                            \
        const float s = (wi >= 0) ? m * s_inv[wi < 0 ? 0 : wi] : neg_inf();                             \
        if (s > ls) {                                                                                     \
            ls = s;                                                                                       \
            lw = wi;                                                                                      \
        }                                                                                                 \
        if constexpr (FULL) {                                                                             \
            if (wi >= 0) {                                                                                \
                const float mw = warp_max(m), sw = mw * s_inv[wi];                                       \
                int t = INT_MAX;                                                                          \
                if (mw != neg_inf())                                                                      \
                    t = large_find_coop<C>(Pw, (1 << J) >> 5, __ballot_sync(kFull, m * s_inv[wi] == sw), lane, \
                                           s_inv[wi], sw);                                                       \
                write_full(wi, sw, t);                                                                    \
            }                                                                                             \
        }                                                                                                 \
    }
            NSFRB_POW2(NSFRB_LARGE_PK)
#undef NSFRB_LARGE_PK
        }
        if (masked && p.new_blk <= 32) {
            // serving: every width's trials that end in the newest block, one per lane, all ending at
            // this lane's P index e; ascending width order with a strict '>' keeps the smallest width
            // index on ties
            const int e = masked_end(L, p.new_blk, lane);
            const float pe = Pw[e >= 0 ? e : 0];
#pragma unroll 4
            for (int wi = 0; wi < p.n_w; ++wi) {
                const int t = e - p.widths[wi];
                const bool ok = e >= 0 && t >= 0;
                const float b = pe - Pw[ok ? t : 0];
                const float s = ok ? b * s_inv[wi] : neg_inf();
                if (s > ls) {
                    ls = s;
                    lw = wi;
                }
            }
        }
        // every other width (and every width of a masked search of longer blocks) from shared memory
        const int n_gen = masked ? (p.new_blk <= 32 ? 0 : p.n_w) : p.n_gen;
#pragma unroll 1
        for (int g = 0; g < n_gen; ++g) {
            const int wi = masked ? g : p.gen_wi[g];
            const int w = p.widths[wi];
            const int tl = masked ? max(0, L - w - p.new_blk + 1) : 0;
            const float m = generic_max(Pw, w, L, tl, lane);
            const float s = m * s_inv[wi];
            if (s > ls || (s == ls && wi < lw)) {
                ls = s;
                lw = wi;
            }
            if constexpr (FULL) {
                const float mw = warp_max(m), sw = mw * s_inv[wi];
                int t = INT_MAX;
                if (mw != neg_inf()) t = warp_min(generic_find(Pw, w, L, tl, lane, s_inv[wi], sw));
                write_full(wi, sw, t);
            }
        }
        if constexpr (FULL) full_store_row(p, info, pix, lane, fs, ft);

        // warp arg-max over (S/N, width index), only when some lane beats the warp's best
        if (__any_sync(kFull, ls > bsnr)) {
            const float ls_own = ls;
            const int lw_own = lw;
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
                // earliest sample reaching this S/N, re-evaluated with the same operations on the
                // lanes whose own best it is
                const unsigned match = __ballot_sync(kFull, ls_own == ls && lw_own == lw);
                const int t = find_t_even<C>(p, D, Pw, lw, s_inv[lw], ls, L, lane, masked, match, Sw);
                bsnr = ls;
                bu = u;
                bwi = lw;
                bt = t;
            }
        }
        __syncwarp();
    }
    return PixRec{bsnr, bu, bwi, bt};
}

// Per-warp row search for chunk size C (pairs for even C).  Odd chunks read FP32 rows only.
template <int C, bool FULL, int ST = 0, typename OnRead = NoReadDone>
__device__ __forceinline__ PixRec search_rows_any(const SearchParams &p, const void *xs, float *Pw, float *Sw,
                                                  const float *s_inv,
                                                  const int32_t *s_info, const int32_t *s_delta,
                                                  const int32_t *s_shift, int u_lo, int u_hi, int64_t pix,
                                                  int lane, int eoff = 0, bool mask_tail = false,
                                                  OnRead on_read = OnRead{}) {
    if constexpr (C % 2 == 0) {
        return search_rows_even<C, FULL, ST, OnRead>(p, xs, Pw, Sw, s_inv, s_info, s_delta, s_shift, u_lo, u_hi, pix,
                                                     lane, eoff, mask_tail, on_read);
    } else {
        static_assert(ST == 0, "odd chunks read FP32 rows");
        return search_rows<C, FULL, OnRead>(p, static_cast<const float *>(xs) + eoff, Pw, s_inv, s_info, s_delta,
                                            s_shift, u_lo, u_hi, pix, lane, on_read);
    }
}

// ------------------------------------------------------------------ the kernel

// FULL mode: -inf S/N and TOA -1 for every (DM, width) of the distinct rows [u0, u1) of a pixel
// (rows whose delays leave no sample, or every row of a pixel without a noise scale); one warp.
__device__ __forceinline__ void full_fill_empty(const SearchParams &p, const int32_t *s_info, int u0, int u1,
                                                int64_t pix, int lane) {
    for (int u = u0; u < u1; ++u) {
        const int32_t *info = s_info + u * kInfo;
        const int fd = info[UI_FIRST_D], ndm = info[UI_N_D];
        for (int i = lane; i < ndm * p.n_w; i += 32) {
            const int64_t o = (pix * p.n_dm + fd) * p.n_w + i;
            p.full_snr[o] = neg_inf();
            p.full_t[o] = -1;
        }
    }
}

template <int C, bool FULL>
__global__ void __launch_bounds__(kThreads, 1) search_kernel(const __grid_constant__ SearchParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const SmemLayout lay = smem_layout(p, C);
    int32_t *s_table = reinterpret_cast<int32_t *>(smem + lay.table);
    float *s_xs = reinterpret_cast<float *>(smem + lay.xs);
    unsigned char *s_stg = smem + lay.stg;
    float *s_pbuf = reinterpret_cast<float *>(smem + lay.pbuf);
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem + lay.hist);
    PixRec *s_wbest = reinterpret_cast<PixRec *>(smem + lay.wbest);
    float *s_inv = reinterpret_cast<float *>(smem + lay.sinv);
    int32_t *s_flag = reinterpret_cast<int32_t *>(smem + lay.sinv + sizeof(float) * kMaxW);
    unsigned long long *s_bar = reinterpret_cast<unsigned long long *>(smem + lay.bar);

    const int tid = threadIdx.x;
    const int t_off = p.t_off_dev ? *p.t_off_dev : p.t_off;
    const int stg_off = t_off & 7;   // 16-bit element offset of the window in an aligned staged row
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int n_sub = p.n_sub, n_t = p.n_t, Tp = p.Tp;

    // ---- tables to shared memory
    const int table_words = p.n_u * kInfo + p.n_deltas + p.n_u * n_sub;
    for (int i = tid; i < table_words; i += kThreads) s_table[i] = p.table[i];
    const int32_t *s_info = s_table;
    const int32_t *s_delta = s_table + p.n_u * kInfo;
    const int32_t *s_shift = s_delta + p.n_deltas;

    // ---- -inf beyond the window in every staged row (never overwritten)
    const int nbuf = (p.stage == 1) ? 2 : 1;
    for (int b = 0; b < nbuf; ++b)
        for (int i = tid; i < n_sub * (Tp - n_t); i += kThreads) {
            const int k = i / (Tp - n_t), t = n_t + i % (Tp - n_t);
            s_xs[(size_t)b * n_sub * Tp + (size_t)k * Tp + t] = neg_inf();
        }
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        s_flag[0] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    __syncthreads();

    int64_t n_items = p.n_items;
    if (p.n_items_dev) n_items = *p.n_items_dev;

    auto item_pixel = [&](int64_t it) -> int64_t {
        return p.pix_list ? static_cast<int64_t>(p.pix_list[it]) : p.pix0 + it;
    };
    // issue the bulk copies of one pixel into buffer b (thread 0 only)
    auto issue = [&](int64_t it, int b) {
        const int64_t pix = item_pixel(it);
        const int64_t row0 = (pix - p.cube_pix0) * n_sub;
        if (p.stage == 1) {
            const float *src = static_cast<const float *>(p.cube);
            float *dst = s_xs + (size_t)b * n_sub * Tp;
            mbar_expect_tx(&s_bar[b], static_cast<uint32_t>(n_sub * n_t * 4));
            for (int k = 0; k < n_sub; ++k)
                bulk_g2s(dst + (size_t)k * Tp, src + (row0 + k) * p.row_len + t_off,
                         static_cast<uint32_t>(n_t * 4), &s_bar[b]);
        } else {
            const unsigned char *src = static_cast<const unsigned char *>(p.cube);
            unsigned char *dst = s_stg + (size_t)b * n_sub * p.stg_pitch;
            const int64_t first = static_cast<int64_t>(t_off - stg_off) * 2;   // 16-byte aligned
            const uint32_t bytes = static_cast<uint32_t>(align_up((size_t)(stg_off + n_t) * 2, 16));
            mbar_expect_tx(&s_bar[b], bytes * n_sub);
            for (int k = 0; k < n_sub; ++k)
                bulk_g2s(dst + (size_t)k * p.stg_pitch, src + (row0 + k) * p.row_len * 2 + first, bytes,
                         &s_bar[b]);
        }
    };

    const int n_ua = p.n_u_active;
    const int u_lo = (warp * n_ua) / kWarps;
    const int u_hi = ((warp + 1) * n_ua) / kWarps;
    float *Pw = s_pbuf + (size_t)warp * 32 * C;
    float *Sw = reinterpret_cast<float *>(smem + lay.fscr) + (size_t)warp * kFindScr;

    uint32_t phase[2] = {0u, 0u};
    if (p.stage != 0 && tid == 0 && blockIdx.x < n_items) issue(blockIdx.x, 0);

    int iter = 0;
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x, ++iter) {
        const int b = (p.stage == 1) ? (iter & 1) : 0;
        const int sb = iter & 1;   // staging / barrier buffer of this item
        const int64_t pix = item_pixel(it);
        const int64_t nxt = it + gridDim.x;
        // prefetch the next item into the other buffer (free since the end of the previous item)
        if (p.stage != 0 && tid == 0 && nxt < n_items) issue(nxt, sb ^ 1);

        float *xs = s_xs + (size_t)b * n_sub * Tp;
        if (p.stage == 0) {
            const int64_t row0 = (pix - p.cube_pix0) * n_sub;
            for (int i = tid; i < n_sub * n_t; i += kThreads) {
                const int k = i / n_t, t = i - k * n_t;
                int tt = t_off + t;
                if (p.t_wrap > 0 && tt >= p.t_wrap) tt -= p.t_wrap;
                const int64_t at = p.t_stride > 0 ? (static_cast<int64_t>(tt) * n_sub + k) * p.t_stride + pix
                                                  : (row0 + k) * p.row_len + tt;
                xs[(size_t)k * Tp + t] = load_elem(p.cube, at, p.dtype);
            }
        } else {
            const bool ok = mbar_wait(&s_bar[sb], phase[sb]);
            phase[sb] ^= 1u;
            if (!ok) atomicOr(&s_flag[0], ERR_WAIT_TIMEOUT);
            if (p.stage == 2) {
                const unsigned char *stg_b = s_stg + (size_t)sb * n_sub * p.stg_pitch;
                if (stg_off == 0 && (n_t & 7) == 0) {
                    // 8 samples per 16-byte word -> two float4 stores
                    const int nv = n_t >> 3;
                    for (int i = tid; i < n_sub * nv; i += kThreads) {
                        const int k = i / nv, v = i - k * nv;
                        const uint4 raw = *reinterpret_cast<const uint4 *>(stg_b + (size_t)k * p.stg_pitch + 16 * v);
                        float4 a, c;
                        if (p.dtype == 1) {
                            a = make_float4(__uint_as_float(raw.x << 16), __uint_as_float(raw.x & 0xffff0000u),
                                            __uint_as_float(raw.y << 16), __uint_as_float(raw.y & 0xffff0000u));
                            c = make_float4(__uint_as_float(raw.z << 16), __uint_as_float(raw.z & 0xffff0000u),
                                            __uint_as_float(raw.w << 16), __uint_as_float(raw.w & 0xffff0000u));
                        } else {
                            const float2 h0 = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
                            const float2 h1 = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
                            const float2 h2 = __half22float2(*reinterpret_cast<const __half2 *>(&raw.z));
                            const float2 h3 = __half22float2(*reinterpret_cast<const __half2 *>(&raw.w));
                            a = make_float4(h0.x, h0.y, h1.x, h1.y);
                            c = make_float4(h2.x, h2.y, h3.x, h3.y);
                        }
                        float4 *dst = reinterpret_cast<float4 *>(xs + (size_t)k * Tp + 8 * v);
                        dst[0] = a;
                        dst[1] = c;
                    }
                } else {
                    // any window offset: pairs of 16-bit samples from the staged 32-bit words,
                    // realigned by a byte permute when the offset is odd (Tp is a multiple of 4)
                    const uint32_t *w32 = reinterpret_cast<const uint32_t *>(stg_b);
                    const int wpitch = p.stg_pitch / 4, w0 = stg_off >> 1, odd = stg_off & 1;
                    const int npair = n_t >> 1;
                    for (int k = 0; k < n_sub; ++k) {
                        const uint32_t *row = w32 + (size_t)k * wpitch + w0;
                        float *dst = xs + (size_t)k * Tp;
                        for (int q = tid; q < npair; q += kThreads) {
                            const uint32_t u = odd ? __byte_perm(row[q], row[q + 1], 0x5432) : row[q];
                            float2 v;
                            if (p.dtype == 1) {
                                v = make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
                            } else {
                                v = __half22float2(*reinterpret_cast<const __half2 *>(&u));
                            }
                            *reinterpret_cast<float2 *>(dst + 2 * q) = v;
                        }
                        if ((n_t & 1) && tid == 0) {
                            const unsigned short *h = reinterpret_cast<const unsigned short *>(stg_b);
                            dst[n_t - 1] = widen16(h[(size_t)k * (p.stg_pitch / 2) + stg_off + n_t - 1], p.dtype);
                        }
                    }
                }
            }
        }
        if (tid < p.n_w) {
            const float sg = (p.sigma && p.noise_mode == 0) ? p.sigma[pix] : p.sigma_default;
            s_inv[tid] = 1.0f / (sg * sqrtf(static_cast<float>(p.widths[tid])));
        }
        __syncthreads();
        if (s_flag[0] & ERR_WAIT_TIMEOUT) {
            // a bulk copy did not complete in time: record and stop this CTA
            if (tid == 0) atomicOr(p.err, ERR_WAIT_TIMEOUT);
            // wait (bounded) for the copies still in flight before leaving
            if (tid == 0 && p.stage != 0 && nxt < n_items) mbar_wait(&s_bar[sb ^ 1], phase[sb ^ 1]);
            return;
        }

        // ---- robust normalisation per (pixel, subband) row (MAD mode)
        bool bad_pixel = false;
        if (p.noise_mode == 1) {
            uint32_t *hist = (p.stage == 2 ? reinterpret_cast<uint32_t *>(s_stg + (size_t)sb * n_sub * p.stg_pitch)
                                           : s_hist) + warp * kHistBins;
            for (int k = warp; k < n_sub; k += kWarps) {
                float *row = xs + (size_t)k * Tp;
                const float med = warp_median(row, n_t, hist, p.dtype == 1);
                for (int t = lane; t < n_t; t += 32) Pw[t] = fabsf(row[t] - med);
                __syncwarp();
                const float mad = warp_median(Pw, n_t, hist, false);
                if (mad == 0.0f) {
                    if (lane == 0) atomicOr(&s_flag[0], ERR_ZERO_MAD);
                } else {
                    const float inv = 1.0f / (1.4826f * mad);
                    for (int t = lane; t < n_t; t += 32) row[t] = (row[t] - med) * inv;
                }
                __syncwarp();
            }
            __syncthreads();
            bad_pixel = (s_flag[0] & ERR_ZERO_MAD) != 0;
        }

        // ---- per-warp search over its rows
        PixRec wr{neg_inf(), -1, -1, -1};
        if (!bad_pixel)
            wr = search_rows_any<C, FULL, 0>(p, xs, Pw, Sw, s_inv, s_info, s_delta, s_shift, u_lo, u_hi, pix, lane);
        const float bsnr = wr.snr;
        const int bu = wr.dm_idx, bwi = wr.w_idx, bt = wr.t_idx;
        // FULL mode: DM rows that have no trial at all
        if (p.full_snr && warp == 0) full_fill_empty(p, s_info, bad_pixel ? 0 : n_ua, p.n_u, pix, lane);
        if (lane == 0) s_wbest[warp] = PixRec{bsnr, bu, bwi, bt};
        __syncthreads();
        if (tid == 0) {
            PixRec best{neg_inf(), -1, -1, -1};
            for (int w = 0; w < kWarps; ++w)
                if (s_wbest[w].snr > best.snr) best = s_wbest[w];
            if (best.dm_idx >= 0) best.dm_idx = s_info[best.dm_idx * kInfo + UI_FIRST_D];
            if (bad_pixel) {
                best = PixRec{neg_inf(), -1, -1, -1};
                atomicOr(p.err, ERR_ZERO_MAD);
                s_flag[0] &= ~ERR_ZERO_MAD;
            }
            p.rec[pix] = best;
        }
        // all reads of this item's buffers are done before they are refilled
        fence_proxy_async();
        __syncthreads();
    }
}


// ------------------------------------------------------------------ barrier-free kernel

// Same search (rows bulk-copied straight into a double buffer, KNOWN noise; per-pixel records, and
// with FULL every (DM, width) result of the pixel) without CTA barriers between pixels.  The CTA's warps form TEAMS teams of W = kWarps / TEAMS warps;
// each team walks its own pixels (items team, team + TEAMS * grid, ... of the CTA) with its own
// double buffer, so a pixel's distinct DM rows are split into W groups (fewer teams: more groups,
// each built from scratch; more teams: more pixels in shared memory).  Within a team every warp
// walks the team's pixels on its own; on the team's i-th pixel warp w takes row group (w + i) mod W,
// so the groups with one row more rotate over the warps.  A warp publishes its group's best and
// counts itself done; the last warp of a pixel combines the groups in row order (the DM tie rule),
// writes the pixel's record, and starts the copy of the team's pixel two ahead into the buffer it
// frees (with that pixel's 1 / (sigma sqrt(w))).  Warps of a team drift apart by at most one pixel.
// With NB = 1 buffer per team (tiles too large for two buffers per team) the copy of the team's
// next pixel starts when the pixel is done, or, for FP32 rows (copies of twice the bytes), as soon
// as every warp of the team has read the pixel's rows for the last time (after the de-dispersion
// of its last row), while the team still runs the boxcars of those rows.  (Measured on the
// full-window workload: 6.82 -> 6.62 ms for FP32 rows, but 5.58 -> 6.06 ms for BF16 rows, which
// keep the copy at the end of the pixel.)  A pixel's records and 1 / (sigma sqrt(w)) live in one
// of two record slots per team, alternating by pixel; its rows in the buffer.
// ST is the storage type of the rows, kept as they are in shared memory: FP32, or BF16 / FP16 read
// in place by the mixed-precision adds (no widening pass).  A window that starts at any sample t_off
// is copied from the 16-byte boundary below it and read from element eoff = t_off mod (16 / size)
// of the staged row; when the copy then carries samples past the window, the de-dispersed samples
// past the valid range are set to -inf instead of relying on -inf past the window.
template <int C, int ST, int TEAMS, int NB, bool FULL>
__global__ void __launch_bounds__(kThreads, 1) search_kernel_pipe(const __grid_constant__ SearchParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int kEs = (ST == 0) ? 4 : 2;          // bytes per stored sample
    constexpr int kEpv = 16 / kEs;                  // samples per 16 bytes
    constexpr int W = kWarps / TEAMS;               // warps (and row groups) per team
    constexpr bool kEarly = NB == 1 && ST == 0;     // next copy started once the rows are read
    static_assert(kWarps % TEAMS == 0, "teams divide the warps");
    const SmemLayout lay = smem_layout(p, C);
    int32_t *s_table = reinterpret_cast<int32_t *>(smem + lay.table);
    unsigned char *s_xs = smem + lay.xs;
    float *s_pbuf = reinterpret_cast<float *>(smem + lay.pbuf);
    PixRec *s_wbest = reinterpret_cast<PixRec *>(smem + lay.wbest);        // [TEAMS][2][kWarps]
    float *s_inv = reinterpret_cast<float *>(smem + lay.sinv);             // [TEAMS][2][kMaxW]
    int32_t *s_cnt = reinterpret_cast<int32_t *>(smem + lay.sinv + sizeof(float) * kMaxW * 2 * TEAMS);
    int32_t *s_flag = s_cnt + 2 * TEAMS;    // error seen by a warp
    int32_t *s_rd = s_flag + 1;             // [TEAMS] warps done reading the team's buffer (NB = 1)
    unsigned long long *s_bar = reinterpret_cast<unsigned long long *>(smem + lay.bar);   // [TEAMS][2]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int team = warp / W, wt = warp % W;
    const int n_sub = p.n_sub, n_t = p.n_t, Tp = p.Tp;
    const int t_off = p.t_off_dev ? *p.t_off_dev : p.t_off;
    const int eoff = t_off & (kEpv - 1);
    const int row_elems = static_cast<int>(align_up(static_cast<size_t>(eoff + n_t), kEpv));
    const bool mask_tail = row_elems != eoff + n_t;
    const size_t buf_bytes = (size_t)n_sub * Tp * kEs;

    const int table_words = p.n_u * kInfo + p.n_deltas + p.n_u * n_sub;
    for (int i = tid; i < table_words; i += kThreads) s_table[i] = p.table[i];
    const int32_t *s_info = s_table;
    const int32_t *s_delta = s_table + p.n_u * kInfo;
    const int32_t *s_shift = s_delta + p.n_deltas;
    // -inf past the copied part of every row of every buffer (never overwritten)
    for (int b = 0; b < NB * TEAMS; ++b)
        for (int i = tid; i < n_sub * (Tp - row_elems); i += kThreads) {
            const int k = i / (Tp - row_elems), t = row_elems + i % (Tp - row_elems);
            unsigned char *row = s_xs + b * buf_bytes + (size_t)k * Tp * kEs;
            if constexpr (ST == 0)
                reinterpret_cast<float *>(row)[t] = neg_inf();
            else
                reinterpret_cast<uint16_t *>(row)[t] = (ST == 1) ? 0xFF80u : 0xFC00u;
        }

    int64_t n_items = p.n_items;
    if (p.n_items_dev) n_items = *p.n_items_dev;
    auto item_pixel = [&](int64_t it) -> int64_t {
        return p.pix_list ? static_cast<int64_t>(p.pix_list[it]) : p.pix0 + it;
    };
    // buffer slot (team, b): pixel buffer and barrier; record slot (team, i mod 2): records,
    // 1 / (sigma sqrt(w)) and done counter of the team's i-th pixel (with NB = 2 the two coincide)
    const int slot0 = NB * team;
    // one warp: 1 / (sigma sqrt(w)) of item `it` into record slot rs, then its rows into buffer sl
    // (lane 0 arms the barrier, lane k copies subband k)
    auto issue_warp = [&](int64_t it, int sl, int rs) {
        const int64_t pix = item_pixel(it);
        if (lane < p.n_w) {
            const float sg = p.sigma ? p.sigma[pix] : p.sigma_default;
            s_inv[rs * kMaxW + lane] = 1.0f / (sg * sqrtf(static_cast<float>(p.widths[lane])));
        }
        __syncwarp();
        const uint32_t bytes = static_cast<uint32_t>(row_elems * kEs);
        if (lane == 0) mbar_expect_tx(&s_bar[sl], bytes * static_cast<uint32_t>(n_sub));
        __syncwarp();
        const unsigned char *src = static_cast<const unsigned char *>(p.cube);
        const int64_t row0 = (pix - p.cube_pix0) * n_sub;
        unsigned char *dst = s_xs + sl * buf_bytes;
        for (int k = lane; k < n_sub; k += 32)
            bulk_g2s(dst + (size_t)k * Tp * kEs, src + ((row0 + k) * p.row_len + t_off - eoff) * kEs, bytes,
                     &s_bar[sl]);
    };
    if (tid == 0) {
        for (int sl = 0; sl < NB * TEAMS; ++sl) mbar_init(&s_bar[sl], 1);
        for (int rs = 0; rs < 2 * TEAMS; ++rs) s_cnt[rs] = 0;
        for (int t = 0; t < TEAMS; ++t) s_rd[t] = 0;
        s_flag[0] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    __syncthreads();
    // the team's items: it0 = CTA * TEAMS + team, then every G = grid * TEAMS
    const int64_t G = static_cast<int64_t>(gridDim.x) * TEAMS;
    const int64_t it0 = static_cast<int64_t>(blockIdx.x) * TEAMS + team;
    if (wt == 0) {
        if (it0 < n_items) issue_warp(it0, slot0, 2 * team);
        if (NB == 2 && it0 + G < n_items) issue_warp(it0 + G, slot0 + 1, 2 * team + 1);
    }

    const int n_ua = p.n_u_active;
    float *Pw = s_pbuf + (size_t)warp * 32 * C;
    float *Sw = reinterpret_cast<float *>(smem + lay.fscr) + (size_t)warp * kFindScr;
    int issued_last = -1;   // local index of the last item whose copy this warp started
    int i = 0;
    for (int64_t it = it0; it < n_items; it += G, ++i) {
        const int b = i % NB, sl = slot0 + b, rs = 2 * team + (i & 1);
        if (*reinterpret_cast<volatile int32_t *>(s_flag)) break;
        if (!mbar_wait(&s_bar[sl], static_cast<uint32_t>(i / NB) & 1u)) {
            if (lane == 0) {
                atomicOr(s_flag, ERR_WAIT_TIMEOUT);
                atomicOr(p.err, ERR_WAIT_TIMEOUT);
            }
            break;
        }
        const int g = (wt + i) % W;
        const int u_lo = (g * n_ua) / W, u_hi = ((g + 1) * n_ua) / W;
        const int64_t pix = item_pixel(it);
        // kEarly: the last warp of the team to read buffer sl for this pixel starts the copy of the
        // team's next pixel into it (its 1 / (sigma sqrt(w)) into the other record slot); each warp's
        // reads of the buffer are done before the async-proxy copy that refills it
        auto read_done = [&]() {
            if constexpr (kEarly) {
                fence_proxy_async();
                int lastr = 0;
                if (lane == 0) {
                    __threadfence_block();
                    lastr = atomicAdd(&s_rd[team], 1) == W - 1;
                    __threadfence_block();
                }
                lastr = __shfl_sync(kFull, lastr, 0);
                if (lastr) {
                    if (lane == 0) s_rd[team] = 0;
                    __syncwarp();
                    if (it + G < n_items) {
                        issue_warp(it + G, sl, 2 * team + ((i + 1) & 1));
                        issued_last = i + 1;
                    }
                }
                __syncwarp();
            }
        };
        PixRec wr;
        if constexpr (kEarly)
            wr = search_rows_any<C, FULL, ST>(p, s_xs + sl * buf_bytes, Pw, Sw, s_inv + rs * kMaxW, s_info, s_delta,
                                              s_shift, u_lo, u_hi, pix, lane, eoff, mask_tail, read_done);
        else
            wr = search_rows_any<C, FULL, ST>(p, s_xs + sl * buf_bytes, Pw, Sw, s_inv + rs * kMaxW, s_info, s_delta,
                                              s_shift, u_lo, u_hi, pix, lane, eoff, mask_tail);
        // FULL mode: a pixel whose MAD is zero has no trial; its rows' entries become -inf / -1
        if constexpr (FULL) {
            if (p.bad_pix && p.bad_pix[pix]) {
                __syncwarp();
                full_fill_empty(p, s_info, u_lo, u_hi, pix, lane);
            }
        }
        // publish; this warp's reads of buffer sl are done before the copy that refills it
        fence_proxy_async();
        int last = 0;
        if (lane == 0) {
            s_wbest[rs * kWarps + g] = wr;
            __threadfence_block();
            last = atomicAdd(&s_cnt[rs], 1) == W - 1;
            __threadfence_block();
        }
        last = __shfl_sync(kFull, last, 0);
        if (last) {
            if (lane == 0) {
                PixRec best{neg_inf(), -1, -1, -1};
                for (int q = 0; q < W; ++q) {
                    const PixRec r = s_wbest[rs * kWarps + q];
                    if (r.snr > best.snr) best = r;
                }
                if (best.dm_idx >= 0) best.dm_idx = s_info[best.dm_idx * kInfo + UI_FIRST_D];
                if (p.bad_pix && p.bad_pix[pix]) {
                    best = PixRec{neg_inf(), -1, -1, -1};
                    atomicOr(p.err, ERR_ZERO_MAD);
                }
                p.rec[pix] = best;
                s_cnt[rs] = 0;
            }
            // FULL mode: DM rows that have no trial at all
            if constexpr (FULL) full_fill_empty(p, s_info, n_ua, p.n_u, pix, lane);
            __syncwarp();
            const int64_t nxt = it + NB * G;
            if (!kEarly && nxt < n_items) {
                issue_warp(nxt, sl, 2 * team + ((i + NB) & 1));
                issued_last = i + NB;
            }
        }
        __syncwarp();
    }
    // after an error: wait (bounded) for copies this warp started that may still be in flight
    if (*reinterpret_cast<volatile int32_t *>(s_flag) && lane == 0 && issued_last >= 0)
        mbar_wait(&s_bar[slot0 + issued_last % NB], static_cast<uint32_t>(issued_last / NB) & 1u);
}

}  // namespace dev

// The barrier-free kernel's pixel x DM tiles (teams, buffers per team), one launcher per chunk size
// and storage type (16-bit rows read in place need the sample-pair path of even chunks).
#define NSFRB_PIPE_CASE(CC, ST, T, B)                                                          \
    case 10 * T + B:                                                                           \
        if (p.full_snr)                                                                        \
            dev::search_kernel_pipe<CC, ST, T, B, true><<<grid, kThreads, smem, s>>>(p);       \
        else                                                                                   \
            dev::search_kernel_pipe<CC, ST, T, B, false><<<grid, kThreads, smem, s>>>(p);      \
        break;
#define NSFRB_PIPE_ATTR1(CC, ST, T, B)                                                         \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(dev::search_kernel_pipe<CC, ST, T, B, false>,                 \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, sm);             \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(dev::search_kernel_pipe<CC, ST, T, B, true>,                  \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
#define NSFRB_INSTANTIATE_PIPE(CC, ST)                                                         \
    cudaError_t launch_pipe_c##CC##_s##ST(const SearchParams &p, int grid, size_t smem, cudaStream_t s) { \
        switch (10 * p.teams + p.nb) {                                                         \
            NSFRB_PIPE_CASE(CC, ST, 1, 2)                                                      \
            NSFRB_PIPE_CASE(CC, ST, 2, 2)                                                      \
            NSFRB_PIPE_CASE(CC, ST, 2, 1)                                                      \
            NSFRB_PIPE_CASE(CC, ST, 3, 1)                                                      \
            NSFRB_PIPE_CASE(CC, ST, 4, 1)                                                      \
            default:                                                                           \
                return cudaErrorInvalidValue;                                                  \
        }                                                                                      \
        return cudaGetLastError();                                                             \
    }                                                                                          \
    cudaError_t prepare_pipe_c##CC##_s##ST(size_t smem) {                                      \
        const int sm = static_cast<int>(smem);                                                 \
        cudaError_t e = cudaSuccess;                                                           \
        NSFRB_PIPE_ATTR1(CC, ST, 1, 2)                                                         \
        NSFRB_PIPE_ATTR1(CC, ST, 2, 2)                                                         \
        NSFRB_PIPE_ATTR1(CC, ST, 2, 1)                                                         \
        NSFRB_PIPE_ATTR1(CC, ST, 3, 1)                                                         \
        NSFRB_PIPE_ATTR1(CC, ST, 4, 1)                                                         \
        return e;                                                                              \
    }

// The barrier kernels of a chunk size and its launch dispatch; the barrier-free kernel's launchers
// come from NSFRB_INSTANTIATE_PIPE (16-bit ones in translation units of their own).
#define NSFRB_INSTANTIATE_SEARCH(CC)                                                           \
    cudaError_t launch_pipe_c##CC##_s0(const SearchParams &, int, size_t, cudaStream_t);      \
    cudaError_t launch_pipe_c##CC##_s1(const SearchParams &, int, size_t, cudaStream_t);      \
    cudaError_t launch_pipe_c##CC##_s2(const SearchParams &, int, size_t, cudaStream_t);      \
    cudaError_t prepare_pipe_c##CC##_s0(size_t);                                               \
    cudaError_t prepare_pipe_c##CC##_s1(size_t);                                               \
    cudaError_t prepare_pipe_c##CC##_s2(size_t);                                               \
    cudaError_t launch_search_c##CC(const SearchParams &p, int grid, size_t smem, cudaStream_t s) { \
        if (p.pipe) {                                                                          \
            if (p.dtype == 0) return launch_pipe_c##CC##_s0(p, grid, smem, s);                 \
            if constexpr (CC % 2 == 0) {                                                       \
                if (p.dtype == 1) return launch_pipe_c##CC##_s1(p, grid, smem, s);             \
                return launch_pipe_c##CC##_s2(p, grid, smem, s);                               \
            }                                                                                  \
            return cudaErrorInvalidValue;                                                      \
        }                                                                                      \
        if (p.full_snr)                                                                        \
            dev::search_kernel<CC, true><<<grid, kThreads, smem, s>>>(p);                      \
        else                                                                                   \
            dev::search_kernel<CC, false><<<grid, kThreads, smem, s>>>(p);                     \
        return cudaGetLastError();                                                             \
    }                                                                                          \
    cudaError_t prepare_search_c##CC(size_t smem) {                                            \
        const int sm = static_cast<int>(smem);                                                 \
        cudaError_t e = cudaFuncSetAttribute(dev::search_kernel<CC, false>,                    \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm); \
        if (e == cudaSuccess)                                                                  \
            e = cudaFuncSetAttribute(dev::search_kernel<CC, true>,                             \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, sm);         \
        if (e == cudaSuccess) e = prepare_pipe_c##CC##_s0(smem);                               \
        if constexpr (CC % 2 == 0) {                                                           \
            if (e == cudaSuccess) e = prepare_pipe_c##CC##_s1(smem);                           \
            if (e == cudaSuccess) e = prepare_pipe_c##CC##_s2(smem);                           \
        }                                                                                      \
        return e;                                                                              \
    }

}  // namespace nsfrb
