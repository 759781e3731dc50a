// Dirty imaging of arXiv 2510.18136 Sec. 2.1: per (134 ms sample, subband),
// the fringe-stopped visibilities of the core baselines (b_min < |b| < b_max,
// polarisations summed) are gridded with Briggs weighting (robustness R) on an
// N x N uv-grid and inverse-FFT'd (shifted before and after, numpy's 1/N^2
// normalisation); the subband's channels are imaged separately and summed.
//
// GB300 design.  The uv support of a compact core is small (|k| <= 21 cells of
// the 175-cell grid at the paper's 10.3" pixel), so the transform is pruned
// to the occupied cells instead of running a full FFT over a mostly empty grid:
//   * the grid is Hermitian, so only the half-plane u >= 0 is built;
//   * A_u(y) = sum_v G[u][v] e^{2 pi i v y'/N} over the occupied v, u = 0..U;
//   * img[y][x] = (A_0(y) + 2 Re sum_{u>=1} A_u(y) e^{2 pi i u x'/N}) / N^2,
//     with y' = y + N/2, x' = x + N/2 (mod N): the two shifts as index offsets.
// The rows y' and N - y' share the cos / sin sums of the first transform, and
// the columns x' and N - x' those of the second: each sum serves two outputs.
// Summing the channels' grids before one transform equals summing the channel
// images (the transform is linear); each channel keeps its own weights.
//
// Two kernels.  grid_kernel, persistent (one CTA per SM): each (subband,
// channel, sample) row of visibilities arrives in shared memory by one bulk
// copy (double-buffered, the next rows in flight while one is gridded); each
// weighted value goes to its precomputed slot of the channel's cell-sorted
// order, then every cell adds its slots in order and the channel's partial
// grid goes to a small workspace.  transform_kernel, one CTA
// per image: adds the channel partial grids in channel order (so the image is
// reproducible bit for bit), then the two transforms as register-tiled
// products from shared memory, written straight to the image rows.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "async_copy.cuh"
#include "plan_internal.h"

namespace nsfrb {
namespace {

constexpr int kGridThreads = 512;
constexpr int kTrThreads = 256;
constexpr double kCLight = 299792458.0;
constexpr int32_t kSlotMask = 0x3fffffff;   // slot index; bit 30 = conjugate; negative = no entry
constexpr int32_t kErrWait = 1;             // a bulk copy did not complete within the wait limit
constexpr int kChunk = 8;                   // slots summed by one thread in the first level

// Slot s is stored at s + s / 8: consecutive chunks (8 slots apart) then fall 9 entries
// apart in shared memory, which spreads the chunk sums' loads over the banks.
__device__ __forceinline__ int slot_pos(int s) { return s + (s >> 3); }

struct GridParams {
    const float4 *vis;        // [n_t][n_sub][n_chan][n_base] (pol0 re, pol0 im, pol1 re, pol1 im)
    const int4 *rec;          // [n_sub][n_chan][n_base]: (slot 1, slot 2 (ku = 0 column) or -1,
                              // weight bits, 0); slot = index | conj << 30, -1 = none
    const int2 *chunks;       // per (subband, channel): runs of <= kChunk slots of one cell,
                              // (first slot, count), in cell order
    const int32_t *chunk0;    // [n_sub * n_chan + 1]: first chunk of each (subband, channel)
    const int32_t *cchunk;    // [n_sub][n_chan][n_cells + 1]: first chunk of each cell (local)
    float2 *part;             // [n_img][n_chan][n_cells] partial grids
    int32_t *err;             // error word (kErrWait)
    int32_t n_t, n_sub, n_chan, n_base, n_cells;
    int64_t n_units;          // n_sub * n_chan * n_t, ordered (subband, channel)-major
};

struct GridSmem {
    size_t bar, vbuf, rec, slots, chunks, ctab, cchunk, total;
};

inline GridSmem grid_smem_plan(int n_base, int max_slots, int max_chunks, int n_cells) {
    GridSmem s;
    s.bar = 0;
    s.vbuf = 128;
    s.rec = s.vbuf + 2 * sizeof(float4) * static_cast<size_t>(n_base);
    s.slots = s.rec + sizeof(int4) * static_cast<size_t>(n_base);
    s.chunks = s.slots + sizeof(float2) * static_cast<size_t>(std::max(max_slots, 1) + max_slots / 8 + 1);
    s.ctab = s.chunks + sizeof(float2) * static_cast<size_t>(std::max(max_chunks, 1));   // chunk table
    s.cchunk = s.ctab + sizeof(int2) * static_cast<size_t>(std::max(max_chunks, 1));
    s.total = s.cchunk + sizeof(int32_t) * static_cast<size_t>(n_cells + 1);
    return s;
}

// Persistent: CTA b takes a contiguous range of (subband, channel, sample) units, so
// consecutive units mostly share the (subband, channel) records, which are copied into
// shared memory when the pair changes.  Each unit's visibility row (n_base x 16 bytes,
// contiguous) arrives by one bulk copy into a double buffer, the copy of unit i + 2 in
// flight while unit i is gridded.
__global__ void __launch_bounds__(kGridThreads, 1) grid_kernel(GridParams p, GridSmem L) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned long long *s_bar = reinterpret_cast<unsigned long long *>(smem_raw + L.bar);
    float4 *s_vis = reinterpret_cast<float4 *>(smem_raw + L.vbuf);
    int4 *s_rec = reinterpret_cast<int4 *>(smem_raw + L.rec);
    float2 *s_slot = reinterpret_cast<float2 *>(smem_raw + L.slots);
    float2 *s_chunk = reinterpret_cast<float2 *>(smem_raw + L.chunks);
    int2 *s_ctab = reinterpret_cast<int2 *>(smem_raw + L.ctab);
    int32_t *s_cchunk = reinterpret_cast<int32_t *>(smem_raw + L.cchunk);
    __shared__ int s_fail;
    const int tid = threadIdx.x;
    const int64_t u_lo = blockIdx.x * p.n_units / gridDim.x, u_hi = (blockIdx.x + 1) * p.n_units / gridDim.x;
    const int n_u = static_cast<int>(u_hi - u_lo);
    const uint32_t row_bytes = static_cast<uint32_t>(p.n_base) * 16u;
    // (pair, t) of the first unit: one division per CTA; both cursors then advance by one
    const int pair_lo = static_cast<int>(u_lo / p.n_t), t_lo = static_cast<int>(u_lo - (int64_t)pair_lo * p.n_t);
    int iss_pair = pair_lo, iss_t = t_lo;   // next unit to copy (thread 0)

    auto issue_next = [&](int buf) {
        const int sub = iss_pair / p.n_chan, ch = iss_pair - sub * p.n_chan;
        const float4 *src = p.vis + (((int64_t)iss_t * p.n_sub + sub) * p.n_chan + ch) * (int64_t)p.n_base;
        dev::mbar_expect_tx(&s_bar[buf], row_bytes);
        dev::bulk_g2s(s_vis + (size_t)buf * p.n_base, src, row_bytes, &s_bar[buf]);
        if (++iss_t == p.n_t) {
            iss_t = 0;
            ++iss_pair;
        }
    };
    if (tid == 0) {
        dev::mbar_init(&s_bar[0], 1);
        dev::mbar_init(&s_bar[1], 1);
        dev::mbar_init(&s_bar[2], 1);   // records
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        dev::fence_proxy_async();
        if (n_u > 0) issue_next(0);
        if (n_u > 1) issue_next(1);
    }
    __syncthreads();

    int cur_pair = -1, pair = pair_lo, t = t_lo, sub = 0, ch = 0;
    uint32_t rec_parity = 0;
    for (int i = 0; i < n_u; ++i) {
        const int buf = i & 1;
        const uint32_t parity = static_cast<uint32_t>(i >> 1) & 1u;
        if (pair != cur_pair) {
            // every read of the previous records finished before the last barrier of the loop
            if (tid == 0) {
                dev::mbar_expect_tx(&s_bar[2], row_bytes);
                dev::bulk_g2s(s_rec, p.rec + (int64_t)pair * p.n_base, row_bytes, &s_bar[2]);
            }
            // the pair's chunk tables, while the records copy is in flight
            const int c0 = p.chunk0[pair], n_ch = p.chunk0[pair + 1] - c0;
            for (int k = tid; k < n_ch; k += kGridThreads) s_ctab[k] = __ldg(p.chunks + c0 + k);
            for (int c = tid; c <= p.n_cells; c += kGridThreads) s_cchunk[c] = __ldg(p.cchunk + (int64_t)pair * (p.n_cells + 1) + c);
            if (!dev::mbar_wait(&s_bar[2], rec_parity)) atomicOr(&s_fail, 1);
            rec_parity ^= 1u;
            cur_pair = pair;
            sub = pair / p.n_chan;
            ch = pair - sub * p.n_chan;
        }
        if (!dev::mbar_wait(&s_bar[buf], parity)) atomicOr(&s_fail, 1);
        __syncthreads();
        if (s_fail) {
            // record, then wait (bounded) for this CTA's copies still in flight before leaving
            if (tid == 0) {
                atomicOr(p.err, kErrWait);
                dev::mbar_wait(&s_bar[2], rec_parity ^ 1u);
                dev::mbar_wait(&s_bar[buf], parity);
                if (i + 1 < n_u) dev::mbar_wait(&s_bar[buf ^ 1], static_cast<uint32_t>((i + 1) >> 1) & 1u);
            }
            return;
        }
        const float4 *vb = s_vis + (size_t)buf * p.n_base;
        for (int b = tid; b < p.n_base; b += kGridThreads) {
            const int4 r = s_rec[b];
            if (r.x < 0) continue;
            const float4 v = vb[b];
            const float w = __int_as_float(r.z);
            const float re = (v.x + v.z) * w, im = (v.y + v.w) * w;
            s_slot[slot_pos(r.x & kSlotMask)] = make_float2(re, (r.x >> 30) ? -im : im);
            // on the ku = 0 column the mirror also lies in the half-plane
            if (r.y >= 0) s_slot[slot_pos(r.y & kSlotMask)] = make_float2(re, (r.y >> 30) ? -im : im);
        }
        // the buffer's (and the records') reads are done before the async proxy refills them
        dev::fence_proxy_async();
        __syncthreads();
        if (tid == 0 && i + 2 < n_u) issue_next(buf);
        // two-level sums in a fixed order: each chunk (<= kChunk slots of one cell) in slot
        // order, then each cell's chunks in order (dense cells spread over many threads)
        const int n_ch = s_cchunk[p.n_cells];
        for (int k = tid; k < n_ch; k += kGridThreads) {
            const int2 ck = s_ctab[k];
            float2 q[kChunk];
#pragma unroll
            for (int j = 0; j < kChunk; ++j) q[j] = j < ck.y ? s_slot[slot_pos(ck.x + j)] : make_float2(0.0f, 0.0f);
            float2 g = q[0];
#pragma unroll
            for (int j = 1; j < kChunk; ++j)
                if (j < ck.y) {
                    g.x += q[j].x;
                    g.y += q[j].y;
                }
            s_chunk[k] = g;
        }
        __syncthreads();
        float2 *out = p.part + ((t * p.n_sub + sub) * p.n_chan + ch) * (int64_t)p.n_cells;
        for (int c = tid; c < p.n_cells; c += kGridThreads) {
            float2 g = make_float2(0.0f, 0.0f);
            const int e = s_cchunk[c + 1];
            for (int k = s_cchunk[c]; k < e; ++k) {
                const float2 q = s_chunk[k];
                g.x += q.x;
                g.y += q.y;
            }
            out[c] = g;
        }
        __syncthreads();
        if (++t == p.n_t) {
            t = 0;
            ++pair;
        }
    }
}

struct TrParams {
    const float2 *part;       // [n_img][n_chan][n_cells]
    const float *tab;         // [2][K + 1][Hp]: cos, sin of 2 pi k j / N, j = 0..H (0 beyond);
                              // Hp a multiple of 96
    float *img;               // [n_img][N][N]
    int32_t n_chan, n_cells, N, H, Hp, Np, U, V, K, ctr;
    float inv_n2;
};

struct TrSmem {
    size_t tab, ar, g, total;
};

inline TrSmem tr_smem(int K, int U, int Hp, int Np, int n_cells) {
    TrSmem s;
    s.tab = 0;
    s.ar = s.tab + sizeof(float) * 2 * static_cast<size_t>(K + 1) * Hp;
    s.g = s.ar + sizeof(float) * 2 * static_cast<size_t>(U + 1) * Np;
    s.total = s.g + sizeof(float2) * static_cast<size_t>(n_cells);
    return s;
}

__global__ void __launch_bounds__(kTrThreads, 3) transform_kernel(TrParams p, TrSmem L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = p.N, Hp = p.Hp, Np = p.Np, U = p.U, V = p.V, nv = 2 * V + 1;
    float *s_cos = reinterpret_cast<float *>(smem_raw + L.tab);   // [K + 1][Hp]
    float *s_sin = s_cos + (size_t)(p.K + 1) * Hp;
    float *s_ar = reinterpret_cast<float *>(smem_raw + L.ar);     // [U + 1][Np], row y of the image
    float *s_ai = s_ar + (size_t)(U + 1) * Np;
    float2 *s_G = reinterpret_cast<float2 *>(smem_raw + L.g);      // [U + 1][2V + 1]
    const int tid = threadIdx.x;
    const int img = blockIdx.x;

    {
        const float4 *src = reinterpret_cast<const float4 *>(p.tab);
        float4 *dst = reinterpret_cast<float4 *>(s_cos);
        for (int i = tid; i < (p.K + 1) * Hp / 2; i += kTrThreads) dst[i] = src[i];
    }
    // channel partial grids added in channel order; the loads of 8 channels in flight at once
    const float2 *part = p.part + (size_t)img * p.n_chan * p.n_cells;
    for (int c = tid; c < p.n_cells; c += kTrThreads) {
        float2 g = part[c];
        for (int ch0 = 1; ch0 < p.n_chan; ch0 += 8) {
            float2 q[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                q[k] = (ch0 + k < p.n_chan) ? __ldcg(part + (size_t)(ch0 + k) * p.n_cells + c) : make_float2(0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (ch0 + k < p.n_chan) {
                    g.x += q[k].x;
                    g.y += q[k].y;
                }
        }
        s_G[c] = g;
    }
    __syncthreads();

    // ---- transform along v for the row pairs y' = j and y' = N - j, j = 0..H
    // A(j) = G_0 + sum_v [P cos + i Q sin], A(N - j) = G_0 + sum_v [P cos - i Q sin],
    // with P = G_v + G_-v, Q = G_v - G_-v: four sums serve both rows.
    const int nj4 = Hp / 4;
    for (int q = tid; q < (U + 1) * nj4; q += kTrThreads) {
        const int u = q / nj4, j0 = 4 * (q - u * nj4);
        const float2 *g = s_G + u * nv + V;
        float x1[4] = {0, 0, 0, 0}, x2[4] = {0, 0, 0, 0}, y1[4] = {0, 0, 0, 0}, y2[4] = {0, 0, 0, 0};
        for (int v = 1; v <= V; ++v) {
            const float2 gp = g[v], gm = g[-v];
            const float px = gp.x + gm.x, py = gp.y + gm.y, qx = gp.x - gm.x, qy = gp.y - gm.y;
            const float4 c4 = *reinterpret_cast<const float4 *>(s_cos + v * Hp + j0);
            const float4 s4 = *reinterpret_cast<const float4 *>(s_sin + v * Hp + j0);
            const float cc[4] = {c4.x, c4.y, c4.z, c4.w}, ss[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                x1[i] = fmaf(px, cc[i], x1[i]);
                x2[i] = fmaf(qy, ss[i], x2[i]);
                y1[i] = fmaf(py, cc[i], y1[i]);
                y2[i] = fmaf(qx, ss[i], y2[i]);
            }
        }
        const float2 g0 = g[0];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int j = j0 + i;
            if (j > p.H) break;
            int y = j - p.ctr;
            if (y < 0) y += N;
            s_ar[u * Np + y] = g0.x + x1[i] - x2[i];
            s_ai[u * Np + y] = g0.y + y1[i] + y2[i];
            if (j != 0 && 2 * j != N) {
                int ym = N - j - p.ctr;
                if (ym < 0) ym += N;
                s_ar[u * Np + ym] = g0.x + x1[i] + x2[i];
                s_ai[u * Np + ym] = g0.y + y1[i] - y2[i];
            }
        }
    }
    __syncthreads();

    // ---- transform along u for the column pairs x' = j and x' = N - j:
    // C = sum_u Ar_u cos, S = sum_u Ai_u sin give (A_0 + 2 (C -+ S)) / N^2.
    // One warp per band of 8 rows; in each block of 96 column pairs lane l takes
    // j = l, l + 32, l + 64 of the block (consecutive lanes write consecutive columns).
    float *out = p.img + (size_t)img * N * N;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int kJ = 3;                     // column pairs per lane per block of 96
    const int n_bands = (N + 7) / 8;
    for (int band = warp; band < n_bands; band += kTrThreads / 32) {
        const int y0 = 8 * band;
        for (int jb = 0; jb <= p.H; jb += 32 * kJ) {
            int xs[kJ], xm[kJ];
            bool jok[kJ], mok[kJ];
#pragma unroll
            for (int k = 0; k < kJ; ++k) {
                const int j = jb + lane + 32 * k;
                jok[k] = j <= p.H;
                mok[k] = jok[k] && j != 0 && 2 * j != N;
                xs[k] = j - p.ctr + (j < p.ctr ? N : 0);
                xm[k] = N - j - p.ctr + (N - j < p.ctr ? N : 0);
            }
            float C[8][kJ], S[8][kJ];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int k = 0; k < kJ; ++k) {
                    C[i][k] = 0.0f;
                    S[i][k] = 0.0f;
                }
            for (int u = 1; u <= U; ++u) {
                const float4 a0 = *reinterpret_cast<const float4 *>(s_ar + u * Np + y0);
                const float4 a1 = *reinterpret_cast<const float4 *>(s_ar + u * Np + y0 + 4);
                const float4 b0 = *reinterpret_cast<const float4 *>(s_ai + u * Np + y0);
                const float4 b1 = *reinterpret_cast<const float4 *>(s_ai + u * Np + y0 + 4);
                const float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float ai[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                float cc[kJ], ss[kJ];
#pragma unroll
                for (int k = 0; k < kJ; ++k) {
                    cc[k] = s_cos[u * Hp + jb + lane + 32 * k];
                    ss[k] = s_sin[u * Hp + jb + lane + 32 * k];
                }
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int k = 0; k < kJ; ++k) {
                        C[i][k] = fmaf(ar[i], cc[k], C[i][k]);
                        S[i][k] = fmaf(ai[i], ss[k], S[i][k]);
                    }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int y = y0 + i;
                if (y >= N) break;
                const float base = s_ar[y];
                float *row = out + (size_t)y * N;
#pragma unroll
                for (int k = 0; k < kJ; ++k) {
                    if (jok[k]) row[xs[k]] = (base + 2.0f * (C[i][k] - S[i][k])) * p.inv_n2;
                    if (mok[k]) row[xm[k]] = (base + 2.0f * (C[i][k] + S[i][k])) * p.inv_n2;
                }
            }
        }
    }
}

}  // namespace
}  // namespace nsfrb

using namespace nsfrb;

struct nsfrb_imager_s {
    int32_t N = 0, Np = 0, H = 0, Hp = 0, n_sub = 0, n_chan = 0, n_base = 0;
    int32_t U = 0, V = 0, K = 0, n_cells = 0, max_slots = 0;
    int64_t n_entries = 0;
    std::vector<float> weights;      // [n_sub][n_chan][n_base]
    int4 *d_rec = nullptr;
    int2 *d_chunks = nullptr;
    int32_t *d_chunk0 = nullptr, *d_cchunk = nullptr;
    int32_t max_chunks = 0;
    float *d_tab = nullptr;
    float2 *d_part = nullptr;        // workspace: partial grids
    int64_t part_images = 0;         // images the workspace holds
    TrSmem tr{};
    GridSmem gs{};
    int32_t *d_err = nullptr;
    int device = -1, n_sm = 0;
};

namespace {

void imager_free(nsfrb_imager_s *im) {
    cudaFree(im->d_rec);
    cudaFree(im->d_chunks);
    cudaFree(im->d_chunk0);
    cudaFree(im->d_cchunk);
    cudaFree(im->d_tab);
    cudaFree(im->d_part);
    cudaFree(im->d_err);
}

struct Entry {
    int32_t ku, kv;  // half-plane coordinates (ku >= 0)
    int32_t b;       // baseline
    int32_t which;   // 0: the baseline's first slot, 1: its second (ku = 0 column)
    bool conj;
};

}  // namespace

extern "C" {

nsfrb_status nsfrb_imager_create(const nsfrb_imager_config *cfg, nsfrb_imager_t *out) {
    if (!cfg || !out) return fail(nullptr, NSFRB_EINVAL, "null argument");
    *out = nullptr;
    const nsfrb_imager_config &c = *cfg;
    if (c.n_grid < 3 || c.n_grid > 1024) return fail(nullptr, NSFRB_EINVAL, "n_grid must be 3..1024");
    if (!(c.pixel_arcsec > 0.0) || !std::isfinite(c.pixel_arcsec)) return fail(nullptr, NSFRB_EINVAL, "bad pixel size");
    if (!std::isfinite(c.robust)) return fail(nullptr, NSFRB_EINVAL, "bad robustness");
    if (!(c.b_min_m >= 0.0) || !(c.b_max_m > c.b_min_m)) return fail(nullptr, NSFRB_EINVAL, "need 0 <= b_min < b_max");
    if (c.n_base < 1 || c.n_sub < 1 || c.n_chan < 1 || !c.uv_m || !c.chan_mhz)
        return fail(nullptr, NSFRB_EINVAL, "need n_base, n_sub, n_chan >= 1 and the uv / frequency arrays");
    if (static_cast<int64_t>(c.n_sub) * c.n_chan * c.n_base >= (int64_t(1) << 31) || c.n_base >= (1 << 29))
        return fail(nullptr, NSFRB_EINVAL, "n_sub * n_chan * n_base too large");
    for (int64_t i = 0; i < 2LL * c.n_base; ++i)
        if (!std::isfinite(c.uv_m[i])) return fail(nullptr, NSFRB_EINVAL, "non-finite uv");
    for (int64_t i = 0; i < static_cast<int64_t>(c.n_sub) * c.n_chan; ++i)
        if (!(c.chan_mhz[i] > 0.0) || !std::isfinite(c.chan_mhz[i]))
            return fail(nullptr, NSFRB_EINVAL, "channel frequencies must be > 0");

    auto *im = new nsfrb_imager_s();
    const int N = c.n_grid, h = (N - 1) / 2, ctr = N / 2;
    im->N = N;
    im->Np = (N + 7) & ~7;
    im->H = N / 2;
    im->Hp = (im->H + 1 + 95) / 96 * 96;   // whole blocks of 96 column pairs (multiple of 4)
    im->n_sub = c.n_sub;
    im->n_chan = c.n_chan;
    im->n_base = c.n_base;
    const size_t n_sc = static_cast<size_t>(c.n_sub) * c.n_chan;
    im->weights.assign(n_sc * c.n_base, 0.0f);
    const double dth = c.pixel_arcsec * M_PI / 648000.0;

    std::vector<uint8_t> kept(c.n_base);
    for (int b = 0; b < c.n_base; ++b) {
        const double u = c.uv_m[2 * b], v = c.uv_m[2 * b + 1];
        const double len = std::sqrt(u * u + v * v);
        kept[b] = len > c.b_min_m && len < c.b_max_m;
    }
    // half-plane entries of every (subband, channel)
    std::vector<std::vector<Entry>> per_sc(n_sc);
    std::vector<double> W(static_cast<size_t>(N) * N);
    std::vector<int32_t> ku(c.n_base), kv(c.n_base);
    std::vector<uint8_t> ok(c.n_base);
    int U = 0, V = 0;
    for (int s = 0; s < c.n_sub; ++s) {
        for (int ch = 0; ch < c.n_chan; ++ch) {
            const double f = c.chan_mhz[s * c.n_chan + ch];
            std::fill(W.begin(), W.end(), 0.0);
            int64_t n_ok = 0;
            for (int b = 0; b < c.n_base; ++b) {
                // cell = rint(u * f_MHz * 1e6 / c * N * dtheta), evaluated left to right
                const double xu = c.uv_m[2 * b] * f * 1.0e6 / kCLight * N * dth;
                const double xv = c.uv_m[2 * b + 1] * f * 1.0e6 / kCLight * N * dth;
                ok[b] = 0;
                if (!kept[b] || !(std::fabs(xu) < 4.0e9) || !(std::fabs(xv) < 4.0e9)) continue;
                ku[b] = static_cast<int32_t>(std::nearbyint(xu));
                kv[b] = static_cast<int32_t>(std::nearbyint(xv));
                if (std::abs(ku[b]) > h || std::abs(kv[b]) > h) continue;
                ok[b] = 1;
                ++n_ok;
                W[static_cast<size_t>(ctr + kv[b]) * N + ctr + ku[b]] += 1.0;
                W[static_cast<size_t>(ctr - kv[b]) * N + ctr - ku[b]] += 1.0;
            }
            if (n_ok == 0) continue;
            double sum_w2 = 0.0;
            for (double x : W) sum_w2 += x * x;
            const double sum_w = 2.0 * static_cast<double>(n_ok);
            const double r = 5.0 * std::pow(10.0, -c.robust);
            const double f2 = r * r / (sum_w2 / sum_w);
            auto &es = per_sc[static_cast<size_t>(s) * c.n_chan + ch];
            for (int b = 0; b < c.n_base; ++b) {
                if (!ok[b]) continue;
                const double wd = 1.0 / (1.0 + W[static_cast<size_t>(ctr + kv[b]) * N + ctr + ku[b]] * f2);
                im->weights[(static_cast<size_t>(s) * c.n_chan + ch) * c.n_base + b] = static_cast<float>(wd);
                auto add = [&](int32_t a, int32_t bb, int which, bool conj) {
                    es.push_back(Entry{a, bb, b, which, conj});
                    U = std::max(U, a);
                    V = std::max(V, std::abs(bb));
                };
                if (ku[b] > 0) add(ku[b], kv[b], 0, false);
                else if (ku[b] < 0) add(-ku[b], -kv[b], 0, true);
                else {
                    add(0, kv[b], 0, false);
                    add(0, -kv[b], 1, true);
                }
            }
        }
    }
    im->U = U;
    im->V = V;
    im->K = std::max(U, V);
    const int nv = 2 * V + 1;
    im->n_cells = (U + 1) * nv;

    // slots: each (subband, channel)'s entries in cell order (stable: baseline order within a cell)
    std::vector<int4> rec(n_sc * c.n_base, make_int4(-1, -1, 0, 0));
    std::vector<int32_t> cstart(n_sc * (im->n_cells + 1));
    std::vector<int2> chunks;
    std::vector<int32_t> chunk0(n_sc + 1, 0), cchunk(n_sc * (im->n_cells + 1));
    for (size_t sc = 0; sc < n_sc; ++sc) {
        auto &es = per_sc[sc];
        std::stable_sort(es.begin(), es.end(), [nv](const Entry &a, const Entry &b) {
            return a.ku * nv + a.kv < b.ku * nv + b.kv;
        });
        im->max_slots = std::max(im->max_slots, static_cast<int32_t>(es.size()));
        im->n_entries += static_cast<int64_t>(es.size());
        int32_t *cs = cstart.data() + sc * (im->n_cells + 1);
        size_t i = 0;
        for (int cell = 0; cell < im->n_cells; ++cell) {
            cs[cell] = static_cast<int32_t>(i);
            while (i < es.size() && es[i].ku * nv + es[i].kv + V == cell) ++i;
        }
        cs[im->n_cells] = static_cast<int32_t>(es.size());
        // chunks of <= kChunk slots that do not cross a cell boundary
        chunk0[sc] = static_cast<int32_t>(chunks.size());
        int32_t *cck = cchunk.data() + sc * (im->n_cells + 1);
        for (int cell = 0; cell < im->n_cells; ++cell) {
            cck[cell] = static_cast<int32_t>(chunks.size()) - chunk0[sc];
            for (int32_t a = cs[cell]; a < cs[cell + 1]; a += kChunk)
                chunks.push_back(make_int2(a, std::min<int32_t>(kChunk, cs[cell + 1] - a)));
        }
        cck[im->n_cells] = static_cast<int32_t>(chunks.size()) - chunk0[sc];
        im->max_chunks = std::max(im->max_chunks, cck[im->n_cells]);
        for (size_t j = 0; j < es.size(); ++j) {
            const Entry &e = es[j];
            const int32_t code = static_cast<int32_t>(j) | (e.conj ? (1 << 30) : 0);
            int4 &r = rec[sc * c.n_base + e.b];
            if (e.which == 0) r.x = code;
            else r.y = code;
            const float w = im->weights[sc * c.n_base + e.b];
            std::memcpy(&r.z, &w, 4);
        }
    }

    // cos, sin of 2 pi k j / N for k = 0..K, j = 0..H, from the exact index (k j) mod N
    const int Hp = im->Hp;
    std::vector<float> tab(2 * static_cast<size_t>(im->K + 1) * Hp, 0.0f);
    for (int k = 0; k <= im->K; ++k)
        for (int j = 0; j <= im->H; ++j) {
            const int64_t m = (static_cast<int64_t>(k) * j) % N;
            double cv, sv;
            if (m == 0) {
                cv = 1.0;
                sv = 0.0;
            } else if (2 * m == N) {
                cv = -1.0;
                sv = 0.0;
            } else {
                const double a = 2.0 * M_PI * static_cast<double>(m) / N;
                cv = std::cos(a);
                sv = std::sin(a);
            }
            tab[static_cast<size_t>(k) * Hp + j] = static_cast<float>(cv);
            tab[(static_cast<size_t>(im->K + 1) + k) * Hp + j] = static_cast<float>(sv);
        }
    im->tr = tr_smem(im->K, U, Hp, im->Np, im->n_cells);
    chunk0[n_sc] = static_cast<int32_t>(chunks.size());
    im->gs = grid_smem_plan(c.n_base, im->max_slots, im->max_chunks, im->n_cells);

    nsfrb_status st = NSFRB_OK;
    int max_smem = 0;
    if ((st = cuda_check(nullptr, cudaGetDevice(&im->device), "device")) ||
        (st = cuda_check(nullptr, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, im->device),
                         "attribute")) ||
        (st = cuda_check(nullptr, cudaDeviceGetAttribute(&im->n_sm, cudaDevAttrMultiProcessorCount, im->device),
                         "attribute"))) {
        delete im;
        return st;
    }
    // the static part of grid_kernel's shared memory (one int) is far below the 1 KB margin
    if (im->tr.total > static_cast<size_t>(max_smem) || im->gs.total + 1024 > static_cast<size_t>(max_smem)) {
        delete im;
        return fail(nullptr, NSFRB_EINVAL, "uv support too large for one CTA's shared memory");
    }
    auto up = [&](void **dst, const void *src, size_t bytes) -> nsfrb_status {
        nsfrb_status s2 = cuda_check(nullptr, cudaMalloc(dst, std::max<size_t>(bytes, 16)), "cudaMalloc");
        if (s2 == NSFRB_OK && bytes)
            s2 = cuda_check(nullptr, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice), "copy");
        return s2;
    };
    if ((st = up(reinterpret_cast<void **>(&im->d_rec), rec.data(), sizeof(int4) * rec.size())) ||
        (st = up(reinterpret_cast<void **>(&im->d_chunks), chunks.data(), sizeof(int2) * chunks.size())) ||
        (st = up(reinterpret_cast<void **>(&im->d_chunk0), chunk0.data(), sizeof(int32_t) * chunk0.size())) ||
        (st = up(reinterpret_cast<void **>(&im->d_cchunk), cchunk.data(), sizeof(int32_t) * cchunk.size())) ||
        (st = up(reinterpret_cast<void **>(&im->d_tab), tab.data(), sizeof(float) * tab.size())) ||
        (st = cuda_check(nullptr, cudaMalloc(&im->d_err, sizeof(int32_t)), "cudaMalloc")) ||
        (st = cuda_check(nullptr, cudaMemset(im->d_err, 0, sizeof(int32_t)), "memset")) ||
        (st = cuda_check(nullptr, cudaFuncSetAttribute(grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      static_cast<int>(im->gs.total)), "smem attribute")) ||
        (st = cuda_check(nullptr, cudaFuncSetAttribute(transform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      static_cast<int>(im->tr.total)), "smem attribute"))) {
        if (st == NSFRB_ECUDA && std::string(nsfrb_last_error()).find("out of memory") != std::string::npos)
            st = NSFRB_ENOMEM;
        imager_free(im);
        delete im;
        return st;
    }
    *out = im;
    return NSFRB_OK;
}

nsfrb_status nsfrb_imager_weights(nsfrb_imager_t im, float *h_w) {
    if (!im || !h_w) return fail(nullptr, NSFRB_EINVAL, "null argument");
    std::memcpy(h_w, im->weights.data(), sizeof(float) * im->weights.size());
    return NSFRB_OK;
}

nsfrb_status nsfrb_imager_status(nsfrb_imager_t im) {
    if (!im) return fail(nullptr, NSFRB_EINVAL, "null argument");
    int32_t e = 0;
    nsfrb_status st = cuda_check(nullptr, cudaMemcpy(&e, im->d_err, sizeof(e), cudaMemcpyDeviceToHost), "copy");
    if (st) return st;
    if (e & kErrWait) {
        cudaMemset(im->d_err, 0, sizeof(int32_t));
        return fail(nullptr, NSFRB_ETIMEOUT, "an imager bulk copy did not complete within the wait limit");
    }
    return NSFRB_OK;
}

nsfrb_status nsfrb_imager_info(nsfrb_imager_t im, int32_t *u_max, int32_t *v_max, int64_t *n_entries) {
    if (!im) return fail(nullptr, NSFRB_EINVAL, "null argument");
    if (u_max) *u_max = im->U;
    if (v_max) *v_max = im->V;
    if (n_entries) *n_entries = im->n_entries;
    return NSFRB_OK;
}

nsfrb_status nsfrb_image(nsfrb_imager_t im, const float *d_vis, int32_t n_t, float *d_img, void *stream) {
    if (!im || n_t < 0 || (n_t > 0 && (!d_vis || !d_img))) return fail(nullptr, NSFRB_EINVAL, "bad argument");
    if ((reinterpret_cast<uintptr_t>(d_vis) & 15u) || (reinterpret_cast<uintptr_t>(d_img) & 3u))
        return fail(nullptr, NSFRB_EINVAL, "visibilities must be 16-byte aligned, images 4-byte aligned");
    if (n_t == 0) return NSFRB_OK;
    const int64_t n_img = static_cast<int64_t>(n_t) * im->n_sub;
    if (n_img * im->n_chan >= (int64_t(1) << 31)) return fail(nullptr, NSFRB_EINVAL, "too many images");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    nsfrb_status st;
    if (n_img > im->part_images) {
        // grow the partial-grid workspace (waits for earlier work that may still use it)
        if ((st = cuda_check(nullptr, cudaDeviceSynchronize(), "synchronise"))) return st;
        cudaFree(im->d_part);
        im->d_part = nullptr;
        im->part_images = 0;
        const size_t bytes = sizeof(float2) * static_cast<size_t>(n_img) * im->n_chan * im->n_cells;
        if (cudaMalloc(&im->d_part, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(nullptr, NSFRB_ENOMEM, "imager workspace");
        }
        im->part_images = n_img;
    }
    GridParams g;
    g.vis = reinterpret_cast<const float4 *>(d_vis);
    g.rec = im->d_rec;
    g.chunks = im->d_chunks;
    g.chunk0 = im->d_chunk0;
    g.cchunk = im->d_cchunk;
    g.part = im->d_part;
    g.err = im->d_err;
    g.n_t = n_t;
    g.n_sub = im->n_sub;
    g.n_chan = im->n_chan;
    g.n_base = im->n_base;
    g.n_cells = im->n_cells;
    g.n_units = n_img * im->n_chan;
    const int grid = static_cast<int>(std::min<int64_t>(g.n_units, im->n_sm));
    grid_kernel<<<grid, kGridThreads, im->gs.total, s>>>(g, im->gs);
    if ((st = cuda_check(nullptr, cudaGetLastError(), "grid launch"))) return st;
    TrParams t;
    t.part = im->d_part;
    t.tab = im->d_tab;
    t.img = d_img;
    t.n_chan = im->n_chan;
    t.n_cells = im->n_cells;
    t.N = im->N;
    t.H = im->H;
    t.Hp = im->Hp;
    t.Np = im->Np;
    t.U = im->U;
    t.V = im->V;
    t.K = im->K;
    t.ctr = im->N / 2;
    t.inv_n2 = static_cast<float>(1.0 / (static_cast<double>(im->N) * im->N));
    transform_kernel<<<static_cast<unsigned>(n_img), kTrThreads, im->tr.total, s>>>(t, im->tr);
    return cuda_check(nullptr, cudaGetLastError(), "transform launch");
}

void nsfrb_imager_destroy(nsfrb_imager_t im) {
    if (!im) return;
    imager_free(im);
    delete im;
}

}  // extern "C"
