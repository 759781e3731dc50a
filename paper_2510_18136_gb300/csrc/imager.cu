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
//   * A_u(y) = sum_v G[u][v] e^{2 pi i v y'/N} over the occupied v, for u = 0..U;
//   * img[y][x] = (A_0(y) + 2 Re sum_{u>=1} A_u(y) e^{2 pi i u x'/N}) / N^2,
//     with y' = y + N/2, x' = x + N/2 (mod N): the two shifts as phase offsets.
// Summing the channels' grids before one transform equals summing the channel
// images (the transform is linear); each channel keeps its own weights.
//
// Gridding is a deterministic gather: the plan sorts every (channel, baseline)
// contribution by half-plane cell and splits each cell's run into items of at
// most 32 entries; a warp reduces one item with a fixed butterfly and the
// items of a cell are added in order.  One CTA per (sample, subband) image.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "plan_internal.h"

namespace nsfrb {
namespace {

constexpr int kImgThreads = 256;
constexpr double kCLight = 299792458.0;

struct ImgParams {
    const float4 *vis;        // [n_t][n_sub][n_chan * n_base] (pol0 re, pol0 im, pol1 re, pol1 im)
    float *img;               // [n_t][n_sub][N][N]
    const int2 *entries;      // (vis index | conj << 31, weight bits)
    const int2 *items;        // (first entry, count <= 32)
    const int32_t *cell_items;  // [n_sub][n_cells + 1] item ranges per half-plane cell
    const float2 *tab;        // [K + 1][N]: e^{2 pi i k (i + N/2) / N}
    int32_t n_sub, n_cb, N, U, V, K, n_cells, max_items;
    float inv_n2;
};

__global__ void __launch_bounds__(kImgThreads) image_kernel(ImgParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = p.N, U = p.U, V = p.V, nv = 2 * V + 1;
    float2 *s_tab = reinterpret_cast<float2 *>(smem_raw);               // [(K + 1) * N]
    float2 *s_A = s_tab + (size_t)(p.K + 1) * N;                          // [(U + 1) * N]
    float2 *s_G = s_A + (size_t)(U + 1) * N;                              // [n_cells]
    float2 *s_part = s_G + p.n_cells;                                     // [max_items]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int img = blockIdx.x;
    const int sub = img % p.n_sub;
    const float4 *vis = p.vis + (size_t)img * p.n_cb;
    const int32_t *ci = p.cell_items + (size_t)sub * (p.n_cells + 1);
    const int it0 = ci[0], n_it = ci[p.n_cells] - it0;

    for (int i = tid; i < (p.K + 1) * N; i += kImgThreads) s_tab[i] = p.tab[i];

    // ---- gridding, phase 1: one warp per item, several items in flight per warp
    constexpr int kUnroll = 4;
    for (int base = warp * kUnroll; base < n_it; base += (kImgThreads / 32) * kUnroll) {
        float re[kUnroll], im[kUnroll];
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) {
            re[q] = 0.0f;
            im[q] = 0.0f;
            const int it = base + q;
            if (it < n_it) {
                const int2 item = p.items[it0 + it];
                if (lane < item.y) {
                    const int2 e = p.entries[item.x + lane];
                    const float4 v = vis[e.x & 0x7fffffff];
                    const float w = __int_as_float(e.y);
                    re[q] = (v.x + v.z) * w;
                    const float vi = (v.y + v.w) * w;
                    im[q] = (e.x < 0) ? -vi : vi;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                re[q] += __shfl_xor_sync(0xffffffffu, re[q], o);
                im[q] += __shfl_xor_sync(0xffffffffu, im[q], o);
            }
            if (lane == 0 && base + q < n_it) s_part[base + q] = make_float2(re[q], im[q]);
        }
    }
    __syncthreads();
    // ---- gridding, phase 2: the items of each cell in order
    for (int c = tid; c < p.n_cells; c += kImgThreads) {
        float2 g = make_float2(0.0f, 0.0f);
        for (int it = ci[c]; it < ci[c + 1]; ++it) {
            const float2 q = s_part[it - it0];
            g.x += q.x;
            g.y += q.y;
        }
        s_G[c] = g;
    }
    __syncthreads();

    // ---- transform along v: A_u(y) for u = 0..U (consecutive threads: consecutive y)
    for (int q = tid; q < (U + 1) * N; q += kImgThreads) {
        const int u = q / N, y = q - u * N;
        const float2 *g = s_G + u * nv + V;       // g[v], v in [-V, V]
        float2 a = g[0];
        for (int v = 1; v <= V; ++v) {
            const float2 t = s_tab[v * N + y];       // e^{+i theta}; v < 0 uses its conjugate
            const float2 gp = g[v], gm = g[-v];
            a.x += (gp.x + gm.x) * t.x - (gp.y - gm.y) * t.y;
            a.y += (gp.y + gm.y) * t.x + (gp.x - gm.x) * t.y;
        }
        s_A[u * N + y] = a;
    }
    __syncthreads();

    // ---- transform along u to real pixels (consecutive threads: consecutive x)
    float *out = p.img + (size_t)img * N * N;
    for (int q = tid; q < N * N; q += kImgThreads) {
        const int y = q / N, x = q - y * N;
        float acc = 0.0f;
        for (int u = 1; u <= U; ++u) {
            const float2 a = s_A[u * N + y];
            const float2 t = s_tab[u * N + x];
            acc = fmaf(a.x, t.x, acc);
            acc = fmaf(-a.y, t.y, acc);
        }
        out[q] = (s_A[y].x + 2.0f * acc) * p.inv_n2;
    }
}

}  // namespace
}  // namespace nsfrb

using namespace nsfrb;

struct nsfrb_imager_s {
    int32_t N = 0, n_sub = 0, n_chan = 0, n_base = 0;
    int32_t U = 0, V = 0, K = 0, n_cells = 0, max_items = 0;
    int64_t n_entries = 0, n_items = 0;
    std::vector<float> weights;      // [n_sub][n_chan][n_base]
    int2 *d_entries = nullptr, *d_items = nullptr;
    int32_t *d_cell_items = nullptr;
    float2 *d_tab = nullptr;
    size_t smem = 0;
    int device = -1;
};

namespace {

void imager_free(nsfrb_imager_s *im) {
    cudaFree(im->d_entries);
    cudaFree(im->d_items);
    cudaFree(im->d_cell_items);
    cudaFree(im->d_tab);
}

struct Entry {
    int32_t cell;    // half-plane cell (u * (2V + 1) + v + V), filled once U, V are known
    int32_t ku, kv;  // half-plane coordinates (ku >= 0)
    int32_t vis;     // ch * n_base + b, bit 31 = conjugate
    float w;
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
    if (static_cast<int64_t>(c.n_chan) * c.n_base >= (int64_t(1) << 31))
        return fail(nullptr, NSFRB_EINVAL, "n_chan * n_base too large");
    for (int64_t i = 0; i < 2LL * c.n_base; ++i)
        if (!std::isfinite(c.uv_m[i])) return fail(nullptr, NSFRB_EINVAL, "non-finite uv");
    for (int64_t i = 0; i < static_cast<int64_t>(c.n_sub) * c.n_chan; ++i)
        if (!(c.chan_mhz[i] > 0.0) || !std::isfinite(c.chan_mhz[i]))
            return fail(nullptr, NSFRB_EINVAL, "channel frequencies must be > 0");

    auto *im = new nsfrb_imager_s();
    const int N = c.n_grid, h = (N - 1) / 2, ctr = N / 2;
    im->N = N;
    im->n_sub = c.n_sub;
    im->n_chan = c.n_chan;
    im->n_base = c.n_base;
    im->weights.assign(static_cast<size_t>(c.n_sub) * c.n_chan * c.n_base, 0.0f);
    const double dth = c.pixel_arcsec * M_PI / 648000.0;

    std::vector<uint8_t> kept(c.n_base);
    for (int b = 0; b < c.n_base; ++b) {
        const double u = c.uv_m[2 * b], v = c.uv_m[2 * b + 1];
        const double len = std::sqrt(u * u + v * v);
        kept[b] = len > c.b_min_m && len < c.b_max_m;
    }
    std::vector<std::vector<Entry>> per_sub(c.n_sub);
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
            for (int b = 0; b < c.n_base; ++b) {
                if (!ok[b]) continue;
                const double wd = 1.0 / (1.0 + W[static_cast<size_t>(ctr + kv[b]) * N + ctr + ku[b]] * f2);
                const float w = static_cast<float>(wd);
                im->weights[(static_cast<size_t>(s) * c.n_chan + ch) * c.n_base + b] = w;
                const int32_t idx = ch * c.n_base + b;
                auto add = [&](int32_t a, int32_t bb, bool conj) {
                    per_sub[s].push_back(Entry{0, a, bb, conj ? static_cast<int32_t>(idx | 0x80000000u) : idx, w});
                    U = std::max(U, a);
                    V = std::max(V, std::abs(bb));
                };
                if (ku[b] > 0) add(ku[b], kv[b], false);
                else if (ku[b] < 0) add(-ku[b], -kv[b], true);
                else {
                    add(0, kv[b], false);
                    add(0, -kv[b], true);
                }
            }
        }
    }
    im->U = U;
    im->V = V;
    im->K = std::max(U, V);
    const int nv = 2 * V + 1;
    im->n_cells = (U + 1) * nv;

    // sort each subband's entries by cell (stable: channel, baseline, conjugate order within a cell)
    std::vector<int2> entries, items;
    std::vector<int32_t> cell_items;
    cell_items.reserve(static_cast<size_t>(c.n_sub) * (im->n_cells + 1));
    for (int s = 0; s < c.n_sub; ++s) {
        auto &es = per_sub[s];
        for (auto &e : es) e.cell = e.ku * nv + e.kv + V;
        std::stable_sort(es.begin(), es.end(), [](const Entry &a, const Entry &b) { return a.cell < b.cell; });
        size_t i = 0;
        int n_items_s = 0;
        for (int cell = 0; cell < im->n_cells; ++cell) {
            cell_items.push_back(static_cast<int32_t>(items.size()));
            while (i < es.size() && es[i].cell == cell) {
                const size_t first = entries.size();
                int cnt = 0;
                while (i < es.size() && es[i].cell == cell && cnt < 32) {
                    int32_t wbits;
                    std::memcpy(&wbits, &es[i].w, 4);
                    entries.push_back(make_int2(es[i].vis, wbits));
                    ++i;
                    ++cnt;
                }
                items.push_back(make_int2(static_cast<int32_t>(first), cnt));
                ++n_items_s;
            }
        }
        cell_items.push_back(static_cast<int32_t>(items.size()));
        im->max_items = std::max(im->max_items, n_items_s);
    }
    im->n_entries = static_cast<int64_t>(entries.size());
    im->n_items = static_cast<int64_t>(items.size());
    if (im->n_entries >= (int64_t(1) << 31)) {
        delete im;
        return fail(nullptr, NSFRB_EINVAL, "too many gridding entries");
    }

    // e^{2 pi i k (i + N/2) / N} for k = 0..K, i = 0..N-1, from the exact index (k (i + N/2)) mod N
    std::vector<float2> tab(static_cast<size_t>(im->K + 1) * N);
    for (int k = 0; k <= im->K; ++k)
        for (int i = 0; i < N; ++i) {
            const int64_t j = (static_cast<int64_t>(k) * ((i + ctr) % N)) % N;
            const double a = 2.0 * M_PI * static_cast<double>(j) / N;
            tab[static_cast<size_t>(k) * N + i] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
        }
    im->smem = sizeof(float2) * (tab.size() + static_cast<size_t>(U + 1) * N + im->n_cells + im->max_items);

    nsfrb_status st = NSFRB_OK;
    int max_smem = 0;
    if ((st = cuda_check(nullptr, cudaGetDevice(&im->device), "device")) ||
        (st = cuda_check(nullptr, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, im->device),
                         "attribute"))) {
        delete im;
        return st;
    }
    if (im->smem > static_cast<size_t>(max_smem)) {
        delete im;
        return fail(nullptr, NSFRB_EINVAL, "uv support too large for one CTA's shared memory");
    }
    auto up = [&](void **dst, const void *src, size_t bytes) -> nsfrb_status {
        nsfrb_status s2 = cuda_check(nullptr, cudaMalloc(dst, std::max<size_t>(bytes, 16)), "cudaMalloc");
        if (s2 == NSFRB_OK && bytes)
            s2 = cuda_check(nullptr, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice), "copy");
        return s2;
    };
    if ((st = up(reinterpret_cast<void **>(&im->d_entries), entries.data(), sizeof(int2) * entries.size())) ||
        (st = up(reinterpret_cast<void **>(&im->d_items), items.data(), sizeof(int2) * items.size())) ||
        (st = up(reinterpret_cast<void **>(&im->d_cell_items), cell_items.data(), sizeof(int32_t) * cell_items.size())) ||
        (st = up(reinterpret_cast<void **>(&im->d_tab), tab.data(), sizeof(float2) * tab.size())) ||
        (st = cuda_check(nullptr, cudaFuncSetAttribute(image_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      static_cast<int>(im->smem)), "smem attribute"))) {
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
    if (n_img >= (int64_t(1) << 31)) return fail(nullptr, NSFRB_EINVAL, "too many images");
    ImgParams p;
    p.vis = reinterpret_cast<const float4 *>(d_vis);
    p.img = d_img;
    p.entries = im->d_entries;
    p.items = im->d_items;
    p.cell_items = im->d_cell_items;
    p.tab = im->d_tab;
    p.n_sub = im->n_sub;
    p.n_cb = im->n_chan * im->n_base;
    p.N = im->N;
    p.U = im->U;
    p.V = im->V;
    p.K = im->K;
    p.n_cells = im->n_cells;
    p.max_items = im->max_items;
    p.inv_n2 = static_cast<float>(1.0 / (static_cast<double>(im->N) * im->N));
    image_kernel<<<static_cast<unsigned>(n_img), kImgThreads, im->smem, static_cast<cudaStream_t>(stream)>>>(p);
    return cuda_check(nullptr, cudaGetLastError(), "image launch");
}

void nsfrb_imager_destroy(nsfrb_imager_t im) {
    if (!im) return;
    imager_free(im);
    delete im;
}

}  // extern "C"
