// Host side of libnsfrb: configuration checks, the integer delay table of
// arXiv 2510.18136 Sec. 2.2 (shift indices pre-computed once per plan and
// loaded onto the GPU), the merged-row tables the search kernel walks, device
// workspace, and the search / result entry points of include/nsfrb.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nsfrb.h"
#include "nsfrb_internal.h"
#include "plan_internal.h"

using namespace nsfrb;

namespace {
thread_local std::string g_last_error;
}

namespace nsfrb {

void set_error(const std::string &msg) { g_last_error = msg; }

nsfrb_status fail(nsfrb_plan_s *p, nsfrb_status st, const std::string &msg) {
    set_error(msg);
    if (p && st == NSFRB_ECUDA && p->latched == NSFRB_OK) p->latched = st;
    return st;
}

nsfrb_status cuda_check(nsfrb_plan_s *p, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return NSFRB_OK;
    return fail(p, NSFRB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

cudaError_t launch_search(int C, const SearchParams &p, int grid, size_t smem, cudaStream_t s) {
    switch (C) {
        case 1: return launch_search_c1(p, grid, smem, s);
        case 3: return launch_search_c3(p, grid, smem, s);
        case 5: return launch_search_c5(p, grid, smem, s);
        case 9: return launch_search_c9(p, grid, smem, s);
        case 17: return launch_search_c17(p, grid, smem, s);
        case 25: return launch_search_c25(p, grid, smem, s);
        case 38: return launch_search_c38(p, grid, smem, s);
        case 39: return launch_search_c39(p, grid, smem, s);
        case kLongC: return launch_search_long(p, grid, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_search(int C, size_t smem) {
    switch (C) {
        case 1: return prepare_search_c1(smem);
        case 3: return prepare_search_c3(smem);
        case 5: return prepare_search_c5(smem);
        case 9: return prepare_search_c9(smem);
        case 17: return prepare_search_c17(smem);
        case 25: return prepare_search_c25(smem);
        case 38: return prepare_search_c38(smem);
        case 39: return prepare_search_c39(smem);
        case kLongC: return prepare_search_long(smem);
        default: return cudaErrorInvalidValue;
    }
}

size_t elem_size(int dtype) { return dtype == NSFRB_F32 ? 4 : 2; }

// Fill the parts of SearchParams that depend only on the plan.
void base_params(const nsfrb_plan_s *pl, SearchParams &sp) {
    std::memset(&sp, 0, sizeof(sp));
    const nsfrb_config &c = pl->cfg;
    sp.n_sub = c.n_sub;
    sp.n_t = c.n_t;
    sp.Tp = pl->Tp;
    sp.noise_mode = c.noise_mode;
    sp.sigma_default = std::sqrt(static_cast<float>(c.n_sub));
    sp.n_u = pl->n_u;
    sp.n_u_active = pl->n_u_active;
    sp.table = pl->d_table;
    sp.n_deltas = pl->n_deltas;
    sp.n_w = c.n_w;
    for (int j = 0; j < kPow2; ++j) sp.pow2_wi[j] = -1;
    for (int i = 0; i < c.n_w; ++i) {
        sp.widths[i] = pl->widths[i];
        sp.wclass[i] = pl->wclass[i];
        const int w = pl->widths[i];
        int j = -1;
        for (int q = 0; q < kPow2; ++q)
            if (w == (1 << q)) j = q;
        if (pl->wclass[i] != WC_GENERIC && j >= 0) {
            sp.pow2_wi[j] = i;
            sp.has_small |= pl->wclass[i] == WC_SMALL;
            sp.has_large |= pl->wclass[i] == WC_LARGE;
        } else {
            sp.gen_wi[sp.n_gen++] = i;
        }
    }
    sp.n_dm = c.n_dm;
    sp.rec = pl->d_rec;
    sp.err = pl->d_err;
    if (c.out_mode == NSFRB_OUT_FULL) {
        sp.full_snr = pl->d_full_snr;
        sp.full_t = pl->d_full_t;
    }
}

// Choose the staging scheme for a cube pointer / row geometry and size the
// shared memory (chunk size C, the device's per-block limit).  Returns false if nothing fits.
// the compiled (teams, buffers per team) tiles of the barrier-free kernel, coded 10 * teams + buffers
const int kTileCodes[NSFRB_N_TILES] = {NSFRB_TILES};
bool tile_is_known(int t) {
    for (const int k : kTileCodes)
        if (k == t) return true;
    return false;
}

bool choose_stage_for(int C, int max_smem, SearchParams &sp, size_t &smem, int tile_pref) {
    if (C == kLongC) {
        // windows beyond the register path: the long-window kernel reads the cube in place; its
        // CTA takes as many warps as their prefix rows fit (the warp count travels in sp.teams)
        sp.pipe = 0;
        sp.stage = 0;
        const int w = long_warps(sp, max_smem);
        if (w < 1) return false;
        sp.teams = w;
        smem = long_smem(sp, w);
        return true;
    }
    const uintptr_t base = reinterpret_cast<uintptr_t>(sp.cube);
    const int n_t = sp.n_t;
    const int epv = 16 / static_cast<int>(elem_size(sp.dtype));   // samples per 16 bytes
    // The barrier-free kernel: rows bulk-copied as stored (FP32, or 16-bit read in place, which
    // needs the sample-pair path of even chunks), KNOWN noise (or MAD-normalised FP32 slabs), records
    // and FULL arrays.  The copy starts at the 16-byte boundary at or below the window start and must
    // stay inside the row.
    if (sp.t_wrap == 0 && sp.t_stride == 0 && sp.noise_mode == 0 &&
        (sp.dtype == NSFRB_F32 || C % 2 == 0) &&
        base % 16 == 0 && sp.row_len % epv == 0) {
        bool fits_row;
        if (sp.t_off_dev)   // a ring row: the window start is below n_t, the row 2 n_t + 8 long
            fits_row = sp.row_len >= 2 * static_cast<int64_t>(n_t) + 8;
        else
            fits_row = (sp.t_off - sp.t_off % epv) + static_cast<int64_t>(align_up(sp.t_off % epv + n_t, epv)) <=
                       sp.row_len;
        // odd chunks read one sample at a time without the tail mask: the copied window must be exact
        const bool exact = !sp.t_off_dev && sp.t_off % epv == 0 && n_t % epv == 0;
        if (fits_row && (C % 2 == 0 || exact)) {
            sp.stage = (sp.dtype == NSFRB_F32) ? 1 : 3;
            sp.stg_pitch = 0;
            sp.pipe = 1;
            // pixel x DM tile: the preferred one where it fits, else the most teams that fit (each
            // team on its own pixel, fewer row groups per pixel to build from scratch and more rows
            // per warp between pixel changes): four, three or two teams of one buffer (two teams of
            // two buffers before two of one), then one team of two buffers
            const int kTiles[6] = {tile_pref, 41, 31, 22, 21, 12};
            for (const int t : kTiles) {
                if (!tile_is_known(t)) continue;
                sp.teams = t / 10;
                sp.nb = t % 10;
                const SmemLayout L = smem_layout(sp, C);
                if (L.total <= static_cast<size_t>(max_smem)) {
                    smem = L.total;
                    return true;
                }
            }
        }
        sp.teams = 1;
        sp.nb = 2;
    }
    sp.pipe = 0;
    int want = 0;
    if (sp.t_wrap > 0 || sp.t_stride > 0) {
        want = 0;   // ring rows or sample-major cubes: plain loads
    } else if (sp.dtype == NSFRB_F32) {
        // bulk copies start at the window start: 16-byte aligned only if it is a multiple of 4
        // samples.  A window start kept on the device (serving) moves by new_blk per block.
        const bool start_aligned = sp.t_off_dev ? (sp.new_blk > 0 && sp.new_blk % 4 == 0) : (sp.t_off % 4 == 0);
        if (base % 16 == 0 && n_t % 4 == 0 && sp.row_len % 4 == 0 && start_aligned) want = 1;
    } else {
        if (base % 16 == 0 && sp.row_len % 8 == 0 &&
            (sp.t_off_dev ? sp.row_len >= 2 * static_cast<int64_t>(n_t) + 8 : sp.t_off + n_t <= sp.row_len))
            want = 2;
    }
    for (int st = want; st >= 0; st = (st == 2 ? 0 : st - 1)) {
        sp.stage = st;
        sp.stg_pitch = (st == 2) ? static_cast<int32_t>(align_up(static_cast<size_t>(7 + n_t) * 2, 16)) : 0;
        const SmemLayout L = smem_layout(sp, C);
        if (L.total <= static_cast<size_t>(max_smem)) {
            smem = L.total;
            return true;
        }
        if (st == 0) break;
    }
    return false;
}

bool choose_stage(const nsfrb_plan_s *pl, SearchParams &sp, size_t &smem) {
    return choose_stage_for(pl->C, pl->max_smem, sp, smem, pl->tile[sp.dtype]);
}

// records which tile the search launch of `sp` takes
void note_tile(nsfrb_plan_s *pl, const SearchParams &sp) {
    pl->last_tile = sp.pipe ? 10 * sp.teams + sp.nb : 0;
    pl->last_tile_st = sp.dtype;
}

nsfrb_status ensure_device(nsfrb_plan_s *pl) {
    if (pl->latched != NSFRB_OK) return fail(pl, pl->latched, "plan has a latched CUDA error");
    if (pl->dev_ready) return NSFRB_OK;
    nsfrb_status st;
    if ((st = cuda_check(pl, cudaGetDevice(&pl->device), "cudaGetDevice")) != NSFRB_OK) return st;
    if ((st = cuda_check(pl, cudaDeviceGetAttribute(&pl->n_sm, cudaDevAttrMultiProcessorCount, pl->device),
                         "sm count")) != NSFRB_OK)
        return st;
    if ((st = cuda_check(pl,
                         cudaDeviceGetAttribute(&pl->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                                pl->device),
                         "smem limit")) != NSFRB_OK)
        return st;
    const nsfrb_config &c = pl->cfg;
    const int64_t n_pix = static_cast<int64_t>(c.ny) * c.nx;
    pl->n_blocks = static_cast<int32_t>((n_pix + kCompactBlock - 1) / kCompactBlock);
    auto alloc = [&](void **ptr, size_t bytes, const char *what) -> nsfrb_status {
        cudaError_t e = cudaMalloc(ptr, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(pl, NSFRB_ENOMEM, std::string("cudaMalloc ") + what);
        }
        return NSFRB_OK;
    };
    if ((st = alloc(reinterpret_cast<void **>(&pl->d_table), pl->table.size() * sizeof(int32_t), "table")) ||
        (st = alloc(reinterpret_cast<void **>(&pl->d_rec), n_pix * sizeof(PixRec), "records")) ||
        (st = alloc(reinterpret_cast<void **>(&pl->d_cand), n_pix * sizeof(CandRec), "candidates")) ||
        (st = alloc(reinterpret_cast<void **>(&pl->d_counts), (pl->n_blocks + 4) * sizeof(int32_t), "counts")) ||
        (st = alloc(reinterpret_cast<void **>(&pl->d_list), n_pix * sizeof(int32_t), "list")))
        return st;
    pl->d_err = pl->d_counts + pl->n_blocks;
    pl->d_ncand = pl->d_counts + pl->n_blocks + 1;
    pl->d_nlist = pl->d_counts + pl->n_blocks + 2;
    if (c.out_mode == NSFRB_OUT_FULL) {
        const size_t n = static_cast<size_t>(n_pix) * c.n_dm * c.n_w;
        if ((st = alloc(reinterpret_cast<void **>(&pl->d_full_snr), n * sizeof(float), "full S/N")) ||
            (st = alloc(reinterpret_cast<void **>(&pl->d_full_t), n * sizeof(int16_t), "full t")))
            return st;
    }
    if ((st = cuda_check(pl,
                         cudaMemcpy(pl->d_table, pl->table.data(), pl->table.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice),
                         "table upload")) != NSFRB_OK)
        return st;
    if ((st = cuda_check(pl, cudaMemset(pl->d_counts, 0, (pl->n_blocks + 4) * sizeof(int32_t)), "memset")))
        return st;
    if ((st = cuda_check(pl, prepare_search(pl->C, pl->max_smem), "smem attribute")) != NSFRB_OK) return st;
    if ((st = cuda_check(pl, cudaEventCreateWithFlags(&pl->done, cudaEventDisableTiming), "event")) ||
        (st = cuda_check(pl, cudaEventCreate(&pl->t_start), "event")) ||
        (st = cuda_check(pl, cudaEventCreate(&pl->t_search), "event")) ||
        (st = cuda_check(pl, cudaEventCreate(&pl->t_end), "event")))
        return st;
    pl->dev_ready = true;
    return NSFRB_OK;
}

// Queue search kernel(s) over pixels [pix0, pix0 + n) of the cube on stream s.
nsfrb_status queue_search(nsfrb_plan_s *pl, const void *cube, int64_t cube_pix0, int dtype, int64_t row_len,
                          int t_off, const float *sigma, int64_t pix0, int64_t n, const int32_t *pix_list,
                          const int32_t *n_items_dev, int new_blk, cudaStream_t s, const int32_t *t_off_dev,
                          int t_wrap, int64_t t_stride) {
    SearchParams sp;
    base_params(pl, sp);
    sp.cube = cube;
    sp.cube_pix0 = cube_pix0;
    sp.dtype = dtype;
    sp.row_len = row_len;
    sp.t_off = t_off;
    sp.t_off_dev = t_off_dev;
    sp.t_wrap = t_wrap;
    sp.t_stride = t_stride;
    sp.sigma = sigma;
    sp.pix0 = pix0;
    sp.n_items = n;
    sp.pix_list = pix_list;
    sp.n_items_dev = n_items_dev;
    sp.new_blk = new_blk;
    size_t smem = 0;
    if (!choose_stage(pl, sp, smem)) return fail(pl, NSFRB_EINVAL, "shared memory does not fit this plan");
    note_tile(pl, sp);
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(n, pl->n_sm)));
    return cuda_check(pl, launch_search(pl->C, sp, grid, smem, s), "search launch");
}

// MAD mode with per-pixel records: the median / MAD normalisation as a pass of its own, slab by
// slab of pixels into an FP32 workspace, each slab then searched by the barrier-free kernel with
// unit noise per sample (sigma_D = sqrt(n_sub)); pixels with a zero-MAD row get invalid records.
// Returns false (nothing queued) where this does not apply: FULL output, or windows whose FP32
// rows do not fill whole 16-byte units.
bool mad_slabs_apply(const nsfrb_plan_s *pl) {
    const nsfrb_config &c = pl->cfg;
    if (c.noise_mode != NSFRB_NOISE_MAD) return false;
    // in either output mode; long windows always (their kernel has no in-kernel selection), other
    // windows when the FP32 slab rows fill whole 16-byte units (the barrier-free kernel's copies)
    return pl->C == kLongC || c.n_t % 4 == 0;
}

nsfrb_status queue_search_mad(nsfrb_plan_s *pl, const void *cube, int dtype, int64_t pix0, int64_t n,
                              cudaStream_t s) {
    const nsfrb_config &c = pl->cfg;
    const int64_t n_pix = static_cast<int64_t>(c.ny) * c.nx;
    nsfrb_status st;
    if (!pl->d_madws) {
        const size_t pix_bytes = sizeof(float) * static_cast<size_t>(c.n_sub) * c.n_t;
        pl->mad_slab = std::min<int64_t>(n_pix, std::max<int64_t>(1, (int64_t(2) << 30) / static_cast<int64_t>(pix_bytes)));
        if (cudaMalloc(reinterpret_cast<void **>(&pl->d_madws), pix_bytes * pl->mad_slab) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void **>(&pl->d_bad), static_cast<size_t>(n_pix)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(pl->d_madws);
            pl->d_madws = nullptr;
            return fail(pl, NSFRB_ENOMEM, "cudaMalloc MAD normalisation workspace");
        }
    }
    if ((st = cuda_check(pl, cudaMemsetAsync(pl->d_bad + pix0, 0, static_cast<size_t>(n), s), "memset"))) return st;
    for (int64_t p0 = pix0; p0 < pix0 + n; p0 += pl->mad_slab) {
        const int64_t m = std::min<int64_t>(pl->mad_slab, pix0 + n - p0);
        if ((st = cuda_check(pl,
                             launch_mad_normalise(cube, dtype, p0, m, c.n_sub, c.n_t, pl->d_madws, pl->d_bad,
                                                  pl->n_sm, s),
                             "MAD normalisation")) != NSFRB_OK)
            return st;
        SearchParams sp;
        base_params(pl, sp);
        sp.noise_mode = NSFRB_NOISE_KNOWN;   // the slab holds normalised samples of unit noise
        sp.bad_pix = pl->d_bad;
        sp.cube = pl->d_madws;
        sp.cube_pix0 = p0;
        sp.dtype = NSFRB_F32;
        sp.row_len = c.n_t;
        sp.pix0 = p0;
        sp.n_items = m;
        size_t smem = 0;
        if (!choose_stage(pl, sp, smem)) return fail(pl, NSFRB_EINVAL, "shared memory does not fit this plan");
        note_tile(pl, sp);
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(m, pl->n_sm)));
        if ((st = cuda_check(pl, launch_search(pl->C, sp, grid, smem, s), "search launch")) != NSFRB_OK) return st;
    }
    return NSFRB_OK;
}

nsfrb_status queue_finish(nsfrb_plan_s *pl, cudaStream_t s) {
    const nsfrb_config &c = pl->cfg;
    const int64_t n_pix = static_cast<int64_t>(c.ny) * c.nx;
    nsfrb_status st = cuda_check(pl, cudaEventRecord(pl->t_search, s), "event");
    if (st != NSFRB_OK) return st;
    st = cuda_check(pl,
                                 launch_compact(pl->d_rec, n_pix, c.nx, c.threshold, pl->d_counts, pl->n_blocks,
                                                pl->d_cand, pl->d_ncand, s),
                                 "compaction");
    if (st != NSFRB_OK) return st;
    if ((st = cuda_check(pl, cudaEventRecord(pl->done, s), "event record")) != NSFRB_OK) return st;
    if ((st = cuda_check(pl, cudaEventRecord(pl->t_end, s), "event record")) != NSFRB_OK) return st;
    pl->searched = true;
    return NSFRB_OK;
}

nsfrb_status wait_done(nsfrb_plan_s *pl) {
    if (pl->latched != NSFRB_OK) return fail(pl, pl->latched, "plan has a latched CUDA error");
    if (!pl->searched) return fail(pl, NSFRB_ENOTREADY, "no search has been run on this plan");
    return cuda_check(pl, cudaEventSynchronize(pl->done), "wait for search");
}

}  // namespace nsfrb

// ============================================================================ C ABI

extern "C" {

const char *nsfrb_strerror(nsfrb_status s) {
    switch (s) {
        case NSFRB_OK: return "ok";
        case NSFRB_EINVAL: return "invalid argument";
        case NSFRB_ENOMEM: return "out of memory";
        case NSFRB_ECUDA: return "CUDA error";
        case NSFRB_ETIMEOUT: return "timed out";
        case NSFRB_ETRUNC: return "output truncated";
        case NSFRB_ENOTREADY: return "not ready";
    }
    return "unknown status";
}

const char *nsfrb_last_error(void) { return g_last_error.c_str(); }

nsfrb_status nsfrb_plan(const nsfrb_config *cfg, nsfrb_plan_t *out) {
    if (!cfg || !out) return fail(nullptr, NSFRB_EINVAL, "null argument");
    *out = nullptr;
    const nsfrb_config &c = *cfg;
    if (c.ny < 1 || c.nx < 1) return fail(nullptr, NSFRB_EINVAL, "ny, nx must be >= 1");
    if (static_cast<int64_t>(c.ny) * c.nx > (int64_t(1) << 30)) return fail(nullptr, NSFRB_EINVAL, "too many pixels");
    if (c.n_sub < 1 || c.n_sub > kMaxSub) return fail(nullptr, NSFRB_EINVAL, "n_sub must be 1..32");
    if (c.n_t < 1 || c.n_t > kMaxT) return fail(nullptr, NSFRB_EINVAL, "n_t must be 1..4096");
    if (!(c.t_samp_ms > 0.0) || !(c.k_dm_ms >= 0.0)) return fail(nullptr, NSFRB_EINVAL, "t_samp_ms, k_dm_ms");
    if (!c.freq_mhz || !c.dm || !c.widths) return fail(nullptr, NSFRB_EINVAL, "null table");
    if (c.n_dm < 1 || c.n_dm > 4096) return fail(nullptr, NSFRB_EINVAL, "n_dm must be 1..4096");
    if (c.n_w < 1 || c.n_w > kMaxW) return fail(nullptr, NSFRB_EINVAL, "n_w must be 1..16");
    if (c.dtype < NSFRB_F32 || c.dtype > NSFRB_F16) return fail(nullptr, NSFRB_EINVAL, "dtype");
    if (c.noise_mode < 0 || c.noise_mode > 1) return fail(nullptr, NSFRB_EINVAL, "noise_mode");
    if (c.out_mode < 0 || c.out_mode > 1) return fail(nullptr, NSFRB_EINVAL, "out_mode");
    if (!std::isfinite(c.threshold)) return fail(nullptr, NSFRB_EINVAL, "threshold");
    for (int k = 0; k < c.n_sub; ++k) {
        if (!(c.freq_mhz[k] > 0.0) || !std::isfinite(c.freq_mhz[k]))
            return fail(nullptr, NSFRB_EINVAL, "frequencies must be positive");
        if (k > 0 && !(c.freq_mhz[k] > c.freq_mhz[k - 1]))
            return fail(nullptr, NSFRB_EINVAL, "frequencies must be strictly increasing");
    }
    for (int d = 0; d < c.n_dm; ++d) {
        if (!(c.dm[d] >= 0.0) || !std::isfinite(c.dm[d])) return fail(nullptr, NSFRB_EINVAL, "DM must be >= 0");
        if (d > 0 && c.dm[d] < c.dm[d - 1]) return fail(nullptr, NSFRB_EINVAL, "DMs must be nondecreasing");
    }
    for (int i = 0; i < c.n_w; ++i) {
        if (c.widths[i] < 1 || c.widths[i] > c.n_t) return fail(nullptr, NSFRB_EINVAL, "widths must be 1..n_t");
        if (i > 0 && c.widths[i] <= c.widths[i - 1])
            return fail(nullptr, NSFRB_EINVAL, "widths must be strictly increasing");
    }

    nsfrb_plan_s *pl = new (std::nothrow) nsfrb_plan_s();
    if (!pl) return fail(nullptr, NSFRB_ENOMEM, "plan allocation");
    pl->cfg = c;
    pl->freq.assign(c.freq_mhz, c.freq_mhz + c.n_sub);
    pl->dm.assign(c.dm, c.dm + c.n_dm);
    pl->widths.assign(c.widths, c.widths + c.n_w);
    pl->cfg.freq_mhz = pl->freq.data();
    pl->cfg.dm = pl->dm.data();
    pl->cfg.widths = pl->widths.data();

    // Delay table (Sec. 2.2), FP64, reference = highest subband centre.
    const int n_sub = c.n_sub, n_dm = c.n_dm;
    const double ftop = pl->freq[n_sub - 1] / 1000.0;
    pl->shifts.resize(static_cast<size_t>(n_dm) * n_sub);
    pl->smax.resize(n_dm);
    for (int d = 0; d < n_dm; ++d) {
        int32_t mx = 0;
        for (int k = 0; k < n_sub; ++k) {
            const double f = pl->freq[k] / 1000.0;
            const double delay_ms = c.k_dm_ms * pl->dm[d] * (1.0 / (f * f) - 1.0 / (ftop * ftop));
            const double v = std::floor(delay_ms / c.t_samp_ms + 0.5);
            if (!(v < 8191.0)) {
                delete pl;
                return fail(nullptr, NSFRB_EINVAL, "dispersion shift exceeds 8191 samples");
            }
            const int32_t s = static_cast<int32_t>(v);
            pl->shifts[static_cast<size_t>(d) * n_sub + k] = s;
            mx = std::max(mx, s);
        }
        pl->smax[d] = mx;
    }

    // Merge consecutive identical rows (sorted DMs make identical rows adjacent).
    std::vector<int> first_d, n_d;
    for (int d = 0; d < n_dm; ++d) {
        const bool same = d > 0 && std::memcmp(&pl->shifts[static_cast<size_t>(d) * n_sub],
                                               &pl->shifts[static_cast<size_t>(d - 1) * n_sub],
                                               sizeof(int32_t) * n_sub) == 0;
        if (same) {
            ++n_d.back();
        } else {
            first_d.push_back(d);
            n_d.push_back(1);
        }
    }
    pl->n_u = static_cast<int>(first_d.size());
    pl->n_u_active = 0;
    std::vector<int32_t> info(static_cast<size_t>(pl->n_u) * kInfo), deltas;
    for (int u = 0; u < pl->n_u; ++u) {
        const int d = first_d[u];
        const int32_t *s = &pl->shifts[static_cast<size_t>(d) * n_sub];
        info[u * kInfo + UI_SMAX] = pl->smax[d];
        info[u * kInfo + UI_FIRST_D] = d;
        info[u * kInfo + UI_N_D] = n_d[u];
        info[u * kInfo + UI_DOFF] = static_cast<int32_t>(deltas.size());
        if (pl->smax[d] < c.n_t) pl->n_u_active = u + 1;
        if (u > 0) {
            const int32_t *sp = &pl->shifts[static_cast<size_t>(first_d[u - 1]) * n_sub];
            for (int k = 0; k < n_sub; ++k)
                if (s[k] != sp[k])
                    deltas.push_back(static_cast<int32_t>(static_cast<uint32_t>(k) |
                                                          (static_cast<uint32_t>(sp[k]) << 6) |
                                                          (static_cast<uint32_t>(s[k]) << 19)));
        }
        info[u * kInfo + UI_ND] = static_cast<int32_t>(deltas.size()) - info[u * kInfo + UI_DOFF];
    }
    pl->n_deltas = static_cast<int32_t>(deltas.size());
    pl->table = info;
    pl->table.insert(pl->table.end(), deltas.begin(), deltas.end());
    for (int u = 0; u < pl->n_u; ++u)
        for (int k = 0; k < n_sub; ++k)
            pl->table.push_back(pl->shifts[static_cast<size_t>(first_d[u]) * n_sub + k]);

    // Kernel geometry.
    pl->C = pick_chunk(c.n_t);
    int smax_active = 0;
    for (int u = 0; u < pl->n_u_active; ++u) smax_active = std::max(smax_active, info[u * kInfo + UI_SMAX]);
    // a row holds the window from element eoff < 8 (a window start below a 16-byte boundary) up to
    // the last sample a lane chunk reads, 32 C + smax - 1, and one more
    const bool long_window = pl->C == kLongC;
    pl->Tp = long_window ? 0 : static_cast<int>(align_up(static_cast<size_t>(32 * pl->C + smax_active + 1 + 7), 8));
    for (int i = 0; i < c.n_w; ++i) {
        const int w = pl->widths[i];
        pl->wclass[i] = WC_GENERIC;
        if (!long_window)
            for (int j = 0; j < kPow2; ++j)
                if (w == (1 << j)) pl->wclass[i] = pow2_class(pl->C, j);
    }
    // The plan must fit at least the plain staging scheme in 227 KB.
    {
        SearchParams sp;
        std::memset(&sp, 0, sizeof(sp));
        sp.n_sub = c.n_sub;
        sp.n_t = c.n_t;
        sp.Tp = pl->Tp;
        sp.n_u = pl->n_u;
        sp.n_deltas = pl->n_deltas;
        sp.noise_mode = c.noise_mode;
        sp.stage = 0;
        if (long_window ? long_smem(sp, 1) > 232448 : smem_layout(sp, pl->C).total > 232448) {
            delete pl;
            return fail(nullptr, NSFRB_EINVAL, "plan tables and window do not fit in shared memory");
        }
    }
    *out = pl;
    return NSFRB_OK;
}

nsfrb_status nsfrb_plan_delays(nsfrb_plan_t plan, int32_t *h_shifts) {
    if (!plan || !h_shifts) return fail(plan, NSFRB_EINVAL, "null argument");
    std::memcpy(h_shifts, plan->shifts.data(), plan->shifts.size() * sizeof(int32_t));
    return NSFRB_OK;
}

nsfrb_status nsfrb_plan_info(nsfrb_plan_t plan, int32_t *n_unique, int32_t *h_smax) {
    if (!plan) return fail(plan, NSFRB_EINVAL, "null plan");
    if (n_unique) *n_unique = plan->n_u;
    if (h_smax) std::memcpy(h_smax, plan->smax.data(), plan->smax.size() * sizeof(int32_t));
    return NSFRB_OK;
}

nsfrb_status nsfrb_search(nsfrb_plan_t plan, const void *d_cube, const float *d_sigma, const void *d_cube_f32,
                          void *stream) {
    if (!plan || !d_cube) return fail(plan, NSFRB_EINVAL, "null argument");
    const nsfrb_config &c = plan->cfg;
    if (c.noise_mode == NSFRB_NOISE_MAD && d_sigma)
        return fail(plan, NSFRB_EINVAL, "d_sigma must be NULL in MAD mode");
    nsfrb_status st = ensure_device(plan);
    if (st != NSFRB_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n_pix = static_cast<int64_t>(c.ny) * c.nx;
    if ((st = cuda_check(plan, cudaMemsetAsync(plan->d_err, 0, sizeof(int32_t), s), "memset")) != NSFRB_OK)
        return st;
    if ((st = cuda_check(plan, cudaEventRecord(plan->t_start, s), "event")) != NSFRB_OK) return st;
    if (mad_slabs_apply(plan))
        st = queue_search_mad(plan, d_cube, c.dtype, 0, n_pix, s);
    else
        st = queue_search(plan, d_cube, 0, c.dtype, c.n_t, 0, d_sigma, 0, n_pix, nullptr, nullptr, 0, s);
    if (st != NSFRB_OK) return st;
    if (c.dtype != NSFRB_F32 && d_cube_f32 && c.rescore_eps > 0.0f) {
        if ((st = cuda_check(plan,
                             launch_rescore_select(plan->d_rec, n_pix, c.threshold, c.rescore_eps, plan->d_list,
                                                   plan->d_nlist, s),
                             "re-score select")) != NSFRB_OK)
            return st;
        if ((st = queue_search(plan, d_cube_f32, 0, NSFRB_F32, c.n_t, 0, d_sigma, 0, n_pix, plan->d_list,
                               plan->d_nlist, 0, s)) != NSFRB_OK)
            return st;
    }
    return queue_finish(plan, s);
}

nsfrb_status nsfrb_search_host(nsfrb_plan_t plan, const void *h_cube, const float *h_sigma, void *stream) {
    if (!plan || !h_cube) return fail(plan, NSFRB_EINVAL, "null argument");
    const nsfrb_config &c = plan->cfg;
    if (c.noise_mode == NSFRB_NOISE_MAD && h_sigma)
        return fail(plan, NSFRB_EINVAL, "h_sigma must be NULL in MAD mode");
    nsfrb_status st = ensure_device(plan);
    if (st != NSFRB_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n_pix = static_cast<int64_t>(c.ny) * c.nx;
    const size_t pix_bytes = static_cast<size_t>(c.n_sub) * c.n_t * elem_size(c.dtype);
    if (!plan->d_hcube) {
        if (cudaMalloc(&plan->d_hcube, pix_bytes * n_pix) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void **>(&plan->d_hsigma), sizeof(float) * n_pix) != cudaSuccess) {
            cudaGetLastError();
            return fail(plan, NSFRB_ENOMEM, "device cube for host search");
        }
        if ((st = cuda_check(plan, cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking),
                             "copy stream")) != NSFRB_OK)
            return st;
        for (int i = 0; i < kSlabs + 1; ++i)
            if ((st = cuda_check(plan, cudaEventCreateWithFlags(&plan->slab_ev[i], cudaEventDisableTiming),
                                 "slab event")) != NSFRB_OK)
                return st;
    }
    // the copy stream may overwrite the device cube only after the previous search read it
    if ((st = cuda_check(plan, cudaEventRecord(plan->slab_ev[kSlabs], s), "event")) != NSFRB_OK) return st;
    if ((st = cuda_check(plan, cudaStreamWaitEvent(plan->copy_stream, plan->slab_ev[kSlabs], 0), "wait")) !=
        NSFRB_OK)
        return st;
    if (h_sigma &&
        (st = cuda_check(plan,
                         cudaMemcpyAsync(plan->d_hsigma, h_sigma, sizeof(float) * n_pix, cudaMemcpyHostToDevice,
                                         plan->copy_stream),
                         "sigma copy")) != NSFRB_OK)
        return st;
    if ((st = cuda_check(plan, cudaMemsetAsync(plan->d_err, 0, sizeof(int32_t), s), "memset")) != NSFRB_OK)
        return st;
    if ((st = cuda_check(plan, cudaEventRecord(plan->t_start, s), "event")) != NSFRB_OK) return st;
    const int64_t slab = (n_pix + kSlabs - 1) / kSlabs;
    for (int i = 0; i < kSlabs; ++i) {
        const int64_t p0 = i * slab;
        const int64_t n = std::min<int64_t>(slab, n_pix - p0);
        if (n <= 0) break;
        const char *src = static_cast<const char *>(h_cube) + p0 * pix_bytes;
        char *dst = static_cast<char *>(plan->d_hcube) + p0 * pix_bytes;
        if ((st = cuda_check(plan,
                             cudaMemcpyAsync(dst, src, n * pix_bytes, cudaMemcpyHostToDevice, plan->copy_stream),
                             "cube copy")) != NSFRB_OK)
            return st;
        if ((st = cuda_check(plan, cudaEventRecord(plan->slab_ev[i], plan->copy_stream), "event")) != NSFRB_OK)
            return st;
        if ((st = cuda_check(plan, cudaStreamWaitEvent(s, plan->slab_ev[i], 0), "wait")) != NSFRB_OK) return st;
        if (mad_slabs_apply(plan))
            st = queue_search_mad(plan, plan->d_hcube, c.dtype, p0, n, s);
        else
            st = queue_search(plan, plan->d_hcube, 0, c.dtype, c.n_t, 0, h_sigma ? plan->d_hsigma : nullptr, p0, n,
                              nullptr, nullptr, 0, s);
        if (st != NSFRB_OK) return st;
    }
    return queue_finish(plan, s);
}

nsfrb_status nsfrb_candidates(nsfrb_plan_t plan, nsfrb_candidate *h_out, int32_t cap, int32_t *n_total) {
    if (!plan || !n_total || cap < 0 || (cap > 0 && !h_out)) return fail(plan, NSFRB_EINVAL, "bad argument");
    nsfrb_status st = wait_done(plan);
    if (st != NSFRB_OK) return st;
    int32_t hdr[2] = {0, 0};   // err, n_cand
    if ((st = cuda_check(plan, cudaMemcpy(hdr, plan->d_err, sizeof(hdr), cudaMemcpyDeviceToHost), "copy")) != NSFRB_OK)
        return st;
    *n_total = hdr[1];
    const int32_t n = std::min(hdr[1], cap);
    if (n > 0 &&
        (st = cuda_check(plan, cudaMemcpy(h_out, plan->d_cand, sizeof(CandRec) * n, cudaMemcpyDeviceToHost),
                         "copy candidates")) != NSFRB_OK)
        return st;
    if (hdr[0] & ERR_WAIT_TIMEOUT) return fail(plan, NSFRB_ETIMEOUT, "a bulk copy into shared memory timed out");
    if (hdr[0] & ERR_ZERO_MAD) return fail(plan, NSFRB_EINVAL, "zero MAD in at least one (pixel, subband) row");
    if (hdr[1] > cap) return fail(plan, NSFRB_ETRUNC, "more candidates than capacity");
    return NSFRB_OK;
}

nsfrb_status nsfrb_best(nsfrb_plan_t plan, float *out_snr, int32_t *out_idx) {
    if (!plan) return fail(plan, NSFRB_EINVAL, "null plan");
    nsfrb_status st = wait_done(plan);
    if (st != NSFRB_OK) return st;
    const int64_t n_pix = static_cast<int64_t>(plan->cfg.ny) * plan->cfg.nx;
    std::vector<PixRec> rec(n_pix);
    if ((st = cuda_check(plan, cudaMemcpy(rec.data(), plan->d_rec, sizeof(PixRec) * n_pix, cudaMemcpyDeviceToHost),
                         "copy records")) != NSFRB_OK)
        return st;
    std::vector<float> snr(out_snr ? n_pix : 0);
    std::vector<int32_t> idx(out_idx ? 3 * n_pix : 0);
    for (int64_t i = 0; i < n_pix; ++i) {
        if (out_snr) snr[i] = rec[i].snr;
        if (out_idx) {
            idx[3 * i] = rec[i].dm_idx;
            idx[3 * i + 1] = rec[i].w_idx;
            idx[3 * i + 2] = rec[i].t_idx;
        }
    }
    if (out_snr &&
        (st = cuda_check(plan, cudaMemcpy(out_snr, snr.data(), sizeof(float) * n_pix, cudaMemcpyDefault), "copy")))
        return st;
    if (out_idx && (st = cuda_check(plan,
                                    cudaMemcpy(out_idx, idx.data(), sizeof(int32_t) * 3 * n_pix, cudaMemcpyDefault),
                                    "copy")))
        return st;
    return NSFRB_OK;
}

nsfrb_status nsfrb_full(nsfrb_plan_t plan, float *out_snr, int16_t *out_t_idx) {
    if (!plan) return fail(plan, NSFRB_EINVAL, "null plan");
    if (plan->cfg.out_mode != NSFRB_OUT_FULL) return fail(plan, NSFRB_EINVAL, "plan is not in FULL mode");
    nsfrb_status st = wait_done(plan);
    if (st != NSFRB_OK) return st;
    const size_t n = static_cast<size_t>(plan->cfg.ny) * plan->cfg.nx * plan->cfg.n_dm * plan->cfg.n_w;
    if (out_snr && (st = cuda_check(plan, cudaMemcpy(out_snr, plan->d_full_snr, n * sizeof(float), cudaMemcpyDefault),
                                    "copy full S/N")))
        return st;
    if (out_t_idx && (st = cuda_check(plan,
                                      cudaMemcpy(out_t_idx, plan->d_full_t, n * sizeof(int16_t), cudaMemcpyDefault),
                                      "copy full t")))
        return st;
    return NSFRB_OK;
}

nsfrb_status nsfrb_last_timing(nsfrb_plan_t plan, float *search_ms, float *total_ms) {
    if (!plan) return fail(plan, NSFRB_EINVAL, "null plan");
    nsfrb_status st = wait_done(plan);
    if (st != NSFRB_OK) return st;
    if ((st = cuda_check(plan, cudaEventSynchronize(plan->t_end), "event sync")) != NSFRB_OK) return st;
    if (search_ms &&
        (st = cuda_check(plan, cudaEventElapsedTime(search_ms, plan->t_start, plan->t_search), "elapsed")))
        return st;
    if (total_ms && (st = cuda_check(plan, cudaEventElapsedTime(total_ms, plan->t_start, plan->t_end), "elapsed")))
        return st;
    return NSFRB_OK;
}

nsfrb_status nsfrb_plan_set_tile(nsfrb_plan_t plan, int32_t dtype, int32_t tile) {
    if (!plan) return fail(plan, NSFRB_EINVAL, "null plan");
    if (dtype < NSFRB_F32 || dtype > NSFRB_F16) return fail(plan, NSFRB_EINVAL, "unknown storage type");
    if (tile != 0 && !tile_is_known(tile)) return fail(plan, NSFRB_EINVAL, "unknown tile");
    plan->tile[dtype] = tile;
    return NSFRB_OK;
}

nsfrb_status nsfrb_plan_get_tile(nsfrb_plan_t plan, int32_t dtype, int32_t *tile) {
    if (!plan || !tile) return fail(plan, NSFRB_EINVAL, "null argument");
    if (dtype < NSFRB_F32 || dtype > NSFRB_F16) return fail(plan, NSFRB_EINVAL, "unknown storage type");
    *tile = plan->tile[dtype];
    return NSFRB_OK;
}

nsfrb_status nsfrb_plan_autotune(nsfrb_plan_t plan, const void *d_cube, const float *d_sigma, int32_t reps,
                                 void *stream, int32_t *h_tile, float *h_ms) {
    if (!plan || !d_cube || reps < 1) return fail(plan, NSFRB_EINVAL, "bad argument");
    if (h_ms)
        for (int k = 0; k < NSFRB_N_TILES; ++k) h_ms[k] = -1.0f;
    // one untimed search finds the storage type the barrier-free kernel would search (the slabs of
    // MAD mode are FP32) or that it does not apply
    nsfrb_status st = nsfrb_search(plan, d_cube, d_sigma, nullptr, stream);
    if (st == NSFRB_OK) st = nsfrb_last_timing(plan, nullptr, nullptr);
    if (st != NSFRB_OK) return st;
    const int s_t = plan->last_tile_st;
    if (plan->last_tile == 0 || s_t < 0) {
        if (h_tile) *h_tile = 0;
        return NSFRB_OK;
    }
    const int32_t keep = plan->tile[s_t];
    int32_t best = 0;
    float best_ms = 0.0f;
    std::vector<float> t(reps);
    for (int k = 0; k < NSFRB_N_TILES; ++k) {
        plan->tile[s_t] = kTileCodes[k];
        for (int r = -1; r < reps; ++r) {   // one warm-up search per tile
            st = nsfrb_search(plan, d_cube, d_sigma, nullptr, stream);
            if (st == NSFRB_OK) st = nsfrb_last_timing(plan, r >= 0 ? &t[r] : nullptr, nullptr);
            if (st != NSFRB_OK) {
                plan->tile[s_t] = keep;
                return st;
            }
            if (plan->last_tile != kTileCodes[k]) break;   // does not fit: another tile ran
        }
        if (plan->last_tile != kTileCodes[k]) continue;
        std::sort(t.begin(), t.end());
        const float med = t[reps / 2];
        if (h_ms) h_ms[k] = med;
        if (best == 0 || med < best_ms) {
            best = kTileCodes[k];
            best_ms = med;
        }
    }
    plan->tile[s_t] = best ? best : keep;
    if (h_tile) *h_tile = plan->tile[s_t];
    // the plan's results are those of a search with the chosen tile
    st = nsfrb_search(plan, d_cube, d_sigma, nullptr, stream);
    if (st == NSFRB_OK) st = nsfrb_last_timing(plan, nullptr, nullptr);
    return st;
}

void nsfrb_destroy(nsfrb_plan_t plan) {
    if (!plan) return;
    destroy_stream_state(plan);
    if (plan->dev_ready) {
        cudaEventSynchronize(plan->done);
        cudaEventDestroy(plan->done);
        cudaEventDestroy(plan->t_start);
        cudaEventDestroy(plan->t_search);
        cudaEventDestroy(plan->t_end);
    }
    cudaFree(plan->d_table);
    cudaFree(plan->d_rec);
    cudaFree(plan->d_cand);
    cudaFree(plan->d_counts);
    cudaFree(plan->d_list);
    cudaFree(plan->d_full_snr);
    cudaFree(plan->d_madws);
    cudaFree(plan->d_bad);
    cudaFree(plan->d_full_t);
    cudaFree(plan->d_hcube);
    cudaFree(plan->d_hsigma);
    cudaFree(plan->d_smax_w);
    if (plan->copy_stream) {
        cudaStreamSynchronize(plan->copy_stream);
        cudaStreamDestroy(plan->copy_stream);
        for (int i = 0; i < kSlabs + 1; ++i)
            if (plan->slab_ev[i]) cudaEventDestroy(plan->slab_ev[i]);
    }
    cudaGetLastError();
    delete plan;
}

}  // extern "C"
