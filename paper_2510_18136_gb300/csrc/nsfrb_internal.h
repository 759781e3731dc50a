// Internal declarations shared by the host planner and the CUDA kernels of
// libnsfrb.  Not part of the public C ABI (see include/nsfrb.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace nsfrb {

constexpr int kWarps = 12;                // warps per search CTA
constexpr int kThreads = kWarps * 32;     // threads per search CTA
constexpr int kMaxW = 16;                 // widths per plan
constexpr int kMaxSub = 32;               // subbands per plan
constexpr int kMaxT = 4096;               // longest window
constexpr int kMaxTRegs = 1247;           // longest window of the register path (32 lanes x 39 samples - 1)
constexpr int kLongC = 128;               // "chunk" of longer windows: the long-window kernel
constexpr int kSmallMax = 16;             // widths <= min(C, 16) use the in-lane path
constexpr int kHistBins = 256;            // radix-select digit bins (MAD mode)

// Width classes of the boxcar stage.
enum : int32_t { WC_SMALL = 0, WC_LARGE = 1, WC_GENERIC = 2 };
constexpr int kPow2 = 11;   // power-of-two widths 1 .. 1024 have compile-time code paths

// Class of the power-of-two width 2^J for chunk size C: in-lane (<= min(C, 16)),
// lane-strided (32 M with M < C), or shared-memory generic.
__host__ __device__ constexpr int pow2_class(int C, int J) {
    return ((1 << J) <= (C < kSmallMax ? C : kSmallMax))
               ? WC_SMALL
               : ((((1 << J) % 32) == 0 && ((1 << J) / 32) < C) ? WC_LARGE : WC_GENERIC);
}

// Per-pixel best trial (written by the search kernel, read by compaction).
struct PixRec {
    float snr;
    int32_t dm_idx, w_idx, t_idx;
};

// Same layout as nsfrb_candidate in the public header.
struct CandRec {
    int32_t row, col, dm_idx, w_idx, t_idx;
    float snr;
};

// Error bits latched by kernels into a device word.
enum : int32_t { ERR_ZERO_MAD = 1, ERR_WAIT_TIMEOUT = 2 };

// Per-unique-row info words (u_info[u * kInfo + ...]).
enum { UI_SMAX = 0, UI_FIRST_D = 1, UI_N_D = 2, UI_DOFF = 3, UI_ND = 4, kInfo = 5 };

struct SearchParams {
    // ---- input cube: element (pixel p, subband k, sample t) lives at
    //      cube[((p - cube_pix0) * n_sub + k) * row_len + t_off + t]
    const void *cube;
    int64_t row_len;       // elements per (pixel, subband) row in memory
    int64_t cube_pix0;     // pixel index of the cube pointer's first pixel
    int32_t t_off;         // first window sample inside a row
    const int32_t *t_off_dev;   // if set, t_off is read from device memory
    int32_t t_wrap;        // > 0: a row is a ring of t_wrap samples, window sample t sits at
                           // (t_off + t) mod t_wrap (t_off < t_wrap; plain loads only)
    int64_t t_stride;      // > 0 (plain loads only): a sample-major cube, element (pixel q,
                           // subband k, ring position j) at cube[(j * n_sub + k) * t_stride + q],
                           // t_stride the pixel count of a sample plane
    int32_t dtype;         // NSFRB_F32 / BF16 / F16
    int32_t n_sub, n_t;
    int32_t Tp;            // shared-memory row pitch (floats)
    int32_t stage;         // 0 plain loads, 1 bulk FP32 direct, 2 bulk 16-bit staging (widened to
                           // FP32), 3 bulk 16-bit direct (read in place by the barrier-free kernel)
    int32_t stg_pitch;     // staging row pitch in bytes (stage 2); fits any t_off % 8
    // ---- work items: item i -> pixel (pix_list ? pix_list[i] : pix0 + i)
    int64_t n_items;
    int64_t pix0;
    const int32_t *pix_list;
    const int32_t *n_items_dev;   // if set, the item count is read from here
    // ---- noise
    const float *sigma;    // per absolute pixel, or nullptr
    float sigma_default;
    int32_t noise_mode;
    // ---- delay tables (device memory; copied to shared memory per CTA)
    int32_t n_u, n_u_active;
    const int32_t *table;  // [n_u*kInfo info][deltas][n_u*n_sub shifts as int32]
    int32_t n_deltas;
    // ---- widths
    int32_t n_w;
    int32_t widths[kMaxW];
    int32_t wclass[kMaxW];
    int32_t pow2_wi[kPow2];     // width index of 2^j if it has a compile-time path, else -1
    int32_t has_small, has_large;
    int32_t n_gen;              // widths evaluated from shared memory
    int32_t gen_wi[kMaxW];
    int32_t n_dm;
    int32_t new_blk;       // > 0: only trials that end in the last new_blk samples
    int32_t pipe;          // 1: barrier-free kernel (stage 1 or 3, KNOWN noise, records only)
    int32_t teams;         // barrier-free kernel: teams of kWarps / teams warps, each on its own
                           // pixel with its own buffers; long-window kernel: warps per CTA
    int32_t nb;            // barrier-free kernel: pixel buffers per team, 2 (the pixel after next
                           // copied while one is searched) or 1 (the next copied after a pixel)
    // ---- outputs (indexed by absolute pixel)
    PixRec *rec;
    float *full_snr;       // [pix][n_dm][n_w] or nullptr
    int16_t *full_t;
    int32_t *err;
    const uint8_t *bad_pix;   // barrier-free kernel: pixels flagged here (by absolute index) get an
                              // invalid record (S/N -inf) and ERR_ZERO_MAD (normalised slabs)
};

// Shared-memory carve-up, identical on host and device.
struct SmemLayout {
    size_t table, xs, stg, pbuf, fscr, hist, wbest, sinv, bar, total;
};

// Floats per warp of the earliest-sample search's scratch (a lane's extended in-lane prefix:
// C + 16 values for the sample-pair chunk C = 38).
constexpr int kFindScr = 64;

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(const SearchParams &p, int C) {
    SmemLayout L{};
    size_t o = 0;
    L.table = o;
    o += align_up(sizeof(int32_t) * ((size_t)p.n_u * kInfo + p.n_deltas + (size_t)p.n_u * p.n_sub), 16);
    L.xs = o;
    const int teams = (p.pipe && p.teams > 1) ? p.teams : 1;
    const int nb = (p.pipe && p.nb == 1) ? 1 : 2;
    const int nbuf = (p.stage == 1 || p.stage == 3) ? nb * teams : 1;
    const size_t es = (p.stage == 3) ? 2 : sizeof(float);
    o += align_up(es * (size_t)nbuf * p.n_sub * p.Tp, 128);
    L.stg = o;
    if (p.stage == 2) o += align_up((size_t)2 * p.n_sub * p.stg_pitch, 128);
    L.pbuf = o;
    o += sizeof(float) * (size_t)kWarps * 32 * C;
    L.fscr = o;
    if (C % 2 == 0) o += sizeof(float) * (size_t)kWarps * kFindScr;
    L.hist = o;
    // MAD histograms: in the staging buffer of the current item when staging, else own space
    if (p.noise_mode == 1 && p.stage != 2) o += sizeof(uint32_t) * (size_t)kWarps * kHistBins;
    L.wbest = o;
    // the barrier-free kernel keeps two pixels' records per team
    const size_t n_slots = p.pipe ? 2 * static_cast<size_t>(teams) : 1;
    o += sizeof(PixRec) * kWarps * n_slots;
    L.sinv = o;
    o += sizeof(float) * kMaxW * n_slots + sizeof(int32_t) * (2 * n_slots + 4);
    o = align_up(o, 8);
    L.bar = o;
    o += sizeof(unsigned long long) * 2 * teams;
    L.total = o;
    return L;
}

// Chunk sizes (samples per lane) with compiled kernels.  Odd chunks read one sample at a
// time (lanes C words apart hit distinct banks); the even chunk 38 (= 2 mod 4) reads and
// computes sample pairs (64-bit accesses of lanes C words apart are conflict-free).
constexpr int kChunks[] = {1, 3, 5, 9, 17, 25, 38, 39};
constexpr int kNumChunks = 8;

inline int pick_chunk(int n_t) {
    for (int i = 0; i < kNumChunks; ++i)
        if (32 * kChunks[i] >= n_t + 1) return kChunks[i];
    return n_t <= kMaxT ? kLongC : -1;
}

// Kernel launchers (one translation unit per chunk size; C = kLongC: the long-window kernel).
cudaError_t launch_search(int C, const SearchParams &p, int grid, size_t smem, cudaStream_t s);
cudaError_t prepare_search(int C, size_t smem);
// The long-window kernel: warps per CTA that fit max_smem (0: none), and its shared memory.
int long_warps(const SearchParams &p, int max_smem);
size_t long_smem(const SearchParams &p, int n_warps);
cudaError_t launch_search_long(const SearchParams &p, int grid, size_t smem, cudaStream_t s);
cudaError_t prepare_search_long(size_t smem);

// Compaction of per-pixel records into the candidate list ordered by pixel.
cudaError_t launch_compact(const PixRec *rec, int64_t n_pix, int32_t nx, float thr,
                           int32_t *block_counts, int32_t n_blocks, CandRec *out,
                           int32_t *n_out, cudaStream_t s);
// Pixels whose S/N lies within +-eps of the threshold -> list (unordered).
cudaError_t launch_rescore_select(const PixRec *rec, int64_t n_pix, float thr, float eps,
                                  int32_t *list, int32_t *n_list, cudaStream_t s);
constexpr int kCompactBlock = 1024;

// Median / MAD normalisation of pixels [pix0, pix0 + n_pix) of a pixel-major cube ([pix][sub][n_t],
// rows of n_t samples in `dtype`) into out ([n_pix][n_sub][n_t] FP32); bad[pixel] = 1 where a row
// has zero MAD (bad must be cleared by the caller).
cudaError_t launch_mad_normalise(const void *cube, int dtype, int64_t pix0, int64_t n_pix, int n_sub, int n_t,
                                 float *out, uint8_t *bad, int n_sm, cudaStream_t s);

}  // namespace nsfrb
