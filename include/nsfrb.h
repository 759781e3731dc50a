/*
 * nsfrb.h -- C ABI of libnsfrb, a GB300 (sm_103a) image-plane single-pulse
 * search over a cube of dirty images (pixel x subband x time), following the
 * DSA-110 NSFRB search of arXiv 2510.18136, Sec. 2.2 ("cerberus Search
 * Pipeline"): per pixel, subbands are shifted by pre-computed integer
 * dispersion delays and summed for each DM trial, boxcar-filtered over a set
 * of widths, normalised to S/N by a noise level, maximised over time, and
 * thresholded (Fig. 1: candidates above the S/N threshold).
 *
 * Conventions shared by every call
 * ---------------------------------
 * - Every call returns an nsfrb_status.  No call aborts, traps or prints.
 *   The first CUDA error seen by a plan is latched and returned again by the
 *   next call on that plan (NSFRB_ECUDA); nsfrb_last_error() gives the text.
 * - Pointers named d_* are device pointers (cudaMalloc / torch tensors on
 *   the current device); pointers named h_* are host pointers.  The caller
 *   owns every buffer it passes.  Arrays inside nsfrb_config are copied by
 *   nsfrb_plan; they need not outlive the call.
 * - A plan owns its delay tables, device workspace and streams; it is not
 *   thread-safe.  Different plans may be used from different threads.
 * - "stream" arguments are a cudaStream_t passed as void* (0 = legacy
 *   default stream).
 *
 * Notation: pixel p = row * nx + col; subband k (increasing frequency);
 * sample t; DM trial d; width index w_idx into widths[]; T = n_t.
 */
#ifndef NSFRB_H
#define NSFRB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nsfrb_plan_s *nsfrb_plan_t;

typedef enum {
    NSFRB_OK = 0,
    NSFRB_EINVAL = 1,    /* invalid argument or configuration, or zero MAD */
    NSFRB_ENOMEM = 2,    /* device or host allocation failed / over budget */
    NSFRB_ECUDA = 3,     /* a CUDA call failed (text: nsfrb_last_error)    */
    NSFRB_ETIMEOUT = 4,  /* a bounded wait ran out                         */
    NSFRB_ETRUNC = 5,    /* more results than the caller's capacity        */
    NSFRB_ENOTREADY = 6  /* no result yet (search not run / block pending) */
} nsfrb_status;

/* Storage type of the input cube.  Arithmetic is always FP32. */
enum { NSFRB_F32 = 0, NSFRB_BF16 = 1, NSFRB_F16 = 2 };

/* Noise model (Sec. 2.2: each pixel's median is removed and the samples are
 * scaled by a running noise estimate).
 * KNOWN: the caller supplies sigma_D(p), the noise of the de-dispersed
 *        series of pixel p (d_sigma), or NULL for sqrt(n_sub) (unit noise
 *        per subband); no median subtraction.
 * MAD:   per (pixel, subband) over the window: x <- (x - median) /
 *        (1.4826 * MAD), then sigma_D = sqrt(n_sub); d_sigma must be NULL. */
enum { NSFRB_NOISE_KNOWN = 0, NSFRB_NOISE_MAD = 1 };

/* Output mode.  CANDIDATES: per-pixel maximum + candidate list.  FULL: also
 * S/N and TOA for every (pixel, DM, width) (Sec. 2.3: S/N and TOA arrays for
 * all pixels, widths and DM trials are saved). */
enum { NSFRB_OUT_CANDIDATES = 0, NSFRB_OUT_FULL = 1 };

typedef struct {
    int32_t ny, nx;          /* image rows, columns (>= 1)                     */
    int32_t n_sub;           /* subbands, 1..32                                */
    int32_t n_t;             /* window length in samples, 1..4096.  Up to 1247
                                (the paper's 25 and 1200) a warp holds a DM
                                row's prefix sums in registers; longer windows
                                run a kernel that reads the cube in place and
                                keeps the prefix sums in shared memory          */
    double t_samp_ms;        /* sampling time, e.g. 134.2                      */
    double k_dm_ms;          /* dispersion constant in ms GHz^2, e.g. 4.149    */
    const double *freq_mhz;  /* [n_sub] subband centres, strictly increasing   */
    int32_t n_dm;            /* DM trials, 1..4096                             */
    const double *dm;        /* [n_dm] pc cm^-3, nondecreasing, >= 0           */
    int32_t n_w;             /* widths, 1..16                                  */
    const int32_t *widths;   /* [n_w] samples, strictly increasing, 1..n_t     */
    float threshold;         /* candidate iff S/N > threshold (strict)         */
    int32_t dtype;           /* NSFRB_F32 / NSFRB_BF16 / NSFRB_F16             */
    int32_t noise_mode;      /* NSFRB_NOISE_KNOWN / NSFRB_NOISE_MAD            */
    int32_t out_mode;        /* NSFRB_OUT_CANDIDATES / NSFRB_OUT_FULL          */
    float rescore_eps;       /* BF16/F16 only: pixels whose best S/N lies within
                                +-rescore_eps of the threshold are searched
                                again in FP32 (offline: from the FP32 cube
                                passed to nsfrb_search; serving: from an FP32
                                copy of the window, in device memory or, where
                                that does not fit, pinned host memory);
                                <= 0 disables re-scoring.  Measured BF16 S/N
                                errors against the FP64 search of the FP32
                                input: <= 0.03 with known noise (full-window
                                and serving workloads), <= 0.08 with MAD
                                normalisation (512x512 Student-t workload);
                                use at least the bound of the workload so that
                                the candidate set equals the FP32 one           */
} nsfrb_config;

/* One candidate: the pixel's best trial (maximum S/N over DM, width, time;
 * ties go to the smallest DM index, then width index, then time). */
typedef struct {
    int32_t row, col;   /* pixel                                               */
    int32_t dm_idx;     /* index into cfg.dm                                   */
    int32_t w_idx;      /* index into cfg.widths                               */
    int32_t t_idx;      /* boxcar start sample in the top-subband frame; the
                           pulse reaches subband k at t_idx + shift[dm_idx][k] */
    float snr;
} nsfrb_candidate;

/* Create a plan (host work only; device memory is allocated on first use).
 * Computes the integer delay table of Sec. 2.2,
 *   shift[d][k] = floor(k_dm_ms * dm[d] * (f_k^-2 - f_top^-2) / t_samp_ms + 0.5)
 * (f in GHz, f_top = highest subband centre), and merges DM trials with
 * identical shift rows (they produce identical S/N; results keep the lowest
 * DM index).  Errors: EINVAL (bad config), ENOMEM. */
nsfrb_status nsfrb_plan(const nsfrb_config *cfg, nsfrb_plan_t *out);

/* Copy the delay table to h_shifts[n_dm * n_sub] (row-major [d][k]). */
nsfrb_status nsfrb_plan_delays(nsfrb_plan_t plan, int32_t *h_shifts);

/* Number of distinct shift rows and the largest shift of each DM trial
 * (h_smax[n_dm], or NULL). */
nsfrb_status nsfrb_plan_info(nsfrb_plan_t plan, int32_t *n_unique, int32_t *h_smax);

/* Search one cube (Sec. 2.2), asynchronously on `stream`.
 * d_cube:     [ny*nx][n_sub][n_t] in cfg.dtype, pixel-major, contiguous.
 * d_sigma:    [ny*nx] FP32 sigma_D per pixel (KNOWN mode) or NULL.
 * d_cube_f32: optional FP32 copy of the cube for re-scoring (BF16/F16 only),
 *             or NULL.
 * The valid trials of DM d and width w are t in [0, n_t - smax_d - w]; a pair
 * with none is skipped (FULL: S/N -inf, t_idx -1).  The caller must keep the
 * inputs alive and unmodified until the stream reaches the search.
 * Errors: EINVAL, ENOMEM, ECUDA.  In-kernel conditions (zero MAD) are
 * reported by nsfrb_candidates. */
nsfrb_status nsfrb_search(nsfrb_plan_t plan, const void *d_cube, const float *d_sigma,
                          const void *d_cube_f32, void *stream);

/* Same search from HOST buffers: h_cube (pinned for full speed) is copied to
 * the device in pixel slabs on a copy stream, overlapped with the search of
 * the previous slab; h_sigma as d_sigma.  Returns when the search is queued. */
nsfrb_status nsfrb_search_host(nsfrb_plan_t plan, const void *h_cube, const float *h_sigma,
                               void *stream);

/* Wait for the last search of this plan and copy its candidates (S/N strictly
 * above the threshold, ordered by pixel index) to h_out[0..cap).  *n_total is
 * always set to the full count.  Errors: ENOTREADY (no search yet), ETRUNC
 * (n_total > cap; the first cap are written), EINVAL (a zero MAD row was
 * met in MAD mode), ECUDA. */
nsfrb_status nsfrb_candidates(nsfrb_plan_t plan, nsfrb_candidate *h_out, int32_t cap,
                              int32_t *n_total);

/* Per-pixel best of the last search: out_snr[ny*nx], out_idx[ny*nx][3] =
 * (dm_idx, w_idx, t_idx), host or device pointers (either may be NULL).
 * A pixel with no valid trial has S/N -inf and indices -1.  Waits. */
nsfrb_status nsfrb_best(nsfrb_plan_t plan, float *out_snr, int32_t *out_idx);

/* FULL mode: S/N [ny*nx][n_dm][n_w] and t_idx (same shape) of the last
 * search, host or device pointers.  Waits.  EINVAL if out_mode != FULL. */
nsfrb_status nsfrb_full(nsfrb_plan_t plan, float *out_snr, int16_t *out_t_idx);

/* Device time of the last search: *search_ms covers the search kernel
 * launch(es) of the last nsfrb_search / nsfrb_search_host (including the
 * re-score pass), *total_ms the whole queued work up to the candidate list
 * (either may be NULL).  Measured with CUDA events on the launching stream;
 * waits for the search.  ENOTREADY before the first search. */
nsfrb_status nsfrb_last_timing(nsfrb_plan_t plan, float *search_ms, float *total_ms);

/* ---- pixel x DM tile of the per-pixel search kernel ---------------------
 * The search of Sec. 2.2 with KNOWN noise (and the FP32 slabs that MAD mode
 * normalises into) runs a persistent kernel in which each CTA's 12 warps form
 * `teams` teams, each team searching its own pixel with the DM row groups
 * (unique delay rows) split among its warps, from `buffers` shared-memory
 * copies of that pixel's rows (2 = the next pixel's copy overlaps this one's
 * search).  A tile is coded 10 * teams + buffers; NSFRB_TILES lists the
 * compiled ones.  Every tile gives the same candidates up to FP32 summation
 * order (different warps build a row group's partial sums from scratch).
 * Tile 0 = the first of 41, 31, 22, 21, 12 whose buffers fit in shared
 * memory (16-bit rows of a full window: 41; FP32 rows: 21). */
#define NSFRB_N_TILES 5
#define NSFRB_TILES 12, 22, 21, 31, 41

/* Preferred tile for rows stored as `dtype` (NSFRB_F32/BF16/F16; MAD-mode
 * slabs are F32): 0 or one of NSFRB_TILES.  A tile whose buffers do not fit
 * falls back to tile 0's order.  Errors: EINVAL (unknown dtype or tile). */
nsfrb_status nsfrb_plan_set_tile(nsfrb_plan_t plan, int32_t dtype, int32_t tile);
nsfrb_status nsfrb_plan_get_tile(nsfrb_plan_t plan, int32_t dtype, int32_t *tile);

/* Time every tile that fits on the caller's cube (nsfrb_search arguments,
 * no re-score), `reps` timed searches each after one warm-up, and keep the
 * one with the smallest median search time as the plan's preference for the
 * storage type the kernel searched.  h_tile (or NULL) gets that tile (0 when
 * the plan's searches do not use this kernel: MAD windows of n_t not a
 * multiple of 4, windows over 1247 samples); h_ms[NSFRB_N_TILES] (or NULL) the medians in
 * NSFRB_TILES order, -1 for tiles that do not fit.  Synchronous: it waits
 * for every search it queues on `stream`.  Afterwards the plan's results are
 * those of one search of the cube with the chosen tile.  Errors: as
 * nsfrb_search; EINVAL for reps < 1. */
nsfrb_status nsfrb_plan_autotune(nsfrb_plan_t plan, const void *d_cube, const float *d_sigma, int32_t reps,
                                 void *stream, int32_t *h_tile, float *h_ms);

/* ---- longer timescales (Sec. 2.2: the search is repeated on data binned by 5
 * samples (0.67 s, DM range x5 so that the same integer shifts apply) and by
 * 75 samples (10.05 s, no de-dispersion)) --------------------------------
 * d_out[r][j] = sum_{q < factor} d_in[r][j*factor + q] for every row r of
 * n_t samples (a (pixel, subband) row of a pixel-major cube: n_rows =
 * ny*nx*n_sub), j < n_t / factor; a trailing remainder is dropped.  d_in in
 * `dtype` storage, d_out FP32; device pointers; asynchronous.  The noise of a
 * binned sample is sqrt(factor) times the unbinned one: search the binned cube
 * with sigma_D scaled by sqrt(factor) (KNOWN mode).  EINVAL on bad sizes. */
nsfrb_status nsfrb_bin_time(const void *d_in, int32_t dtype, int64_t n_rows, int32_t n_t, int32_t factor,
                            float *d_out, void *stream);

/* ---- PSF-based candidate clustering (Sec. 2.3: the top candidates by S/N
 * are compared with the point-spread function; the PSF thresholded at its
 * 90th percentile is a binary mask centred on each candidate in turn, the
 * other candidates inside it are possible sidelobes, a weighted mean S/N is
 * formed over the central and sidelobe candidates, and the central candidate
 * of the largest one is the final, most likely candidate) ----------------- */
typedef struct {
    nsfrb_candidate final_cand;   /* central candidate of the best cluster      */
    float weighted_snr;           /* its PSF-weighted mean S/N                    */
    int32_t n_top;                /* candidates considered (min(top_k, n))        */
    int32_t final_rank;           /* index of final_cand in the top list, or -1   */
    uint32_t members;             /* bit j set: top candidate j is in its cluster */
} nsfrb_cluster_result;

/* d_cand[n]: candidates (device, e.g. a copy of nsfrb_candidates' output);
 * nx: image width (pixel index = row*nx + col, used only to order equal S/N);
 * d_psf[ph][pw]: PSF image (device FP32, peak at (ph/2, pw/2)), ph*pw <= 4096;
 * percentile: mask threshold (90 in the paper; linear interpolation between
 * order statistics); top_k (10 in the paper, <= 32).
 * Outputs (device): d_top[min(top_k, n)] the top candidates by S/N (ties:
 * smaller pixel index first) and one nsfrb_cluster_result at d_result.
 * Score of a cluster (the paper says "weighted mean S/N" and gives no
 * formula), psf_j the PSF value at member j's offset from the central
 * candidate (1 for the central one of a peak-normalised PSF):
 *   score_mode NSFRB_CLUSTER_PSF_MEAN (0): the PSF-weighted mean
 *     sum_j psf_j snr_j / sum_j psf_j;
 *   score_mode NSFRB_CLUSTER_LSQ (1): the members' S/N referred to the
 *     central lobe (snr_j / psf_j) averaged with inverse-variance weights
 *     psf_j^2, sum_j psf_j snr_j / sum_j psf_j^2 (the least-squares source
 *     S/N under the PSF template).
 * Highest score wins, the first in top order on ties.  Asynchronous.
 * EINVAL on a bad size, percentile or score_mode. */
enum { NSFRB_CLUSTER_PSF_MEAN = 0, NSFRB_CLUSTER_LSQ = 1 };
nsfrb_status nsfrb_psf_cluster(const nsfrb_candidate *d_cand, int32_t n, int32_t nx, const float *d_psf,
                               int32_t ph, int32_t pw, float percentile, int32_t top_k, int32_t score_mode,
                               nsfrb_candidate *d_top, void *d_result, void *stream);

/* ---- search without device allocation -------------------------------------
 * The paper has no counterpart to this call.  It serves callers that cannot
 * allocate device memory at search time: code that runs while another
 * allocator (a framework's caching pool, a fixed real-time memory map) owns
 * all free device memory, or a latency-bound loop that cannot afford
 * cudaMalloc (which may synchronise the device).  It runs the same search and
 * candidate compaction as nsfrb_search + nsfrb_candidates, but its scratch
 * (delay tables, per-pixel best records, counters) lives in one fixed
 * array inside the library, held by every GPU that loads the library until
 * the process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine; the plan must have been made by nsfrb_plan (host memory only).
 *
 * d_cube, d_sigma: as nsfrb_search (device pointers, contiguous).
 * d_out[cap]:      device buffer for the candidates (pixel order); only the
 *                  first cap are written.
 * d_n_total:       device int32: the full candidate count, or -1 if a zero
 *                  MAD row was met (MAD mode), -2 if a bulk copy timed out.
 * Asynchronous on `stream`.  Limits: ny*nx <= NSFRB_STATIC_MAX_PIX and the
 * plan's tables <= NSFRB_STATIC_MAX_TABLE_WORDS int32 words (EINVAL beyond);
 * candidate output mode only; no re-scoring; MAD normalisation only for
 * windows of at most 1247 samples (longer ones need nsfrb_search's
 * normalisation workspace: EINVAL).  The first call on a device
 * looks up the array's device address there (and sets the kernel's shared
 * memory limit), so make that first call before any stream capture.  The
 * array is reserved on a device when the library's code for this call is
 * first loaded there, which with CUDA's default lazy module loading is that
 * first call, not the library load: make the first call (a tiny plan will
 * do) before another allocator claims the device's free memory.  Each call
 * copies the plan's delay tables (at most NSFRB_STATIC_MAX_TABLE_WORDS int32
 * words) from the plan's pageable host memory into the array, a copy that
 * blocks the calling thread until it is staged.  Every
 * call shares the one array and overwrites what the previous call left in
 * it: calls whose work overlaps on the GPU (different streams, or different
 * plans at once) race and must be serialised by the caller. */
#define NSFRB_STATIC_MAX_PIX 262144
#define NSFRB_STATIC_MAX_TABLE_WORDS 65536
nsfrb_status nsfrb_search_static(nsfrb_plan_t plan, const void *d_cube, const float *d_sigma,
                                 nsfrb_candidate *d_out, int32_t cap, int32_t *d_n_total, void *stream);

/* ---- serving (Sec. 2.2: real-time search of 25-sample blocks arriving every
 * 3.35 s, with a 3.35 s timeout for missing subband images) ---------------
 * A plan opened for streaming keeps a rolling on-device window of the last
 * n_t samples (cfg.dtype storage).  Each pushed block holds n_blk samples in
 * imager order [n_blk][n_sub][ny][nx] FP32 on the host; it is copied and
 * transposed into the window, and only the trials that end inside the new
 * block are searched (t + w - 1 + smax_d >= n_t - n_blk).  The per-block
 * search runs as a captured CUDA graph.  Subbands missing from
 * present_mask are zero-filled for that block.
 * Re-scoring (16-bit storage with cfg.rescore_eps > 0): the stream also keeps
 * the window in FP32 (ny*nx*n_sub*n_t*4 bytes, written by the device as blocks
 * arrive, sample plane by sample plane in the block's [n_sub][ny][nx] layout):
 * in device memory when the free device memory measured at admission covers
 * the stream's bytes (nsfrb_stream_bytes), the window and hbm_reserve;
 * otherwise in pinned, mapped host memory (written and read over the host
 * link).  After each block the pixels whose
 * best S/N over the new trials lies within +-rescore_eps of the threshold are
 * searched again from it in FP32 (same new-trial mask) before the candidate
 * list is formed. */

/* Admit a stream: allocates the window and block buffers if the device has
 * hbm_reserve bytes free beyond what this stream needs (ENOMEM otherwise;
 * also ENOMEM if the re-score window fits neither the device nor pinned host
 * memory).
 * n_blk: samples per block (1..n_t).  One plan serves one field; concurrent
 * fields are separate plans (each with its own stream and graph). */
nsfrb_status nsfrb_stream_open(nsfrb_plan_t plan, int32_t n_blk, size_t hbm_reserve);

/* Bytes of device memory a stream of this plan needs (without the re-score
 * FP32 window, which goes to the device only if it also fits). */
nsfrb_status nsfrb_stream_bytes(nsfrb_plan_t plan, int32_t n_blk, size_t *bytes);

/* Where the open stream keeps its re-score FP32 window: *fp32_window = 1 in
 * device memory, 2 in pinned host memory, 0 no window (no re-scoring).
 * ENOTREADY without an open stream. */
nsfrb_status nsfrb_stream_window_info(nsfrb_plan_t plan, int32_t *fp32_window);

/* Queue one block (asynchronous; h_block must stay valid until the next
 * nsfrb_stream_poll returns).  ENOTREADY if the previous block has not been
 * polled yet. */
nsfrb_status nsfrb_stream_push(nsfrb_plan_t plan, const float *h_block, uint32_t present_mask);

/* Wait up to timeout_ms for the last pushed block and copy its candidates
 * (as nsfrb_candidates; t_idx refers to the current window).  ETIMEOUT if it
 * is not done in time (it stays queued: poll again).  *latency_ms (or NULL)
 * receives push -> completion device time. */
nsfrb_status nsfrb_stream_poll(nsfrb_plan_t plan, int32_t timeout_ms, nsfrb_candidate *h_out,
                               int32_t cap, int32_t *n_total, float *latency_ms);

/* Number of blocks pushed so far (windows before n_t / n_blk blocks are
 * partly empty: their missing samples are zero). */
nsfrb_status nsfrb_stream_blocks(nsfrb_plan_t plan, int64_t *n_blocks);

/* Device-resident blocks, for an imager on the same GPU (Sec. 2.1 images
 * feeding the Sec. 2.2 search without a host round trip).
 * nsfrb_stream_block: *d_block = the stream's block buffer, device FP32
 * [n_blk][n_sub][ny][nx], owned by the plan (valid until nsfrb_destroy).
 * Write the next block there only after the previous block has been polled.
 * nsfrb_stream_push_device: queue the block already in that buffer; the
 * search waits for the work queued so far on `stream` (the producer's
 * stream; NULL = legacy default stream).  Otherwise as nsfrb_stream_push. */
nsfrb_status nsfrb_stream_block(nsfrb_plan_t plan, float **d_block);
nsfrb_status nsfrb_stream_push_device(nsfrb_plan_t plan, uint32_t present_mask, void *stream);

/* ---- imager (Sec. 2.1, fringe-stopping and imaging: core baselines longer
 * than b_min, polarisations summed, Briggs weighting with robustness R on an
 * N x N uv-grid, 2-D inverse FFT with the grid and the image shifted by
 * ifftshift; each channel imaged separately and the channel images summed
 * into one image per subband and 134 ms sample) ----------------------------
 * Definitions (u, v in metres, f the channel frequency, dtheta the pixel):
 *   a baseline is kept when b_min < sqrt(u^2 + v^2) < b_max;
 *   its cell is k = rint(u * f_MHz * 1e6 / c * N * dtheta) per axis (FP64,
 *   left to right, ties to even), its conjugate goes to -k; cells with
 *   |k| > (N - 1) / 2 are dropped with their mirror;
 *   per channel, W_cell counts the visibilities in each cell (mirrors
 *   included), f^2 = (5 * 10^-R)^2 / (sum_cells W^2 / sum w) and each
 *   visibility is weighted 1 / (1 + W_cell f^2);
 *   image[y][x] = Re sum_k G_k exp(2 pi i (ku (x + N/2) + kv (y + N/2)) / N) / N^2
 *   (integer N/2), summed over the subband's channels: numpy's
 *   ifftshift(ifft2(ifftshift(G))).real with the zero frequency at N/2. */
typedef struct nsfrb_imager_s *nsfrb_imager_t;
typedef struct {
    int32_t n_grid;           /* N, uv-grid and image side: 175 in Sec. 2.1; 3..1024        */
    double pixel_arcsec;      /* image pixel: 10.3 arcsec in Sec. 2.1                          */
    double robust;            /* Briggs robustness R: -2 in Sec. 2.1                           */
    double b_min_m, b_max_m;  /* kept baselines: b_min < |b| < b_max (20 m, 485 m)             */
    int32_t n_base;           /* baselines                                                     */
    const double *uv_m;       /* [n_base][2] (u, v) in metres, host, copied                    */
    int32_t n_sub, n_chan;    /* subbands (16) and channels per subband (8)                    */
    const double *chan_mhz;   /* [n_sub][n_chan] channel centres in MHz, host, copied          */
} nsfrb_imager_config;

/* Plan the imager on the current device: selection, cells and weights in
 * FP64 on the host, gridding tables and twiddles on the device.  EINVAL on a
 * bad configuration or a uv support too large for one CTA's shared memory;
 * ENOMEM / ECUDA from the device. */
nsfrb_status nsfrb_imager_create(const nsfrb_imager_config *cfg, nsfrb_imager_t *out);

/* h_w[n_sub][n_chan][n_base] (host): the Briggs weight of every baseline at
 * every channel, 0 where the baseline is dropped. */
nsfrb_status nsfrb_imager_weights(nsfrb_imager_t im, float *h_w);

/* Extent of the occupied half-plane uv support (0 <= ku <= u_max,
 * |kv| <= v_max) and the number of gridding entries; any pointer may be NULL. */
nsfrb_status nsfrb_imager_info(nsfrb_imager_t im, int32_t *u_max, int32_t *v_max, int64_t *n_entries);

/* d_vis: device FP32 [n_t][n_sub][n_chan][n_base][2 pol][re, im], 16-byte
 * aligned.  d_img: device FP32 [n_t][n_sub][N][N] (the serving block layout
 * when N x N is the search plan's ny x nx).  Asynchronous on `stream`.
 * Accumulates in FP32 (gridding in a fixed order: results are reproducible
 * bit for bit).  The first call with more images than any before allocates
 * the imager's workspace (n_t * n_sub * n_chan partial grids) and
 * synchronises the device. */
nsfrb_status nsfrb_image(nsfrb_imager_t im, const float *d_vis, int32_t n_t, float *d_img, void *stream);

/* Synchronous check of the imaging calls so far: ETIMEOUT if a bulk copy of
 * visibilities into shared memory did not complete within the kernel's 2 s
 * wait limit (the images of that call are then incomplete; the flag is
 * cleared), OK otherwise. */
nsfrb_status nsfrb_imager_status(nsfrb_imager_t im);
void nsfrb_imager_destroy(nsfrb_imager_t im);

/* ---- candidate classifier (Sec. 2.3: convolutional blocks with batch
 * normalisation, a non-linearity and max-pooling, a small fully connected
 * head with dropout, one logit per candidate interpreted through a sigmoid as
 * the RFI probability p_rfi; binary cross-entropy; Adam) ------------------
 * Network: 4 x {conv3d 3x3x3 (padding 1, no bias) -> batch norm -> ReLU ->
 * max-pool 2x2x2} over cutouts [d][h][w][c0] (time, rows, cols, subbands as
 * channels, BF16, channels last), then FC(f) -> ReLU -> dropout -> FC(1).
 * Convolutions run as BF16 tensor-core GEMMs with FP32 accumulation; the
 * parameters, batch-norm statistics, head, loss and Adam are FP32.
 * Parameter vector layout (FP32, flat): for l = 0..3: W_l[c_l][27][c_{l-1}]
 * (tap k = (kz*3+ky)*3+kx), gamma_l[c_l], beta_l[c_l]; then fc1_w[f][fin],
 * fc1_b[f], fc2_w[f], fc2_b[1], fin = d/16 * h/16 * w/16 * c_3.
 * Dropout keeps hidden unit (b, j) at training step s iff the first word of
 * Philox4x32-10 (counter (b*f + j, s, 0, 0), key = seed) >> 8, times 2^-24,
 * is >= dropout; kept units are scaled by 1/(1 - dropout). */
typedef struct nsfrb_clf_s *nsfrb_clf_t;

typedef struct {
    int32_t batch;          /* largest batch per call                              */
    int32_t d, h, w;        /* cutout time samples, rows, columns (multiples of 16) */
    int32_t c0;             /* subbands = input channels (multiple of 8)            */
    int32_t c[4];           /* channels of the four conv blocks (multiples of 8, <= 256) */
    int32_t f;              /* hidden units of the head (1..1024)                   */
    float dropout;          /* dropout rate of the hidden units, [0, 1)             */
    uint64_t seed;          /* dropout key                                          */
    float lr, beta1, beta2, eps;   /* Adam                                          */
    float bn_momentum;      /* running statistics: r <- (1-m) r + m batch value
                               (variance: unbiased)                                 */
} nsfrb_clf_config;

/* Create a classifier (device memory for the batch size; parameters zero,
 * running mean 0 and variance 1, Adam state zero, step 0).  EINVAL, ENOMEM. */
nsfrb_status nsfrb_clf_create(const nsfrb_clf_config *cfg, nsfrb_clf_t *out);
nsfrb_status nsfrb_clf_n_params(nsfrb_clf_t clf, int64_t *n);
/* Host copies of the flat FP32 parameter vector / the gradient of the last
 * training step / the running statistics ([sum c_l] each, block after block). */
nsfrb_status nsfrb_clf_set_params(nsfrb_clf_t clf, const float *h_params);
nsfrb_status nsfrb_clf_get_params(nsfrb_clf_t clf, float *h_params);
nsfrb_status nsfrb_clf_get_grads(nsfrb_clf_t clf, float *h_grads);
nsfrb_status nsfrb_clf_get_bn_stats(nsfrb_clf_t clf, float *h_run_mean, float *h_run_var);
nsfrb_status nsfrb_clf_set_bn_stats(nsfrb_clf_t clf, const float *h_run_mean, const float *h_run_var);

/* One training step on d_x[batch][d][h][w][c0] (BF16, device) with labels
 * d_labels[batch] (FP32 0 = astrophysical, 1 = artefact): forward with batch
 * statistics (running statistics updated), mean BCE, backward into the
 * gradient vector, and, if update != 0, one Adam step (then the step counter,
 * which also indexes the dropout masks, advances).  *h_loss (optional, waits)
 * receives the batch loss.  Asynchronous otherwise. */
nsfrb_status nsfrb_clf_train_step(nsfrb_clf_t clf, const void *d_x, const float *d_labels, int32_t batch,
                                  int32_t update, float *h_loss, void *stream);

/* Inference (running statistics, no dropout): d_logit[batch] (device);
 * p_rfi = 1 / (1 + exp(-logit)). */
nsfrb_status nsfrb_clf_infer(nsfrb_clf_t clf, const void *d_x, int32_t batch, float *d_logit, void *stream);

/* Cutouts around candidates of a plan's cube: d_out[n][d][h][w][n_sub] BF16.
 * The window is centred on the candidate pixel and on t_idx + (w + smax)/2
 * (w its width, smax its DM's largest shift); time is averaged in bins of
 * b = max(1, ceil((w + smax) / (d/2))) samples so that the dispersed pulse
 * spans at most half the cutout; values are divided by the candidate pixel's
 * noise per subband and sample (sigma_D / sqrt(n_sub); d_sigma NULL: 1);
 * zero outside the image and the window.  d_cube as for nsfrb_search. */
nsfrb_status nsfrb_clf_cutouts(nsfrb_plan_t plan, const void *d_cube, const float *d_sigma,
                               const nsfrb_candidate *d_cand, int32_t n, int32_t d, int32_t h, int32_t w,
                               void *d_out, void *stream);

/* Checkpoint: configuration, parameters, Adam state, running statistics and
 * the step counter, to / from a binary file.  EINVAL on a mismatched file. */
nsfrb_status nsfrb_clf_save(nsfrb_clf_t clf, const char *path);
nsfrb_status nsfrb_clf_load(nsfrb_clf_t clf, const char *path);
void nsfrb_clf_destroy(nsfrb_clf_t clf);

/* Release everything the plan owns (device memory, streams, graphs). */
void nsfrb_destroy(nsfrb_plan_t plan);

/* Static text for a status, and the last error text recorded on this thread. */
const char *nsfrb_strerror(nsfrb_status s);
const char *nsfrb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NSFRB_H */
