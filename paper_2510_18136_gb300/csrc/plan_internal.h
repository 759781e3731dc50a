// The plan object behind nsfrb_plan_t and helpers shared by the host files.
#pragma once

#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "nsfrb.h"
#include "nsfrb_internal.h"

namespace nsfrb {
constexpr int kSlabs = 8;   // host-buffer search: H2D copy / search pipeline depth
}

struct nsfrb_plan_s {
    nsfrb_config cfg{};
    std::vector<double> freq, dm;
    std::vector<int32_t> widths;
    std::vector<int32_t> shifts;   // [n_dm][n_sub]
    std::vector<int32_t> smax;     // [n_dm]
    std::vector<int32_t> table;    // info | deltas | unique-row shifts (see SearchParams)
    int n_u = 0, n_u_active = 0, n_deltas = 0;
    int C = 0, Tp = 0;
    int32_t wclass[nsfrb::kMaxW] = {};
    // barrier-free kernel pixel x DM tile (10 * teams + buffers per team) per storage type of the
    // searched rows (FP32, BF16, FP16); 0 = the first of the default order that fits
    int32_t tile[3] = {0, 0, 0};
    int32_t last_tile = 0, last_tile_st = -1;   // tile and storage type of the last search launch

    // device state (allocated on first use)
    bool dev_ready = false;
    int device = 0, n_sm = 0, max_smem = 0;
    int32_t n_blocks = 0;
    int32_t *d_table = nullptr;
    nsfrb::PixRec *d_rec = nullptr;
    nsfrb::CandRec *d_cand = nullptr;
    int32_t *d_counts = nullptr;   // [n_blocks] | err | n_cand | n_list | spare
    int32_t *d_err = nullptr, *d_ncand = nullptr, *d_nlist = nullptr;
    int32_t *d_list = nullptr;
    float *d_madws = nullptr;      // MAD mode: normalised FP32 slab [mad_slab][n_sub][n_t]
    uint8_t *d_bad = nullptr;      //   and the per-pixel zero-MAD flags [n_pix]
    int64_t mad_slab = 0;
    float *d_full_snr = nullptr;
    int16_t *d_full_t = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t t_start = nullptr, t_search = nullptr, t_end = nullptr;   // timing of the last search
    bool searched = false;
    nsfrb_status latched = NSFRB_OK;

    // host-buffer search
    void *d_hcube = nullptr;
    float *d_hsigma = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t slab_ev[nsfrb::kSlabs + 1] = {};

    // serving
    bool streaming = false;
    int32_t n_blk = 0;
    int64_t ring_len = 0;          // samples per (pixel, subband) ring row
    void *d_ring = nullptr;
    float *d_blk = nullptr;        // [n_blk][n_sub][n_pix] FP32 block on the device
    int32_t *d_sstate = nullptr;   // [0] window start in the ring row, [1] samples written mod n_t
    float *h_fring = nullptr;      // re-score: FP32 window [n_t][n_sub][n_pix], a ring of n_t sample
    float *d_fring = nullptr;      //   planes: in device memory (d_fring, h_fring null) when the
    bool fring_dev = false;        //   admission budget allows, else pinned host memory (h_fring,
                                   //   mapped; d_fring its device address)
    cudaStream_t s_stream = nullptr;
    cudaGraphExec_t s_graph = nullptr;
    cudaEvent_t s_ev_push = nullptr, s_ev_done = nullptr;
    uint32_t *d_mask = nullptr;

    // classifier cutouts: per-DM largest shift and the widths, on the device
    int32_t *d_smax_w = nullptr;
    int64_t n_pushed = 0;
    bool pending = false;
};

namespace nsfrb {
void set_error(const std::string &msg);
nsfrb_status fail(nsfrb_plan_s *p, nsfrb_status st, const std::string &msg);
nsfrb_status cuda_check(nsfrb_plan_s *p, cudaError_t e, const char *what);
nsfrb_status ensure_device(nsfrb_plan_s *pl);
nsfrb_status queue_search(nsfrb_plan_s *pl, const void *cube, int64_t cube_pix0, int dtype, int64_t row_len,
                          int t_off, const float *sigma, int64_t pix0, int64_t n, const int32_t *pix_list,
                          const int32_t *n_items_dev, int new_blk, cudaStream_t s,
                          const int32_t *t_off_dev = nullptr, int t_wrap = 0, int64_t t_stride = 0);
size_t elem_size(int dtype);
void destroy_stream_state(nsfrb_plan_s *pl);
void base_params(const nsfrb_plan_s *pl, SearchParams &sp);
bool choose_stage(const nsfrb_plan_s *pl, SearchParams &sp, size_t &smem);
bool choose_stage_for(int C, int max_smem, SearchParams &sp, size_t &smem, int tile_pref = 0);

cudaError_t launch_search_c1(const SearchParams &, int, size_t, cudaStream_t);
cudaError_t launch_search_c3(const SearchParams &, int, size_t, cudaStream_t);
cudaError_t launch_search_c5(const SearchParams &, int, size_t, cudaStream_t);
cudaError_t launch_search_c9(const SearchParams &, int, size_t, cudaStream_t);
cudaError_t launch_search_c17(const SearchParams &, int, size_t, cudaStream_t);
cudaError_t launch_search_c25(const SearchParams &, int, size_t, cudaStream_t);
cudaError_t launch_search_c38(const SearchParams &, int, size_t, cudaStream_t);
cudaError_t launch_search_c39(const SearchParams &, int, size_t, cudaStream_t);
cudaError_t prepare_search_c1(size_t);
cudaError_t prepare_search_c3(size_t);
cudaError_t prepare_search_c5(size_t);
cudaError_t prepare_search_c9(size_t);
cudaError_t prepare_search_c17(size_t);
cudaError_t prepare_search_c25(size_t);
cudaError_t prepare_search_c38(size_t);
cudaError_t prepare_search_c39(size_t);
}  // namespace nsfrb
