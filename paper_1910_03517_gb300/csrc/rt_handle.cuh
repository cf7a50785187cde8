// The host runtime's handle (rt.h's opaque rt_handle) and the helpers the
// runtime's translation units share (rt_api.cu, rt_surrogate.cu).
#pragma once
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "rt_internal.cuh"

typedef struct rt_mlp rt_mlp;

namespace rt {
namespace host {

struct SurrogateState;   // rt_surrogate.cu

constexpr int kEvRing = 4;
constexpr int kQRing = 3;
#ifndef RT_STRIP_ROWS
#define RT_STRIP_ROWS 64
#endif
constexpr int kStripRows = RT_STRIP_ROWS;   // rows of one pass-A work item
constexpr uint32_t kStateMagic = 0x52545331u;
constexpr int kMaxProfiled = 4096;  // frame sets whose pass times one collection keeps

// CUDA events around the passes of one frame set (profiling)
struct ProfEv {
    cudaEvent_t a0, a1, s0, s1, b0, b1, c1;
    bool crops, all;
};

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace host
}  // namespace rt

struct rt_handle {
    using ProfEv = rt::host::ProfEv;
    static constexpr int kEvRing = rt::host::kEvRing, kQRing = rt::host::kQRing;
    rt_array_params p{};
    std::vector<rt_camera_desc> cams;
    int dev = 0, sm_count = 0;
    cudaStream_t user = nullptr, s_stats = nullptr, s_solve = nullptr, s_main = nullptr, s_copy = nullptr,
                 s_d2h = nullptr;
    cudaStream_t s_prof[3] = {nullptr, nullptr, nullptr};   // timing branches of s_stats, s_solve, s_main
    rt::ArrayGeom geom{};
    int Hmax = 0;
    // outputs and statistics
    uint8_t *rgb[2] = {nullptr, nullptr};
    std::vector<size_t> rgb_off;
    size_t rgb_bytes = 0;
    uint32_t *frame_hist[2] = {nullptr, nullptr};
    uint32_t *thumbs[3] = {nullptr, nullptr, nullptr};   // ring of three: frame set t in slot t % 3
    uint32_t *strip_hist[3] = {nullptr, nullptr, nullptr};
    uint32_t *strip_n[3] = {nullptr, nullptr, nullptr};
    unsigned long long *strip_sum[3] = {nullptr, nullptr, nullptr}, *strip_sumsq[3] = {nullptr, nullptr, nullptr};
    unsigned long long *strip_joint[3] = {nullptr, nullptr, nullptr};   // [K][2][B][10] (3 x 3 maps)
    uint8_t *luma[2] = {nullptr, nullptr};
    size_t luma_cam_stride = 0;
    double *maps_new = nullptr, *E = nullptr;
    int32_t *q16[kQRing] = {nullptr, nullptr, nullptr};
    int32_t *q16_identity = nullptr;
    // seam maps applied per block: the column coefficients of each Q16 slot
    // (and of the identity) for the table variant of pass B, written after
    // each solve
    uint4 *coef[kQRing] = {nullptr, nullptr, nullptr};
    uint4 *coef_identity = nullptr;
    int32_t *ramp = nullptr;
    rt::StripItem *items = nullptr;
    int n_items = 0;
    int32_t *group_start = nullptr, *group_members = nullptr, *left_nbr = nullptr, *right_nbr = nullptr,
            *cam_H = nullptr;
    int n_groups = 0;
    rt::SolveTopo solve_topo{};
    // seams (left camera, right camera) in chain order, and their costs
    std::vector<int2> seam_list;
    int2 *seams = nullptr;
    double *seam_cost[2] = {nullptr, nullptr};
    double *seam_rows = nullptr;   // per averaged row terms [seams][seam_max_rows]
    int seam_max_rows = 0;
    // difference attention
    rt::AttnArgs attn{};
    uint8_t *luma_copy[2] = {nullptr, nullptr};
    uint32_t *attn_cells = nullptr;
    rt_crop *props[2] = {nullptr, nullptr};
    int32_t *prop_count[2] = {nullptr, nullptr};
    cudaStream_t s_attn = nullptr, s_aux = nullptr;   // attention; seam costs
    cudaEvent_t ev_attn[4] = {}, ev_pb[4] = {}, ev_seam[4] = {};
    bool crops_from_props[2] = {false, false};
    bool attn_valid = false;       // luma_copy of the previous frame set holds its luma
    int32_t *q16_rows[2] = {nullptr, nullptr};   // per-row blended maps [K][2][Hmax][3][2]
    __half *crops[2] = {nullptr, nullptr};
    rt_crop *crop_dev[2] = {nullptr, nullptr};
    rt_crop *crop_host = nullptr;          // pinned [2][max_crops]
    int n_crops[2] = {0, 0};
    // host-input staging
    uint8_t *stage[2] = {nullptr, nullptr};
    std::vector<size_t> stage_y_off, stage_uv_off;
    size_t stage_bytes = 0;
    // events
    cudaEvent_t ev_user = nullptr, ev_in = nullptr, ev_tmp = nullptr;
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;   // autotuner timing
    cudaEvent_t ev_a[kEvRing] = {}, ev_solved[kEvRing] = {}, ev_done[kEvRing] = {}, ev_out[kEvRing] = {};
    bool launched[kEvRing] = {}, out_launched[kEvRing] = {};
    int64_t t = 0;                 // frame sets submitted
    bool restart = true;           // next submit starts a sequence
    bool last_first = true;        // the last frame set started its sequence
    // profiling
    bool prof_on = false, prof_all = true;
    std::vector<ProfEv> prof, cap_prof;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_pool_used = 0;
    bool last_was_graph = false;
    bool graph_launched = false;   // the captured graph ran since profiling started
    // captured sequence
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int cap_n = 0;
    int64_t cap_t0 = 0;
    bool capturing = false;
    rt_crop *cap_crops = nullptr;
    size_t cap_crops_n = 0;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_mark = nullptr;
    bool prof_branch[3] = {false, false, false};   // the capture in progress used s_prof[i]
    // launch shapes (rt_autotune / rt_set_tuning)
    int pb_grid = 0, pb_threads = RT_PASS_B_RUN_THREADS, pb_ctas = RT_PASS_B_RUN_CTAS;
    // threads of the 128-register pass B variants (thumbnails, seam maps
    // computed per unit): the tuned pb_threads once a shape is set
    int pb_threads_wide = RT_PASS_B_WIDE_RUN_THREADS;
    int pa_rows = rt::host::kStripRows, pa_threads = 64, crop_threads = 256, crop_grid = 64;
    rt_tuning tuned{};
    size_t pb_smem = 0;
    std::string err;
    size_t n_maps = 0;             // K*2*B*6, or K*2*B*12 for the 3 x 3 maps
    // surrogate inference buffers (allocated on first use)
    void *sg_x = nullptr;          // BF16 [K][6912]
    float *sg_y = nullptr;         // [K][3]
    double *sg_maps = nullptr, *sg_err = nullptr;
    // the handle's own surrogate network and its training / pipeline state
    // (rt_surrogate.cu)
    rt::host::SurrogateState *sg = nullptr;
};


namespace rt {
namespace host {

extern thread_local std::string g_config_error;

inline rt_status fail(rt_handle *h, rt_status s, const std::string &msg)
{
    if (h) h->err = msg;
    else g_config_error = msg;
    return s;
}

inline rt_status cuda_fail(rt_handle *h, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, m);
}

#define RT_CUDA(h, call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

inline rt_status wait_event(rt_handle *h, cudaEvent_t ev, int32_t timeout_ms)
{
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return RT_OK;
        if (e != cudaErrorNotReady) return cuda_fail(h, e, "cudaEventQuery");
        if (timeout_ms >= 0) {
            auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
            if (ms >= timeout_ms) return fail(h, RT_ERR_TIMEOUT, "timed out waiting for the GPU");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

template <class T>
rt_status dalloc(rt_handle *h, T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) return RT_OK;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");
    e = cudaMemset(*p, 0, n * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemset");
    return RT_OK;
}

// Learned surrogate (rt_surrogate.cu): the pipeline hooks of the surrogate
// mode and the handle's network.
rt_status surrogate_ready(rt_handle *h);
const int32_t *surrogate_gate(rt_handle *h);
rt_status surrogate_predict_step(rt_handle *h, const uint32_t *prev_thumbs, bool first);
rt_status surrogate_select_step(rt_handle *h, int32_t *q16, bool first);
void surrogate_free(rt_handle *h);
size_t surrogate_state_bytes(const rt_handle *h);
rt_status surrogate_state_save(rt_handle *h, uint8_t *out);
rt_status surrogate_state_load(rt_handle *h, const uint8_t *in);
rt_mlp *surrogate_net(rt_handle *h);

}  // namespace host
}  // namespace rt
