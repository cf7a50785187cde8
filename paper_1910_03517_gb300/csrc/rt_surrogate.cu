// The learned gain surrogate of a camera array (include/rt_surrogate.h): its
// training on synthetic arrays labelled by the array's own plain fit, its
// evaluation, checkpoints, and the surrogate mode of the frame-set pipeline.
//
// Training set.  A frame set of the array's own cameras is painted on the
// device (k_synth.cu) with a random scene, a random illuminant common to the
// array and random per-camera per-channel gains; the band statistics (pass
// A), the per-camera gain fit (the solve, first frame set of a sequence, no
// smoothing) and the thumbnails (pass B) of the handle's kernels give one
// sample per camera: features = thumbnail cell means / 255 - 0.5 (BF16),
// label = the fit's three log-gains.  Everything stays on the device.
//
// Surrogate mode (rt_array_params.surrogate_mode = 1).  Per frame set t, on
// the statistics stream: the thumbnails of frame set t-1 (from pass B(t-1))
// go through the network; the predicted log-gains are re-gauged per seam
// chain (the chain's mean subtracted, the fit's gauge) and clamped like the
// fit's gains.  A device-side decision then sets whether the plain fit runs
// for t: always while the surrogate is on probation (fallback), on the
// first frame set of a sequence, and every judge_every-th frame set.  When
// it runs (pass A and the fit, gated on the device), it judges the
// prediction: error = max |g_pred / g_fit - 1| over cameras and channels;
// above fallback_tol the plain fit is applied and the fallback stays (or
// switches) on, otherwise the prediction is applied and the fallback is
// cleared.  The chosen gains are smoothed and quantised exactly as the solve
// does.  No host synchronisation: the whole mode captures into a graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "rt_handle.cuh"
#include "mlp_internal.cuh"
#include "q16.cuh"
#include "../../include/rt_surrogate.h"

using namespace rt;
using namespace rt::host;

namespace rt {
namespace host {

// Device state of the surrogate mode.
struct SgDev {
    int32_t need_plain;     // this frame set runs the band statistics and the fit (pass A's gate[0])
    int32_t motion_ok;      // pass A may use the previous frame set's band luma (gate[1])
    int32_t ran_a;          // the last frame set's pass A ran
    int32_t fallback;       // the plain fit is applied until a judgement passes
    int32_t have_pred;      // this frame set has a prediction
    int32_t count;          // frame sets since the sequence started
    int32_t frames, predicted, plain, judged, judged_failed, pad;
    double tol, last_err, max_err;
};

struct SurrogateState {
    rt_mlp *net = nullptr;
    int64_t train_calls = 0;
    // training set: features [n][6912] BF16, labels [n][3], shuffle order
    __nv_bfloat16 *ds_x = nullptr;
    float *ds_t = nullptr;
    int32_t *ds_idx = nullptr;
    int64_t ds_cap = 0, ds_n = 0;
    uint64_t ds_seed = 0;
    bool ds_valid = false;
    // evaluation set and outputs
    __nv_bfloat16 *ev_x = nullptr;
    float *ev_t = nullptr, *ev_y = nullptr;
    double *ev_err = nullptr, *ev_err_id = nullptr;
    int64_t ev_cap = 0;
    // one generated frame set and the kernels' working buffers for it
    uint8_t *gen = nullptr;
    std::vector<size_t> gen_y, gen_uv;
    uint8_t *gen_rgb = nullptr, *gen_luma = nullptr;
    uint32_t *gen_hist = nullptr, *gen_thumbs[2] = {nullptr, nullptr};
    unsigned long long *gen_sum = nullptr;
    double *gen_maps = nullptr, *gen_E = nullptr;
    int32_t *gen_q16 = nullptr;
    int gen_par = 0;
    float *loss_hist = nullptr;
    int64_t loss_cap = 0;
    std::vector<float> losses;     // of the last rt_surrogate_train
    // surrogate mode
    SgDev *dev = nullptr;
    double *pred = nullptr;        // predicted gains, layout of the maps [K][2][1][3][2]
    int skip_pred = 0;             // frame sets without a prediction (after a state restore)
};

}  // namespace host
}  // namespace rt

namespace {

constexpr uint32_t kFileMagic = 0x47535452u;   // "RTSG"
constexpr uint32_t kFileVersion = 1;

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double unif(uint64_t &s) { return (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// labels[k][c] = log g of the fit (maps [K][2][1][3][2], side 0)
__global__ void labels_kernel(const double *__restrict__ maps, int K, float *__restrict__ out)
{
    const int i = threadIdx.x;
    if (i < K * 3) out[i] = (float)log(maps[((i / 3) * 2 * 3 + i % 3) * 2]);
}

// Re-gauged predicted log-gains per chain, clamped gains.  y [K][3].
__device__ __forceinline__ void predict_chain(const float *y, const SolveTopo &topo, int grp, int c, double gmin,
                                              double gmax, double *pred)
{
    const int g0 = topo.gstart[grp], n = topo.gstart[grp + 1] - g0;
    double mean = 0.0;
    for (int i = 0; i < n; ++i) mean += (double)y[topo.member[g0 + i] * 3 + c];
    mean /= n;
    for (int i = 0; i < n; ++i) {
        const int cam = topo.member[g0 + i];
        const double g = fmin(fmax(exp((double)y[cam * 3 + c] - mean), gmin), gmax);
        for (int side = 0; side < 2; ++side) {
            pred[((cam * 2 + side) * 3 + c) * 2] = g;
            pred[((cam * 2 + side) * 3 + c) * 2 + 1] = 0.0;
        }
    }
}

// Per-camera evaluation error of predictions y [sets][K][3] against labels:
// max over channels of |exp(re-gauged y - label) - 1|.  One thread per
// (set, chain).
__global__ void eval_err_kernel(const float *__restrict__ y, const float *__restrict__ lab, int K, int sets,
                                const SolveTopo topo, int n_groups, double *__restrict__ err,
                                double *__restrict__ err_id)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= sets * n_groups) return;
    const int s = t / n_groups, grp = t % n_groups;
    const int g0 = topo.gstart[grp], n = topo.gstart[grp + 1] - g0;
    double mean[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) mean[c] += (double)y[((size_t)s * K + topo.member[g0 + i]) * 3 + c];
    for (int i = 0; i < n; ++i) {
        const size_t row = (size_t)s * K + topo.member[g0 + i];
        double e = 0.0, e0 = 0.0;
        for (int c = 0; c < 3; ++c) {
            e = fmax(e, fabs(exp((double)y[row * 3 + c] - mean[c] / n - (double)lab[row * 3 + c]) - 1.0));
            e0 = fmax(e0, fabs(exp(-(double)lab[row * 3 + c]) - 1.0));
        }
        err[row] = e;
        err_id[row] = e0;
    }
}

// Surrogate mode, before pass A: the prediction for this frame set (from the
// network's outputs y for the previous frame set's thumbnails) and whether
// the plain fit runs.  One CTA.
__global__ void __launch_bounds__(128) sg_decide_kernel(SgDev *__restrict__ st, const float *__restrict__ y, int first,
                                                        int no_pred, int lag, int judge_every, const SolveTopo topo,
                                                        int n_groups, double gmin, double gmax,
                                                        double *__restrict__ pred)
{
    __shared__ int s_have;
    if (threadIdx.x == 0) {
        if (first) {
            st->count = 0;
            st->fallback = 1;
            st->ran_a = 0;
        } else {
            st->count += 1;
        }
        // a prediction needs frame set t - lag inside the sequence
        st->have_pred = !(first || no_pred) && st->count >= lag;
        const int need = !st->have_pred || st->fallback || (st->count % judge_every) == 0;
        st->motion_ok = !first && st->ran_a;
        st->need_plain = need;
        st->ran_a = need;
        s_have = st->have_pred;
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (s_have && t < n_groups * 3) predict_chain(y, topo, t / 3, t % 3, gmin, gmax, pred);
}

// Surrogate mode, after the (gated) fit: the judgement, the choice between the
// fit and the prediction, then the solve's smoothing and Q16 quantisation of
// the chosen gains.  One CTA of 128 threads, one (camera, channel) each.
__global__ void __launch_bounds__(128) sg_select_kernel(SgDev *__restrict__ st, const double *__restrict__ fit,
                                                        const double *__restrict__ pred, double *__restrict__ E,
                                                        int32_t *__restrict__ q16, int K, int first, double alpha,
                                                        double one_m_alpha)
{
    __shared__ double s_err[128];
    __shared__ int s_plain;
    const int t = threadIdx.x;
    const bool judge = st->need_plain && st->have_pred;
    double e = 0.0;
    if (judge && t < K * 3) {
        const size_t i0 = (((size_t)(t / 3) * 2) * 3 + t % 3) * 2;
        e = fabs(pred[i0] / fit[i0] - 1.0);
    }
    s_err[t] = e;
    __syncthreads();
    if (t == 0) {
        double m = 0.0;
        for (int i = 0; i < 128; ++i) m = fmax(m, s_err[i]);
        if (judge) {
            st->judged += 1;
            st->last_err = m;
            st->max_err = fmax(st->max_err, m);
            const int fail = !(m <= st->tol);
            st->judged_failed += fail;
            st->fallback = fail;
        }
        const int plain = st->need_plain && (st->fallback || !st->have_pred);
        st->frames += 1;
        st->plain += plain;
        st->predicted += !plain;
        s_plain = plain;
    }
    __syncthreads();
    if (t >= K * 3) return;
    const int cam = t / 3, c = t % 3;
    const size_t i0 = (((size_t)cam * 2) * 3 + c) * 2, i1 = (((size_t)cam * 2 + 1) * 3 + c) * 2;
    const double g = s_plain ? fit[i0] : pred[i0];
    double2 ev;
    if (first) {
        ev = make_double2(g, 0.0);
    } else {
        const double2 old = *reinterpret_cast<const double2 *>(E + i0);
        ev.x = fma(one_m_alpha, old.x, alpha * g);
        ev.y = one_m_alpha * old.y;
    }
    const int2 q = make_int2(q16_round(ev.x), q16_round(ev.y));
    *reinterpret_cast<double2 *>(E + i0) = ev;
    *reinterpret_cast<double2 *>(E + i1) = ev;
    *reinterpret_cast<int2 *>(q16 + i0) = q;
    *reinterpret_cast<int2 *>(q16 + i1) = q;
}

__global__ void sg_set_tol_kernel(SgDev *st, double tol, int reset)
{
    st->tol = tol;
    if (reset) {
        st->frames = st->predicted = st->plain = st->judged = st->judged_failed = 0;
        st->last_err = st->max_err = 0.0;
    }
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------

bool surrogate_config_ok(const rt_handle *h)
{
    return h->p.fit_mode == RT_FIT_GLOBAL && h->p.num_blocks == 1 && (h->p.flags & RT_FLAG_THUMBNAILS);
}

rt_status ensure_state(rt_handle *h)
{
    if (!h->sg) h->sg = new SurrogateState();
    return RT_OK;
}

// He-style initial weights (normal, variance 2 / fan-in; the output layer's
// halved), zero biases, drawn from the seed.
rt_status init_net(rt_handle *h, uint64_t seed)
{
    SurrogateState &S = *h->sg;
    rt_status s = rt_mlp_create(&S.net, h->s_main);
    if (s != RT_OK) return fail(h, s, "rt_mlp_create");
    std::vector<float> P(RT_MLP_PARAMS, 0.0f);
    uint64_t st = seed ^ 0xA5A5A5A55A5A5A5Aull;
    auto normal = [&]() {
        const double u1 = (unif(st) + 1e-300), u2 = unif(st);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
    };
    const size_t n1 = (size_t)256 * kMlpIn, n2 = (size_t)256 * 256, n3 = (size_t)3 * 256;
    const size_t o1 = 0, o2 = n1 + 256, o3 = o2 + n2 + 256;
    for (size_t i = 0; i < n1; ++i) P[o1 + i] = (float)(normal() * std::sqrt(2.0 / kMlpIn));
    for (size_t i = 0; i < n2; ++i) P[o2 + i] = (float)(normal() * std::sqrt(2.0 / 256.0));
    for (size_t i = 0; i < n3; ++i) P[o3 + i] = (float)(0.5 * normal() * std::sqrt(2.0 / 256.0));
    if ((s = rt_mlp_set_params(S.net, P.data(), P.size())) != RT_OK)
        return fail(h, s, std::string("surrogate network: ") + rt_mlp_last_error(S.net));
    return RT_OK;
}

// Working buffers of frame-set generation (allocated on first use).
rt_status ensure_gen(rt_handle *h)
{
    SurrogateState &S = *h->sg;
    if (S.gen) return RT_OK;
    const int K = h->p.num_cameras;
    size_t off = 0;
    S.gen_y.resize(K);
    S.gen_uv.resize(K);
    for (int k = 0; k < K; ++k) {
        const rt_camera_desc &c = h->cams[k];
        S.gen_y[k] = off;
        off += align_up((size_t)c.y_pitch * c.height, 256);
        S.gen_uv[k] = off;
        if (c.format == RT_NV12) off += align_up((size_t)c.uv_pitch * (c.height / 2), 256);
    }
    rt_status s;
    const size_t nb = (size_t)K * 2;
    if ((s = dalloc(h, &S.gen, off)) != RT_OK) return s;
    if ((s = dalloc(h, &S.gen_rgb, h->rgb_bytes + 64)) != RT_OK) return s;
    if ((s = dalloc(h, &S.gen_luma, (size_t)K * h->luma_cam_stride)) != RT_OK) return s;
    if ((s = dalloc(h, &S.gen_hist, nb * 768 + nb * 3)) != RT_OK) return s;
    if ((s = dalloc(h, &S.gen_sum, nb * 3 * 2)) != RT_OK) return s;
    for (int i = 0; i < 2; ++i)
        if ((s = dalloc(h, &S.gen_thumbs[i], (size_t)K * kMlpIn)) != RT_OK) return s;
    if ((s = dalloc(h, &S.gen_maps, h->n_maps)) != RT_OK) return s;
    if ((s = dalloc(h, &S.gen_E, h->n_maps)) != RT_OK) return s;
    if ((s = dalloc(h, &S.gen_q16, h->n_maps)) != RT_OK) return s;
    return RT_OK;
}

// One synthetic frame set of the array (index `set` of the stream `seed`),
// its plain fit and thumbnails: features x_out [K][6912], labels t_out [K][3].
rt_status gen_sample(rt_handle *h, uint64_t seed, int64_t set, __nv_bfloat16 *x_out, float *t_out)
{
    SurrogateState &S = *h->sg;
    const rt_array_params &p = h->p;
    const int K = p.num_cameras;
    cudaStream_t st = h->s_main;
    uint64_t rs = seed * 0x2545F4914F6CDD1Dull + (uint64_t)set * 0x9E3779B97F4A7C15ull + 0x1234567ull;
    SynthArgs sa;
    memset(&sa, 0, sizeof sa);
    sa.K = K;
    for (int i = 0; i < 16; ++i) sa.ph[i] = (float)unif(rs);
    double illum[3];
    for (int c = 0; c < 3; ++c) illum[c] = 0.8 + 0.45 * unif(rs);
    // panorama column of each camera: cameras of a chain side by side
    std::vector<float> x0(K, 0.0f);
    for (int g = 0; g < h->n_groups; ++g) {
        float x = 0.0f;
        for (int i = h->solve_topo.gstart[g]; i < h->solve_topo.gstart[g + 1]; ++i) {
            const int k = h->solve_topo.member[i];
            x0[k] = x;
            x += (float)h->cams[k].width;
        }
    }
    uint32_t blocks = 0;
    ArrayGeom g = h->geom;
    for (int k = 0; k < K; ++k) {
        const rt_camera_desc &c = h->cams[k];
        sa.y[k] = S.gen + S.gen_y[k];
        sa.uv[k] = c.format == RT_NV12 ? S.gen + S.gen_uv[k] : nullptr;
        sa.W[k] = c.width; sa.H[k] = c.height; sa.y_pitch[k] = c.y_pitch; sa.uv_pitch[k] = c.uv_pitch;
        sa.fmt[k] = c.format; sa.bits[k] = c.format == RT_MONO16 ? 12 : 8;
        if (c.format == RT_MONO16) sa.bits[k] = std::min(std::max(c.bit_depth, 8), 15);
        sa.x0[k] = x0[k];
        for (int ch = 0; ch < 3; ++ch)
            sa.gain[k][ch] = (float)std::min(std::max((0.6 + 0.9 * unif(rs)) * illum[ch], 0.45), 1.9);
        sa.block_base[k] = blocks;
        blocks += (uint32_t)(c.width / 2) * (uint32_t)(c.height / 2);
        g.cam[k].y = sa.y[k];
        g.cam[k].uv = sa.uv[k];
        g.cam[k].rgb = S.gen_rgb + h->rgb_off[k];
    }
    sa.block_base[K] = blocks;
    sa.noise = 4.0f;
    sa.key_lo = (uint32_t)splitmix(rs);
    sa.key_hi = (uint32_t)splitmix(rs);
    RT_CUDA(h, launch_synth(sa, st));
    // band statistics of the first frame set of a sequence (no motion test)
    const size_t nb = (size_t)K * 2;
    RT_CUDA(h, cudaMemsetAsync(S.gen_hist, 0, (nb * 768 + nb * 3) * 4, st));
    RT_CUDA(h, cudaMemsetAsync(S.gen_sum, 0, nb * 3 * 2 * 8, st));
    PassAArgs pa{};
    pa.items = h->items; pa.n_items = h->n_items; pa.S = p.strip_width; pa.T = p.motion_threshold; pa.first = 1;
    pa.prev_luma = nullptr; pa.cur_luma = S.gen_luma; pa.luma_cam_stride = (int32_t)h->luma_cam_stride;
    pa.hist = S.gen_hist; pa.n = S.gen_hist + nb * 768; pa.sum = S.gen_sum; pa.sumsq = S.gen_sum + nb * 3;
    RT_CUDA(h, launch_pass_a(g, pa, h->pa_threads, st));
    SolveArgs sv{};
    sv.n = pa.n; sv.sum = pa.sum; sv.sumsq = pa.sumsq; sv.hist = pa.hist;
    sv.maps_new = S.gen_maps; sv.E = S.gen_E; sv.q16 = S.gen_q16;
    sv.K = K; sv.B = 1; sv.S = p.strip_width; sv.fit_mode = RT_FIT_GLOBAL; sv.min_valid = p.min_valid;
    sv.first = 1; sv.alpha = p.alpha; sv.lambda = p.lambda; sv.gmin = p.gain_min; sv.gmax = p.gain_max;
    sv.n_groups = h->n_groups; sv.group_start = h->group_start; sv.group_members = h->group_members;
    sv.left_nbr = h->left_nbr; sv.right_nbr = h->right_nbr; sv.cam_H = h->cam_H; sv.topo = h->solve_topo;
    sv.fit_only = 1;
    RT_CUDA(h, launch_solve(sv, st));
    // thumbnails (pass B without frame statistics, identity maps); the buffers
    // alternate, each pass B clearing the other for the next
    PassBArgs pb{};
    pb.q16 = h->q16_identity;
    pb.thumbs = S.gen_thumbs[S.gen_par];
    pb.clear_b = S.gen_thumbs[S.gen_par ^ 1];
    pb.clear_b_n = (uint32_t)K * kMlpIn;
    RT_CUDA(h, launch_pass_b(g, pb, h->sm_count, h->pb_threads_wide, h->pb_smem, st));
    RT_CUDA(h, launch_thumb_features(g, S.gen_thumbs[S.gen_par], x_out, st));
    S.gen_par ^= 1;
    labels_kernel<<<1, 96, 0, st>>>(S.gen_maps, K, t_out);
    RT_CUDA(h, cudaGetLastError());
    return RT_OK;
}

rt_status gen_set(rt_handle *h, uint64_t seed, int64_t n_sets, __nv_bfloat16 *x, float *t)
{
    const int K = h->p.num_cameras;
    for (int64_t i = 0; i < n_sets; ++i) {
        rt_status s = gen_sample(h, seed, i, x + (size_t)i * K * kMlpIn, t + (size_t)i * K * 3);
        if (s != RT_OK) return s;
    }
    return RT_OK;
}

rt_status check_common(rt_handle *h)
{
    if (!surrogate_config_ok(h))
        return fail(h, RT_ERR_STATE, "the surrogate needs per-camera gains, one block and RT_FLAG_THUMBNAILS");
    if (h->capturing) return fail(h, RT_ERR_STATE, "not while a sequence is being captured");
    if (h->n_groups * 3 > 96) return fail(h, RT_ERR_INVALID, "at most 32 seam chains");
    return RT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// pipeline hooks (called by rt_api.cu's enqueue)
// ---------------------------------------------------------------------------

namespace rt {
namespace host {

rt_status surrogate_ready(rt_handle *h)
{
    if (!h->sg || !h->sg->net) return fail(h, RT_ERR_STATE, "no surrogate network (rt_surrogate_train or rt_surrogate_load)");
    rt_status s;
    SurrogateState &S = *h->sg;
    if (!S.dev) {
        if ((s = dalloc(h, &S.dev, 1)) != RT_OK) return s;
        if ((s = dalloc(h, &S.pred, h->n_maps)) != RT_OK) return s;
        sg_set_tol_kernel<<<1, 1, 0, h->s_solve>>>(S.dev, h->p.fallback_tol, 1);
        RT_CUDA(h, cudaGetLastError());
    }
    return RT_OK;
}

const int32_t *surrogate_gate(rt_handle *h) { return &h->sg->dev->need_plain; }

// Statistics stream, before pass A(t): predict from the thumbnails of frame
// set t - lag (lag = surrogate_mode: 1, or 2 so that the inference overlaps
// pass B(t-1)); none for the first lag frame sets of a sequence or after a
// state restore (thumbnails are not part of the state).
rt_status surrogate_predict_step(rt_handle *h, const uint32_t *prev_thumbs, bool first)
{
    SurrogateState &S = *h->sg;
    const int K = h->p.num_cameras;
    const bool no_pred = S.skip_pred > 0 && !h->capturing;
    if (!first && !no_pred) {
        RT_CUDA(h, launch_thumb_features(h->geom, prev_thumbs, mlp_input(S.net), h->s_stats));
        RT_CUDA(h, mlp_forward_async(S.net, K, h->s_stats));
    }
    sg_decide_kernel<<<1, 128, 0, h->s_stats>>>(S.dev, mlp_output(S.net), first ? 1 : 0, no_pred ? 1 : 0,
                                                h->p.surrogate_mode, h->p.judge_every, h->solve_topo, h->n_groups,
                                                h->p.gain_min, h->p.gain_max, S.pred);
    RT_CUDA(h, cudaGetLastError());
    if (!h->capturing && S.skip_pred > 0) --S.skip_pred;
    return RT_OK;
}

size_t surrogate_state_bytes(const rt_handle *h) { return h->p.surrogate_mode ? sizeof(SgDev) : 0; }

rt_status surrogate_state_save(rt_handle *h, uint8_t *out)
{
    if (!h->p.surrogate_mode) return RT_OK;
    if (h->sg && h->sg->dev) {
        RT_CUDA(h, cudaMemcpy(out, h->sg->dev, sizeof(SgDev), cudaMemcpyDeviceToHost));
    } else {
        SgDev d{};
        d.fallback = 1;
        d.tol = h->p.fallback_tol;
        memcpy(out, &d, sizeof d);
    }
    return RT_OK;
}

rt_status surrogate_state_load(rt_handle *h, const uint8_t *in)
{
    if (!h->p.surrogate_mode) return RT_OK;
    if (!h->sg || !h->sg->net) return RT_OK;   // nothing to restore into before a network exists
    rt_status s = surrogate_ready(h);
    if (s != RT_OK) return s;
    RT_CUDA(h, cudaMemcpy(h->sg->dev, in, sizeof(SgDev), cudaMemcpyHostToDevice));
    h->sg->skip_pred = h->p.surrogate_mode;     // their thumbnails are not part of the state
    return RT_OK;
}

// Solve stream, after the gated fit of t: judge, choose, smooth, quantise.
rt_status surrogate_select_step(rt_handle *h, int32_t *q16, bool first)
{
    SurrogateState &S = *h->sg;
    sg_select_kernel<<<1, 128, 0, h->s_solve>>>(S.dev, h->maps_new, S.pred, h->E, q16, h->p.num_cameras,
                                                first ? 1 : 0, h->p.alpha, 1.0 - h->p.alpha);
    RT_CUDA(h, cudaGetLastError());
    return RT_OK;
}

void surrogate_free(rt_handle *h)
{
    if (!h->sg) return;
    SurrogateState &S = *h->sg;
    auto F = [](void *p) { if (p) cudaFree(p); };
    if (S.net) rt_mlp_destroy(S.net);
    F(S.ds_x); F(S.ds_t); F(S.ds_idx); F(S.ev_x); F(S.ev_t); F(S.ev_y); F(S.ev_err); F(S.ev_err_id);
    F(S.gen); F(S.gen_rgb); F(S.gen_luma); F(S.gen_hist); F(S.gen_sum); F(S.gen_thumbs[0]); F(S.gen_thumbs[1]);
    F(S.gen_maps); F(S.gen_E); F(S.gen_q16); F(S.loss_hist); F(S.dev); F(S.pred);
    delete h->sg;
    h->sg = nullptr;
}

rt_mlp *surrogate_net(rt_handle *h) { return h->sg ? h->sg->net : nullptr; }

}  // namespace host
}  // namespace rt

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

rt_status rt_surrogate_train(rt_handle *h, int64_t n_samples, int32_t batch, double lr, uint64_t seed)
{
    if (!h) return RT_ERR_INVALID;
    rt_status s;
    if ((s = check_common(h)) != RT_OK) return s;
    const int K = h->p.num_cameras;
    if (batch < 1 || batch > kMlpMaxRows) return fail(h, RT_ERR_INVALID, "batch must be in 1..256");
    if (n_samples < batch || n_samples > (int64_t)1 << 26) return fail(h, RT_ERR_INVALID, "n_samples out of range");
    if (!(lr > 0.0) || !(lr < 1.0)) return fail(h, RT_ERR_INVALID, "lr must be in (0, 1)");
    if ((s = rt_sync(h, -1)) != RT_OK) return s;
    if ((s = ensure_state(h)) != RT_OK) return s;
    SurrogateState &S = *h->sg;
    if (!S.net && (s = init_net(h, seed)) != RT_OK) return s;
    if ((s = ensure_gen(h)) != RT_OK) return s;
    const int64_t n_sets = (n_samples + K - 1) / K;
    const int64_t rows = n_sets * K;
    if (!(S.ds_valid && S.ds_seed == seed && S.ds_n >= n_samples)) {
        if (S.ds_cap < rows) {
            cudaFree(S.ds_x); cudaFree(S.ds_t); cudaFree(S.ds_idx);
            S.ds_x = nullptr; S.ds_t = nullptr; S.ds_idx = nullptr; S.ds_cap = 0;
            if ((s = dalloc(h, &S.ds_x, (size_t)rows * kMlpIn)) != RT_OK) return s;
            if ((s = dalloc(h, &S.ds_t, (size_t)rows * 3)) != RT_OK) return s;
            if ((s = dalloc(h, &S.ds_idx, (size_t)rows)) != RT_OK) return s;
            S.ds_cap = rows;
        }
        S.ds_valid = false;
        if ((s = gen_set(h, seed, n_sets, S.ds_x, S.ds_t)) != RT_OK) return s;
        S.ds_valid = true;
        S.ds_seed = seed;
        S.ds_n = rows;
    }
    // the order of this pass over the samples (differs from call to call)
    std::vector<int32_t> order((size_t)n_samples);
    for (int64_t i = 0; i < n_samples; ++i) order[(size_t)i] = (int32_t)i;
    std::mt19937_64 rng(seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(S.train_calls + 1)));
    std::shuffle(order.begin(), order.end(), rng);
    RT_CUDA(h, cudaMemcpyAsync(S.ds_idx, order.data(), order.size() * 4, cudaMemcpyHostToDevice, h->s_main));
    const int64_t steps = n_samples / batch;
    if (S.loss_cap < steps) {
        cudaFree(S.loss_hist);
        S.loss_hist = nullptr;
        S.loss_cap = 0;
        if ((s = dalloc(h, &S.loss_hist, (size_t)steps)) != RT_OK) return s;
        S.loss_cap = steps;
    }
    for (int64_t i = 0; i < steps; ++i)
        RT_CUDA(h, mlp_train_batch_async(S.net, S.ds_x, S.ds_t, S.ds_idx + i * batch, batch, lr, S.loss_hist + i,
                                         h->s_main));
    std::string msg;
    if ((s = mlp_check(S.net, h->s_main, &msg)) != RT_OK) return fail(h, s, msg);
    S.losses.assign((size_t)steps, 0.0f);
    RT_CUDA(h, cudaMemcpy(S.losses.data(), S.loss_hist, (size_t)steps * 4, cudaMemcpyDeviceToHost));
    S.train_calls += 1;
    return RT_OK;
}

rt_status rt_surrogate_losses(rt_handle *h, float *losses, int64_t cap, int64_t *n)
{
    if (!h || !n) return RT_ERR_INVALID;
    *n = 0;
    if (!h->sg) return fail(h, RT_ERR_STATE, "no surrogate training yet");
    const std::vector<float> &L = h->sg->losses;
    *n = (int64_t)L.size();
    if (losses) memcpy(losses, L.data(), sizeof(float) * (size_t)std::min<int64_t>(cap, (int64_t)L.size()));
    return RT_OK;
}

rt_status rt_surrogate_evaluate(rt_handle *h, int64_t n_samples, uint64_t seed, double *errors,
                                double *errors_identity, int64_t cap, int64_t *n_out)
{
    if (!h) return RT_ERR_INVALID;
    rt_status s;
    if ((s = check_common(h)) != RT_OK) return s;
    if (!h->sg || !h->sg->net) return fail(h, RT_ERR_STATE, "no surrogate network (rt_surrogate_train or rt_surrogate_load)");
    const int K = h->p.num_cameras;
    if (n_samples < 1 || n_samples > (int64_t)1 << 24) return fail(h, RT_ERR_INVALID, "n_samples out of range");
    if ((s = rt_sync(h, -1)) != RT_OK) return s;
    if ((s = ensure_gen(h)) != RT_OK) return s;
    SurrogateState &S = *h->sg;
    const int64_t n_sets = (n_samples + K - 1) / K, rows = n_sets * K;
    if (S.ev_cap < rows) {
        cudaFree(S.ev_x); cudaFree(S.ev_t); cudaFree(S.ev_y); cudaFree(S.ev_err); cudaFree(S.ev_err_id);
        S.ev_x = nullptr; S.ev_t = nullptr; S.ev_y = nullptr; S.ev_err = nullptr; S.ev_err_id = nullptr;
        S.ev_cap = 0;
        if ((s = dalloc(h, &S.ev_x, (size_t)rows * kMlpIn)) != RT_OK) return s;
        if ((s = dalloc(h, &S.ev_t, (size_t)rows * 3)) != RT_OK) return s;
        if ((s = dalloc(h, &S.ev_y, (size_t)rows * 3)) != RT_OK) return s;
        if ((s = dalloc(h, &S.ev_err, (size_t)rows)) != RT_OK) return s;
        if ((s = dalloc(h, &S.ev_err_id, (size_t)rows)) != RT_OK) return s;
        S.ev_cap = rows;
    }
    if ((s = gen_set(h, seed, n_sets, S.ev_x, S.ev_t)) != RT_OK) return s;
    for (int64_t r0 = 0; r0 < rows; r0 += kMlpMaxRows) {
        const int n = (int)std::min<int64_t>(kMlpMaxRows, rows - r0);
        RT_CUDA(h, cudaMemcpyAsync(mlp_input(S.net), S.ev_x + (size_t)r0 * kMlpIn, (size_t)n * kMlpIn * 2,
                                   cudaMemcpyDeviceToDevice, h->s_main));
        RT_CUDA(h, mlp_forward_async(S.net, n, h->s_main));
        RT_CUDA(h, cudaMemcpyAsync(S.ev_y + (size_t)r0 * 3, mlp_output(S.net), (size_t)n * 12,
                                   cudaMemcpyDeviceToDevice, h->s_main));
    }
    const int threads = (int)(n_sets * h->n_groups);
    eval_err_kernel<<<(threads + 127) / 128, 128, 0, h->s_main>>>(S.ev_y, S.ev_t, K, (int)n_sets, h->solve_topo,
                                                                   h->n_groups, S.ev_err, S.ev_err_id);
    RT_CUDA(h, cudaGetLastError());
    std::string msg;
    if ((s = mlp_check(S.net, h->s_main, &msg)) != RT_OK) return fail(h, s, msg);
    if (errors) RT_CUDA(h, cudaMemcpy(errors, S.ev_err, (size_t)std::min(cap, rows) * 8, cudaMemcpyDeviceToHost));
    if (errors_identity)
        RT_CUDA(h, cudaMemcpy(errors_identity, S.ev_err_id, (size_t)std::min(cap, rows) * 8, cudaMemcpyDeviceToHost));
    if (n_out) *n_out = rows;
    return RT_OK;
}

rt_status rt_surrogate_save(rt_handle *h, const char *path)
{
    if (!h) return RT_ERR_INVALID;
    if (!path) return fail(h, RT_ERR_INVALID, "path is NULL");
    if (!h->sg || !h->sg->net) return fail(h, RT_ERR_STATE, "no surrogate network to save");
    rt_status s;
    if ((s = rt_sync(h, -1)) != RT_OK) return s;
    std::vector<uint8_t> blob;
    if ((s = mlp_serialize(h->sg->net, h->s_main, &blob)) != RT_OK) return fail(h, s, "reading the network back");
    FILE *f = fopen(path, "wb");
    if (!f) return fail(h, RT_ERR_INVALID, std::string("cannot open ") + path);
    const uint64_t nb = blob.size();
    const int64_t calls = h->sg->train_calls;
    bool ok = fwrite(&kFileMagic, 4, 1, f) == 1 && fwrite(&kFileVersion, 4, 1, f) == 1 &&
              fwrite(&calls, 8, 1, f) == 1 && fwrite(&nb, 8, 1, f) == 1 && fwrite(blob.data(), 1, nb, f) == nb;
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(h, RT_ERR_INVALID, std::string("cannot write ") + path);
    return RT_OK;
}

rt_status rt_surrogate_load(rt_handle *h, const char *path)
{
    if (!h) return RT_ERR_INVALID;
    if (!path) return fail(h, RT_ERR_INVALID, "path is NULL");
    rt_status s;
    if ((s = check_common(h)) != RT_OK) return s;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(h, RT_ERR_INVALID, std::string("cannot open ") + path);
    uint32_t magic = 0, ver = 0;
    int64_t calls = 0;
    uint64_t nb = 0;
    bool ok = fread(&magic, 4, 1, f) == 1 && fread(&ver, 4, 1, f) == 1 && fread(&calls, 8, 1, f) == 1 &&
              fread(&nb, 8, 1, f) == 1 && magic == kFileMagic && ver == kFileVersion && calls >= 0 &&
              nb < ((uint64_t)1 << 32);
    std::vector<uint8_t> blob;
    if (ok) {
        blob.resize(nb);
        ok = fread(blob.data(), 1, nb, f) == nb;
    }
    fclose(f);
    if (!ok) return fail(h, RT_ERR_INVALID, std::string("not a surrogate checkpoint: ") + path);
    if ((s = rt_sync(h, -1)) != RT_OK) return s;
    if ((s = ensure_state(h)) != RT_OK) return s;
    if (!h->sg->net && (s = rt_mlp_create(&h->sg->net, h->s_main)) != RT_OK) return fail(h, s, "rt_mlp_create");
    if ((s = mlp_deserialize(h->sg->net, h->s_main, blob.data(), blob.size())) != RT_OK)
        return fail(h, s, std::string("not a surrogate checkpoint of this network: ") + path);
    h->sg->train_calls = calls;
    return RT_OK;
}

rt_status rt_surrogate_get_params(rt_handle *h, float *params, size_t n)
{
    if (!h) return RT_ERR_INVALID;
    if (!h->sg || !h->sg->net) return fail(h, RT_ERR_STATE, "no surrogate network");
    rt_status s = rt_mlp_get_params(h->sg->net, params, n);
    if (s != RT_OK) return fail(h, s, rt_mlp_last_error(h->sg->net));
    return RT_OK;
}

rt_status rt_surrogate_set_tolerance(rt_handle *h, double tol)
{
    if (!h) return RT_ERR_INVALID;
    if (!(tol >= 0.0)) return fail(h, RT_ERR_INVALID, "the tolerance must be >= 0");
    if (h->capturing) return fail(h, RT_ERR_STATE, "not while a sequence is being captured");
    h->p.fallback_tol = tol;
    if (h->sg && h->sg->dev) {
        sg_set_tol_kernel<<<1, 1, 0, h->s_solve>>>(h->sg->dev, tol, 0);
        RT_CUDA(h, cudaGetLastError());
    }
    return RT_OK;
}

rt_status rt_surrogate_get_report(rt_handle *h, rt_surrogate_report *out, int32_t timeout_ms)
{
    if (!h || !out) return RT_ERR_INVALID;
    memset(out, 0, sizeof *out);
    out->tolerance = h->p.fallback_tol;
    if (!h->sg || !h->sg->dev) return RT_OK;
    rt_status s;
    if ((s = rt_sync(h, timeout_ms)) != RT_OK) return s;
    SgDev d;
    RT_CUDA(h, cudaMemcpy(&d, h->sg->dev, sizeof d, cudaMemcpyDeviceToHost));
    out->frame_sets = d.frames;
    out->predicted = d.predicted;
    out->plain = d.plain;
    out->judged = d.judged;
    out->judged_failed = d.judged_failed;
    out->fallback = d.fallback;
    out->last_error = d.last_err;
    out->max_error = d.max_err;
    out->tolerance = d.tol;
    return RT_OK;
}

}  // extern "C"
