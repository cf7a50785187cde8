// Detection post-processing and tracking (Sec. "AI-based video tracking").
//
// rt_nms: one CTA stages the boxes in shared memory, sorts them by (valid
// first, category, probability descending, index) with a bitonic sort; each
// category is then a contiguous run, walked greedily by one warp (runs of
// different categories in parallel): a box still alive is kept and the
// warp's lanes kill the later boxes of the run whose IoU with it exceeds
// the tolerance.  The device copies of
// the boxes and flags live in a static device array (calls are serialised
// by a host mutex): no allocation per call.
//
// rt_tracker: host code -- the assignment problems are a few dozen rows.
// The linear sum assignment is the Hungarian method with row and column
// potentials and shortest augmenting paths (Kuhn 1955; the O(R^2 C) form for
// R <= C rows), run per category.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "rt_internal.cuh"
#include "../../include/rt_track.h"

namespace rt {

namespace {

constexpr int kNmsMax = 4096;
constexpr int kNmsThreads = 1024;

__device__ rt_box g_nms_boxes[kNmsMax];
__device__ int32_t g_nms_keep[kNmsMax];
std::mutex g_nms_mutex;

__device__ __forceinline__ float box_iou(const rt_box &a, const rt_box &b)
{
    const float ix = fmaxf(0.0f, fminf(a.x1, b.x1) - fmaxf(a.x0, b.x0));
    const float iy = fmaxf(0.0f, fminf(a.y1, b.y1) - fmaxf(a.y0, b.y0));
    const float inter = ix * iy;
    const float uni = (a.x1 - a.x0) * (a.y1 - a.y0) + (b.x1 - b.x0) * (b.y1 - b.y0) - inter;
    return uni > 0.0f ? inter / uni : 0.0f;
}

__global__ void __launch_bounds__(kNmsThreads) nms_kernel(const rt_box *__restrict__ boxes, int n, float smin,
                                                          float thr, int32_t *__restrict__ keep)
{
    extern __shared__ unsigned long long key[];          // [n2], then the boxes [n]
    __shared__ uint8_t dead[kNmsMax];
    __shared__ int run_start[kNmsMax];
    __shared__ int n_runs;
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    rt_box *sbox = reinterpret_cast<rt_box *>(key + n2);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    if (tid == 0) n_runs = 0;
    for (int i = tid; i < n; i += blockDim.x) sbox[i] = boxes[i];
    __syncthreads();
    // key: bit 63 invalid, bits 48..62 category, bits 16..47 ~(probability bits), bits 0..15 index
    for (int i = tid; i < n2; i += blockDim.x) {
        unsigned long long k = ~0ull;
        if (i < n) {
            const rt_box b = sbox[i];
            const bool valid = b.score >= smin && b.score >= 0.0f;
            const uint32_t sb = __float_as_uint(fmaxf(b.score, 0.0f));
            k = ((unsigned long long)(valid ? 0u : 1u) << 63) | ((unsigned long long)(b.cls & 0x7FFF) << 48) |
                ((unsigned long long)(~sb) << 16) | (unsigned long long)i;
        }
        key[i] = k;
        if (i < n) keep[i] = 0;
    }
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < n2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long a = key[i], b = key[j];
                    if ((a > b) == up) { key[i] = b; key[j] = a; }
                }
            }
            __syncthreads();
        }
    // runs of one category among the valid boxes (contiguous after the sort)
    for (int i = tid; i < n; i += blockDim.x) {
        dead[i] = 0;
        const unsigned long long k = key[i];
        if (!(k >> 63) && (i == 0 || (key[i - 1] >> 48) != (k >> 48))) run_start[atomicAdd(&n_runs, 1)] = i;
    }
    __syncthreads();
    // one warp per category run: the greedy walk needs only warp barriers
    for (int r = warp; r < n_runs; r += nwarps) {
        const int s = run_start[r];
        const unsigned long long cat = key[s] >> 48;
        int e = s + 1;
        while (true) {   // end of the run: the first later key of another category (or invalid)
            const int q = e + lane;
            const bool other = q >= n || (key[q] >> 48) != cat;
            const unsigned m = __ballot_sync(0xffffffffu, other);
            if (m) { e += __ffs(m) - 1; break; }
            e += 32;
        }
        for (int p = s; p < e; ++p) {
            if (dead[p]) continue;                        // uniform across the warp
            const unsigned long long kp = key[p];
            const rt_box bp = sbox[kp & 0xFFFF];
            if (lane == 0) keep[kp & 0xFFFF] = 1;
            for (int q = p + 1 + lane; q < e; q += 32)
                if (!dead[q] && box_iou(bp, sbox[key[q] & 0xFFFF]) > thr) dead[q] = 1;
            __syncwarp();
        }
    }
}

double host_iou(const rt_box &a, const rt_box &b)
{
    const double ix = std::max(0.0, std::min((double)a.x1, (double)b.x1) - std::max((double)a.x0, (double)b.x0));
    const double iy = std::max(0.0, std::min((double)a.y1, (double)b.y1) - std::max((double)a.y0, (double)b.y0));
    const double inter = ix * iy;
    const double uni = ((double)a.x1 - a.x0) * ((double)a.y1 - a.y0) + ((double)b.x1 - b.x0) * ((double)b.y1 - b.y0) -
                       inter;
    return uni > 0.0 ? inter / uni : 0.0;
}

// Minimum-cost one-to-one assignment of the rows of an R x C cost matrix
// (R <= C) to columns: col_of_row[r].  Potentials u (rows), v (columns);
// each row is added by a shortest augmenting path over reduced costs.
void assign_rows(const std::vector<double> &cost, int R, int C, std::vector<int> &col_of_row)
{
    const double inf = 1e300;
    std::vector<double> u(R + 1, 0.0), v(C + 1, 0.0), minv(C + 1);
    std::vector<int> row_of(C + 1, 0), way(C + 1, 0);
    std::vector<char> used(C + 1);
    for (int r = 1; r <= R; ++r) {
        row_of[0] = r;
        int j0 = 0;
        std::fill(minv.begin(), minv.end(), inf);
        std::fill(used.begin(), used.end(), 0);
        do {
            used[j0] = 1;
            const int r0 = row_of[j0];
            double delta = inf;
            int j1 = 0;
            for (int j = 1; j <= C; ++j) {
                if (used[j]) continue;
                const double cur = cost[(size_t)(r0 - 1) * C + (j - 1)] - u[r0] - v[j];
                if (cur < minv[j]) { minv[j] = cur; way[j] = j0; }
                if (minv[j] < delta) { delta = minv[j]; j1 = j; }
            }
            for (int j = 0; j <= C; ++j) {
                if (used[j]) { u[row_of[j]] += delta; v[j] -= delta; }
                else minv[j] -= delta;
            }
            j0 = j1;
        } while (row_of[j0] != 0);
        do {
            const int j1 = way[j0];
            row_of[j0] = row_of[j1];
            j0 = j1;
        } while (j0 != 0);
    }
    col_of_row.assign(R, -1);
    for (int j = 1; j <= C; ++j)
        if (row_of[j] > 0) col_of_row[row_of[j] - 1] = j - 1;
}

}  // namespace

}  // namespace rt

struct rt_tracker {
    double a = 0.99, tol_iou = 0.05, tol_new = 0.001;
    struct Obj {
        int32_t id, cls;
        rt_box box;
        int64_t frame;
        int32_t history;
    };
    std::vector<Obj> objs;
};

extern "C" {

rt_status rt_nms(const rt_box *boxes, int32_t n, float score_min, float iou_max, int32_t *keep, void *cuda_stream)
{
    if (!boxes || !keep || n < 1 || n > rt::kNmsMax) return RT_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaPointerAttributes attr{};
    const bool on_device = cudaPointerGetAttributes(&attr, boxes) == cudaSuccess && attr.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    if (!on_device)
        for (int i = 0; i < n; ++i)
            if (boxes[i].cls < 0 || boxes[i].cls > 32767) return RT_ERR_INVALID;
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    const size_t smem = sizeof(unsigned long long) * n2 + sizeof(rt_box) * n;   // <= 32 KB + 96 KB
    std::lock_guard<std::mutex> lock(rt::g_nms_mutex);
    // the kernel's shared-memory limit, once per device
    static bool smem_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && (dev < 0 || dev >= 64)) e = cudaErrorInvalidDevice;
    if (e == cudaSuccess && !smem_set[dev]) {
        e = cudaFuncSetAttribute(rt::nms_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(unsigned long long) * rt::kNmsMax + sizeof(rt_box) * rt::kNmsMax));
        smem_set[dev] = e == cudaSuccess;
    }
    rt_box *d_boxes = nullptr;
    int32_t *d_keep = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&d_boxes, rt::g_nms_boxes);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&d_keep, rt::g_nms_keep);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_boxes, boxes, sizeof(rt_box) * n, cudaMemcpyDefault, st);
    if (e == cudaSuccess) {
        rt::nms_kernel<<<1, rt::kNmsThreads, smem, st>>>(d_boxes, n, score_min, iou_max, d_keep);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(keep, d_keep, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

rt_status rt_tracker_create(rt_tracker **out, double a, double tol_iou, double tol_new)
{
    if (!out) return RT_ERR_INVALID;
    *out = nullptr;
    if (!(a > 0.0 && a <= 1.0) || !(tol_iou >= 0.0 && tol_iou < 1.0) || !(tol_new >= 0.0 && tol_new < 1.0))
        return RT_ERR_INVALID;
    rt_tracker *t = new rt_tracker;
    t->a = a;
    t->tol_iou = tol_iou;
    t->tol_new = tol_new;
    *out = t;
    return RT_OK;
}

rt_status rt_tracker_update(rt_tracker *t, const rt_box *dets, int32_t n, int64_t frame, int32_t *object_of)
{
    if (!t || n < 0 || (n > 0 && (!dets || !object_of))) return RT_ERR_INVALID;
    for (int i = 0; i < n; ++i) object_of[i] = -1;
    std::vector<int32_t> classes;
    for (int i = 0; i < n; ++i) classes.push_back(dets[i].cls);
    std::sort(classes.begin(), classes.end());
    classes.erase(std::unique(classes.begin(), classes.end()), classes.end());
    for (int32_t cls : classes) {
        std::vector<int> di, oi;
        for (int i = 0; i < n; ++i)
            if (dets[i].cls == cls) di.push_back(i);
        for (size_t j = 0; j < t->objs.size(); ++j)
            if (t->objs[j].cls == cls) oi.push_back((int)j);
        const int R = (int)di.size(), C = (int)oi.size();
        std::vector<double> cost((size_t)R * C);
        for (int r = 0; r < R; ++r)
            for (int c = 0; c < C; ++c) {
                const auto &o = t->objs[oi[c]];
                cost[(size_t)r * C + c] = 1.0 - rt::host_iou(dets[di[r]], o.box) * std::pow(t->a, (double)(frame - o.frame));
            }
        std::vector<int> col_of(R, -1);
        if (R > 0 && C > 0) {
            if (R <= C) {
                rt::assign_rows(cost, R, C, col_of);
            } else {          // more detections than objects: assign the objects to detections
                std::vector<double> tr((size_t)C * R);
                for (int r = 0; r < R; ++r)
                    for (int c = 0; c < C; ++c) tr[(size_t)c * R + r] = cost[(size_t)r * C + c];
                std::vector<int> row_of_col;
                rt::assign_rows(tr, C, R, row_of_col);
                for (int c = 0; c < C; ++c)
                    if (row_of_col[c] >= 0) col_of[row_of_col[c]] = c;
            }
        }
        std::vector<std::pair<int, int>> joined;
        for (int r = 0; r < R; ++r) {
            const int i = di[r];
            if (col_of[r] >= 0 && 1.0 - cost[(size_t)r * C + col_of[r]] > t->tol_iou) {
                joined.emplace_back(i, oi[col_of[r]]);
                continue;
            }
            double best = 1.0;
            for (int c = 0; c < C; ++c) best = std::min(best, cost[(size_t)r * C + c]);
            if (C == 0 || 1.0 - best < t->tol_new) {
                rt_tracker::Obj o;
                o.id = (int32_t)t->objs.size();
                o.cls = cls;
                o.box = dets[i];
                o.frame = frame;
                o.history = 1;
                t->objs.push_back(o);
                object_of[i] = o.id;
            }
        }
        for (auto &jo : joined) {
            auto &o = t->objs[jo.second];
            o.box = dets[jo.first];
            o.frame = frame;
            o.history += 1;
            object_of[jo.first] = o.id;
        }
    }
    return RT_OK;
}

rt_status rt_tracker_objects(rt_tracker *t, int32_t *id, int32_t *cls, rt_box *last, int64_t *last_frame,
                             int32_t *history, int32_t cap, int32_t *n)
{
    if (!t || cap < 0) return RT_ERR_INVALID;
    const int cnt = (int)t->objs.size();
    if (n) *n = cnt;
    for (int i = 0; i < std::min(cnt, cap); ++i) {
        const auto &o = t->objs[i];
        if (id) id[i] = o.id;
        if (cls) cls[i] = o.cls;
        if (last) last[i] = o.box;
        if (last_frame) last_frame[i] = o.frame;
        if (history) history[i] = o.history;
    }
    return RT_OK;
}

void rt_tracker_destroy(rt_tracker *t) { delete t; }

}  // extern "C"
