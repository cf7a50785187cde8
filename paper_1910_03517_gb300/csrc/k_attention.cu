// Difference attention (Sec. "Attention mechanisms", the difference
// approach): the change map |Y_t - Y_{t-1}| > T of every camera's luma
// (NV12 Y, or the 8-bit value of a mono camera) is counted per square cell
// of side attn_window / 2; square windows of side attn_window, 2 x 2 cells,
// slide at stride attn_window / 2, and a window with at least min_on
// on-pixels becomes a proposal.
//
// attention_kernel: a thread takes 16 luma bytes of one row (one 16-byte
// load, and one of the previous frame set's copy of them), writes the copy
// for the next frame set, and adds its on-pixels to their cell (cells are
// multiples of 16 columns wide, so the 16 bytes never straddle two).
// proposals_kernel: one CTA walks the windows in order (camera, window row,
// window column) with a block-wide scan, so the list is deterministic.
#include "rt_internal.cuh"

namespace rt {

namespace {

__device__ __forceinline__ uint4 ld16(const uint8_t *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

// on-pixels among the 4 bytes of a, b: |a_i - b_i| > T, bytes selected by keep
__device__ __forceinline__ int on4(uint32_t a, uint32_t b, uint32_t t4, uint32_t keep)
{
    const uint32_t m = __vcmpgtu4(__vabsdiffu4(a, b), t4) & keep;   // 0xFF per byte that changed
    return __popc(m) >> 3;
}

__global__ void __launch_bounds__(256) attention_kernel(const ArrayGeom g, const AttnArgs a)
{
    const uint32_t total = a.unit_base[g.K];
    const uint32_t t4 = (uint32_t)a.T * 0x01010101u;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < g.K && a.unit_base[k + 1] <= u) ++k;
        const CamGeom &cg = g.cam[k];
        const uint32_t local = u - a.unit_base[k];
        const int cpr = (cg.W + 15) >> 4;
        const int y = (int)(local / (uint32_t)cpr), x0 = (int)(local - (uint32_t)y * cpr) * 16;
        uint32_t w[4];
        if (cg.fmt == RT_NV12) {
            const uint4 v = ld16(cg.y + (size_t)y * cg.y_pitch + x0);
            w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
        } else {
            // 16 samples of 16 bits -> 8-bit values min(255, v >> shift)
            const uint8_t *p = cg.y + (size_t)y * cg.y_pitch + 2 * x0;
            const int nv = min(16, cg.W - x0);
            const uint4 lo = ld16(p);
            const uint4 hi = nv > 8 ? ld16(p + 16) : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t s[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t word = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int q = 4 * i + j;
                    const uint32_t v = ((s[q >> 1] >> (16 * (q & 1))) & 0xFFFFu) >> cg.shift;
                    word |= (v > 255u ? 255u : v) << (8 * j);
                }
                w[i] = word;
            }
        }
        const size_t off = a.copy_off[k] + (size_t)y * a.copy_pitch[k] + x0;
        *reinterpret_cast<uint4 *>(a.cur + off) = make_uint4(w[0], w[1], w[2], w[3]);
        if (a.prev) {
            const uint4 pv = ld16(a.prev + off);
            const uint32_t pw[4] = {pv.x, pv.y, pv.z, pv.w};
            const int nv = min(16, cg.W - x0);     // bytes of this row inside the frame
            int cnt = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int b = min(max(nv - 4 * i, 0), 4);
                const uint32_t keep = b >= 4 ? 0xFFFFFFFFu : ((1u << (8 * b)) - 1u);
                cnt += on4(w[i], pw[i], t4, keep);
            }
            if (cnt) atomicAdd(a.cells + a.cell_off[k] + (y / a.cell) * a.ncx[k] + x0 / a.cell, (uint32_t)cnt);
        }
    }
}

constexpr int kPropThreads = 1024;

__global__ void __launch_bounds__(kPropThreads) proposals_kernel(const ArrayGeom g, const AttnArgs a)
{
    __shared__ int warp_hits[kPropThreads / 32];
    __shared__ int s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_base = 0;
    __syncthreads();
    const int total = (int)a.win_base[g.K];
    for (int start = 0; start < total; start += kPropThreads) {
        const int wi = start + tid;
        bool hit = false;
        rt_crop r{};
        if (wi < total) {
            int k = 0;
            while (k + 1 < g.K && (int)a.win_base[k + 1] <= wi) ++k;
            const CamGeom &cg = g.cam[k];
            const int local = wi - (int)a.win_base[k];
            const int nx = a.ncx[k], ny = a.ncy[k];
            const int nwx = max(nx - 1, 1);
            const int j = local / nwx, i = local - j * nwx;
            const uint32_t *c = a.cells + a.cell_off[k];
            uint32_t n = c[j * nx + i];
            if (i + 1 < nx) n += c[j * nx + i + 1];
            if (j + 1 < ny) n += c[(j + 1) * nx + i];
            if (i + 1 < nx && j + 1 < ny) n += c[(j + 1) * nx + i + 1];
            hit = n >= (uint32_t)a.min_on;
            r.cam = k;
            r.x0 = i * a.cell;
            r.y0 = j * a.cell;
            r.w = min(2 * a.cell, cg.W - r.x0);
            r.h = min(2 * a.cell, cg.H - r.y0);
        }
        // position of this window among the hits of this chunk, in order
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) warp_hits[warp] = __popc(bal);
        __syncthreads();
        int before = 0;
        for (int w2 = 0; w2 < warp; ++w2) before += warp_hits[w2];
        const int pos = s_base + before + __popc(bal & ((1u << lane) - 1u));
        if (hit && pos < a.max) a.out[pos] = r;
        __syncthreads();
        if (tid == kPropThreads - 1) s_base = pos + (hit ? 1 : 0);
        __syncthreads();
    }
    if (tid == 0) *a.count = min(s_base, a.max);
    // the cells are read only here: clear them for the next frame set
    for (uint32_t i = tid; i < a.cell_off[g.K]; i += kPropThreads) a.cells[i] = 0u;
}

}  // namespace

cudaError_t launch_attention(const ArrayGeom &g, const AttnArgs &a, int sm_count, cudaStream_t s)
{
    const uint32_t total = a.unit_base[g.K];
    if (total > 0) {
        const uint32_t blocks = (total + 255) / 256;
        const uint32_t cap = (uint32_t)sm_count * 8;
        attention_kernel<<<blocks < cap ? blocks : cap, 256, 0, s>>>(g, a);
    }
    proposals_kernel<<<1, kPropThreads, 0, s>>>(g, a);
    return cudaGetLastError();
}

}  // namespace rt
