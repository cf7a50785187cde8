// Pass A: the measured spectra of Sec. "White balance and exposure
// correction" -- per camera, band side (first / last S columns), vertical
// block and channel, the histogram of the band's converted RGB values, with
// (i) moving pixels removed: |Y_t - Y_{t-1}| > T on the band's luma
// (object removal, Fig. "thresholded difference"; the first frame set of a
// sequence has no previous frame and removes nothing), and (ii) saturated
// values 0 and 255 left out per channel.  Counts, sums and sums of squares
// are the histogram's moments, reduced from it at the end of every CTA.
// For the 3 x 3 cross-channel maps the kernel also sums the joint moments
// {n, R, G, B, RR, RG, RB, GG, GB, BB} over the pixels that are not moving
// and have no saturated channel (registers, then a warp reduction).
//
// One CTA per work item (camera, side, rows inside one block); a thread
// converts 16 band pixels of one row per iteration with one 16-byte load of
// Y (plus one of UV) and one of the previous frame's band luma, and writes
// this frame's band luma for the next frame set.
#include "rt_internal.cuh"
#include "pixel.cuh"

namespace rt {

namespace {

__device__ __forceinline__ uint4 ld16(const uint8_t *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

// 16 bytes at any address: one vector load when 16-byte aligned, else byte
// loads (the right band starts at W - S, unaligned when W is not a multiple
// of 16; only such ragged cameras take this path).
__device__ __forceinline__ uint4 ld16_any(const uint8_t *p)
{
    if (((uintptr_t)p & 15u) == 0) return ld16(p);
    uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i >> 2] |= (uint32_t)__ldg(p + i) << (8 * (i & 3));
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Two conversions' rounding step in one packed FP32x2 FMA: bits of
// (2^23 + 255 z) for z = z0, z1 (each already saturated to [0, 1]).
__device__ __forceinline__ void magic2(float z0, float z1, uint32_t &b0, uint32_t &b1)
{
    asm("{\n .reg .b64 a, k, m, r;\n"
        " mov.b64 a, {%2, %3};\n"
        " mov.b64 k, {%4, %4};\n"
        " mov.b64 m, {%5, %5};\n"
        " fma.rn.f32x2 r, a, k, m;\n"
        " mov.b64 {%0, %1}, r;\n}\n"
        : "=r"(b0), "=r"(b1) : "f"(z0), "f"(z1), "f"(255.0f), "f"(kMagic));
}

// Histogram slot of value bits vb (channel c) for a pixel that passed the
// motion test (ok): the bin, or the spare slot 768 for a moving pixel or a
// saturated value (0 or 255) -- no branch per pixel.
__device__ __forceinline__ uint32_t slot_of(uint32_t vb, int c, bool ok)
{
    const uint32_t v = vb - kMagicBits;
    return (ok && v - 1u < 254u) ? (uint32_t)c * 256u + v : 768u;
}

template <bool JOINT>
__global__ void __launch_bounds__(256) pass_a_kernel(const ArrayGeom g, const PassAArgs a, int Hmax)
{
    __shared__ uint32_t sh[3 * 256 + 1];   // + the spare slot
    const StripItem it = a.items[blockIdx.x];
    const CamGeom &cg = g.cam[it.cam];
    const ConvConsts &k = g.conv;
    for (int i = threadIdx.x; i < 769; i += blockDim.x) sh[i] = 0;
    {
        const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
        for (size_t i = tid; i < a.clear_u32_n; i += nt) a.clear_u32[i] = 0u;
        for (size_t i = tid; i < a.clear_u64_n; i += nt) a.clear_u64[i] = 0ull;
    }
    // surrogate mode: gate[0] = this frame set's band statistics are needed,
    // gate[1] = the previous frame set's band luma is there for the motion test
    if (a.gate && !a.gate[0]) return;
    const bool first = a.first || (a.gate && !a.gate[1]);
    __syncthreads();

    const int upr = a.S / kUnitCols;
    const int xb = it.side == 0 ? 0 : cg.W - a.S;
    const int nrows = it.row1 - it.row0;
    const size_t lbase = (size_t)it.cam * a.luma_cam_stride + (size_t)it.side * Hmax * a.S;
    // joint moments: n and sums in u32, products in u64 (per unit in u32)
    uint32_t jn = 0, js[3] = {0u, 0u, 0u};
    unsigned long long jp[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    for (int u = threadIdx.x; u < nrows * upr; u += blockDim.x) {
        const int y = it.row0 + u / upr;
        const int x0 = xb + (u % upr) * kUnitCols;
        uint32_t luma[4];
        uint32_t vb[16][3];
        if (cg.fmt == RT_NV12) {
            const uint4 Y = ld16_any(cg.y + (size_t)y * cg.y_pitch + x0);
            const uint4 UV = ld16_any(cg.uv + (size_t)(y >> 1) * cg.uv_pitch + x0);
            luma[0] = Y.x; luma[1] = Y.y; luma[2] = Y.z; luma[3] = Y.w;
            const uint32_t uvw[4] = {UV.x, UV.y, UV.z, UV.w};
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const float Uf = byte_f(uvw[p >> 1], (p & 1) * 2);
                const float Vf = byte_f(uvw[p >> 1], (p & 1) * 2 + 1);
                const float cz[3] = {fmaf(Vf, k.krv, k.c_r0), fmaf(Uf, k.kgu, fmaf(Vf, k.kgv, k.c_g0)),
                                     fmaf(Uf, k.kbu, k.c_b0)};
                const float Y0f = byte_f(luma[p >> 1], 2 * (p & 1)), Y1f = byte_f(luma[p >> 1], 2 * (p & 1) + 1);
                float z0[3], z1[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    z0[c] = __saturatef(fmaf(Y0f, k.ky, cz[c]));
                    z1[c] = __saturatef(fmaf(Y1f, k.ky, cz[c]));
                }
                magic2(z0[0], z0[1], vb[2 * p][0], vb[2 * p][1]);
                magic2(z1[0], z1[1], vb[2 * p + 1][0], vb[2 * p + 1][1]);
                magic2(z0[2], z1[2], vb[2 * p][2], vb[2 * p + 1][2]);
            }
        } else {
            const uint8_t *p = cg.y + (size_t)y * cg.y_pitch + 2 * x0;
            const uint4 A = ld16_any(p), Bv = ld16_any(p + 16);
            const uint32_t w[8] = {A.x, A.y, A.z, A.w, Bv.x, Bv.y, Bv.z, Bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) luma[i] = 0;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const uint32_t b = mono_bits((w[i >> 1] >> (16 * (i & 1))) & 0xFFFFu, cg.shift);
                vb[i][0] = vb[i][1] = vb[i][2] = b;
                luma[i >> 2] |= (b - kMagicBits) << (8 * (i & 3));
            }
        }
        const size_t lo = lbase + (size_t)y * a.S + (x0 - xb);
        *reinterpret_cast<uint4 *>(a.cur_luma + lo) = make_uint4(luma[0], luma[1], luma[2], luma[3]);
        uint32_t prev[4] = {luma[0], luma[1], luma[2], luma[3]};
        if (!first) {
            const uint4 P = ld16(a.prev_luma + lo);
            prev[0] = P.x; prev[1] = P.y; prev[2] = P.z; prev[3] = P.w;
        }
        const float T = (float)a.T;
        uint32_t up[6] = {0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float d = byte_f(luma[i >> 2], i & 3) - byte_f(prev[i >> 2], i & 3);   // exact
            const bool ok = fabsf(d) <= T;
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(&sh[slot_of(vb[i][c], c, ok)], 1u);
            if constexpr (JOINT) {
                const uint32_t r = vb[i][0] - kMagicBits, gr = vb[i][1] - kMagicBits, b = vb[i][2] - kMagicBits;
                const bool jv = ok && r - 1u < 254u && gr - 1u < 254u && b - 1u < 254u;
                const uint32_t m = jv ? 0xFFFFFFFFu : 0u;
                const uint32_t rm = r & m, gm = gr & m, bm = b & m;
                jn += jv ? 1u : 0u;
                js[0] += rm; js[1] += gm; js[2] += bm;
                up[0] += rm * rm; up[1] += rm * gm; up[2] += rm * bm;
                up[3] += gm * gm; up[4] += gm * bm; up[5] += bm * bm;
            }
        }
        if constexpr (JOINT) {
#pragma unroll
            for (int q = 0; q < 6; ++q) jp[q] += up[q];
        }
    }
    __syncthreads();
    const size_t slot = ((size_t)(it.cam * 2 + it.side) * g.B + it.block) * 3;
    for (int b = threadIdx.x; b < 768; b += blockDim.x) {
        const uint32_t cnt = sh[b];
        if (cnt) atomicAdd(a.hist + slot * 256 + b, cnt);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (JOINT) {
        unsigned long long v[10] = {jn, js[0], js[1], js[2], jp[0], jp[1], jp[2], jp[3], jp[4], jp[5]};
#pragma unroll
        for (int q = 0; q < 10; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0 && v[0]) {
            unsigned long long *dst = a.joint + ((size_t)(it.cam * 2 + it.side) * g.B + it.block) * 10;
#pragma unroll
            for (int q = 0; q < 10; ++q) atomicAdd(dst + q, v[q]);
        }
    }
    // moments of the three channel histograms, one warp per channel in turn
    for (int c = warp; c < 3; c += (int)(blockDim.x >> 5)) {
        unsigned long long n = 0, s = 0, ss = 0;
        for (int b = lane; b < 256; b += 32) {
            const unsigned long long cnt = sh[c * 256 + b];
            n += cnt;
            s += cnt * (unsigned long long)b;
            ss += cnt * (unsigned long long)(b * b);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n += __shfl_xor_sync(0xffffffffu, n, o);
            s += __shfl_xor_sync(0xffffffffu, s, o);
            ss += __shfl_xor_sync(0xffffffffu, ss, o);
        }
        if (lane == 0 && n) {
            atomicAdd(a.n + slot + c, (uint32_t)n);
            atomicAdd(a.sum + slot + c, s);
            atomicAdd(a.sumsq + slot + c, ss);
        }
    }
}

}  // namespace

cudaError_t launch_pass_a(const ArrayGeom &g, const PassAArgs &a, int threads, cudaStream_t s)
{
    if (a.n_items == 0) return cudaSuccess;
    const int Hmax = a.luma_cam_stride / (2 * a.S);
    if (a.joint) pass_a_kernel<true><<<a.n_items, threads, 0, s>>>(g, a, Hmax);
    else pass_a_kernel<false><<<a.n_items, threads, 0, s>>>(g, a, Hmax);
    return cudaGetLastError();
}

}  // namespace rt
