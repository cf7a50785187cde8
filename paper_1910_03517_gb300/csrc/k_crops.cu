// S6: attention windows -> fixed square detector inputs (Sec. "Detection":
// the detector takes square inputs of a fixed size, so windows are cut from
// the camera images and resized).  Bilinear, half-pixel centres, source
// coordinates clamped to the window, values / 255, FP16 planar NCHW.
//
// A thread computes two horizontally adjacent output pixels of one row (one
// row computation, half2 stores into each channel plane).  Per output pixel
// and source row the two taps (6 bytes of RGB24) come from two aligned
// 8-byte loads; the horizontal lerp is an exact integer dot product (Q15
// weights, dp2a), the vertical one FP32 with the 1/255 scale folded in.
#include <cuda_fp16.h>

#include "rt_internal.cuh"

namespace rt {

namespace {

// The 6 bytes at p (any alignment) as two words: lo = bytes 0..3, hi = 4..5.
// Reads the aligned 16 bytes around them (the output buffer is padded so
// that this stays inside the allocation).
__device__ __forceinline__ void load6(const uint8_t *p, uint32_t &lo, uint32_t &hi)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint2 *b = reinterpret_cast<const uint2 *>(a & ~(uintptr_t)7);
    const uint2 u = __ldg(b), v = __ldg(b + 1);
    const uint32_t off = (uint32_t)(a & 7);
    const uint32_t s = 8u * (off & 3u);
    const bool up = off >= 4;
    const uint32_t w0 = up ? u.y : u.x, w1 = up ? v.x : u.y, w2 = up ? v.y : v.x;
    lo = __funnelshift_r(w0, w1, s);
    hi = __funnelshift_r(w1, w2, s);
}

constexpr float kTwo23 = 8388608.0f;

// x (0 <= x < 2^23, an integer) as a float without a conversion instruction
__device__ __forceinline__ float int_f(int x) { return __int_as_float(0x4B000000 + x) - kTwo23; }

// floor of 0 <= f < 2^22 and the remainder, without a conversion instruction
__device__ __forceinline__ int floor_frac(float f, float &frac)
{
    const float fl = __fadd_rd(f, kTwo23);
    frac = f - __fsub_rn(fl, kTwo23);
    return __float_as_int(fl) - 0x4B000000;
}

// Horizontal lerp of one source row at left tap pixel p (right tap p + 1):
// the 6 bytes regrouped as (left, right) pairs per channel, then dot
// products with the Q15 weights wq = [(1 - wx) 2^15, wx 2^15] (exact
// integers, at most 255 x 2^15).
__device__ __forceinline__ void row_lerp(const uint8_t *p, uint32_t wq, uint32_t (&t)[3])
{
    uint32_t lo, hi;
    load6(p, lo, hi);                                  // [Lr Lg Lb Rr] [Rg Rb . .]
    const uint32_t rg = __byte_perm(lo, hi, 0x4130u);  // [Lr Rr Lg Rg]
    const uint32_t bb = __byte_perm(lo, hi, 0x5252u);  // [Lb Rb . .]
    t[0] = __dp2a_lo(wq, rg, 0u);
    t[1] = __dp2a_hi(wq, rg, 0u);
    t[2] = __dp2a_lo(wq, bb, 0u);
}

// Channel values of one output pixel at column x of the window, source rows
// r0 (weight s0 = (1 - wy) / (255 2^15)) and r1 (s1 = wy / (255 2^15)).  At
// the window's last column wx = 0, so the right tap (read past it) has no
// weight.
__device__ __forceinline__ void pixel(const uint8_t *r0, const uint8_t *r1, float sxs, int w, float x, float s0,
                                      float s1, float (&v)[3])
{
    const float fx = fminf(fmaxf(fmaf(x + 0.5f, sxs, -0.5f), 0.0f), (float)(w - 1));
    float wx;
    const int xlo = floor_frac(fx, wx);
    const uint32_t w1 = (uint32_t)__float_as_int(fmaf(wx, 32768.0f, kTwo23)) - 0x4B000000u;   // round(wx 2^15)
    const uint32_t wq = (32768u - w1) | (w1 << 16);
    uint32_t t[3], b[3];
    row_lerp(r0 + 3 * xlo, wq, t);
    row_lerp(r1 + 3 * xlo, wq, b);
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = fmaf(int_f((int)b[c]), s1, int_f((int)t[c]) * s0);
}

__global__ void __launch_bounds__(256) crops_kernel(const ArrayGeom g, const CropArgs a)
{
    const int n = blockIdx.y;
    if (a.count && n >= *a.count) return;
    const rt_crop cr = a.crops[n];
    const CamGeom &cg = g.cam[cr.cam];
    const int S = a.S, hp = (S + 1) >> 1;          // pixel pairs per output row
    const float sxs = (float)cr.w / (float)S, sys = (float)cr.h / (float)S;
    const size_t plane = (size_t)S * S;
    __half *out = a.out + (size_t)n * 3 * plane;
    const uint8_t *base = cg.rgb + (size_t)cr.y0 * cg.rgb_pitch + 3 * cr.x0;
    const bool even = (S & 1) == 0;
    const float kScale = 1.0f / (255.0f * 32768.0f);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < S * hp; p += gridDim.x * blockDim.x) {
        const int oy = p / hp, ox = 2 * (p - oy * hp);
        const float fy = fminf(fmaxf(fmaf(int_f(oy) + 0.5f, sys, -0.5f), 0.0f), (float)(cr.h - 1));
        float wy;
        const int ylo = floor_frac(fy, wy), yhi = min(ylo + 1, cr.h - 1);
        const float s1 = wy * kScale, s0 = kScale - s1;
        const uint8_t *r0 = base + (size_t)ylo * cg.rgb_pitch, *r1 = base + (size_t)yhi * cg.rgb_pitch;
        const float fox = int_f(ox);
        float v0[3], v1[3];
        pixel(r0, r1, sxs, cr.w, fox, s0, s1, v0);
        const size_t o = (size_t)oy * S + ox;
        if (even) {
            pixel(r0, r1, sxs, cr.w, fox + 1.0f, s0, s1, v1);
#pragma unroll
            for (int c = 0; c < 3; ++c)
                *reinterpret_cast<__half2 *>(out + c * plane + o) = __floats2half2_rn(v0[c], v1[c]);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) out[c * plane + o] = __float2half_rn(v0[c]);
            if (ox + 1 < S) {
                pixel(r0, r1, sxs, cr.w, fox + 1.0f, s0, s1, v1);
#pragma unroll
                for (int c = 0; c < 3; ++c) out[c * plane + o + 1] = __float2half_rn(v1[c]);
            }
        }
    }
}

// Column-stationary variant: a thread owns one output pixel pair column
// (blockDim = pairs per row) and walks the rows blockIdx.x, +gridDim.x, ...,
// two rows a round so that both rows' tap loads are in flight together;
// the columns' taps, weights and load alignment are set up once.  The
// arithmetic is the row-major kernel's, operation for operation.
struct ColTap {
    int aoff;          // byte offset of the aligned 4-byte word holding the left tap
    uint32_t sh;       // funnel shift of the 6 tap bytes within the words
    uint32_t wq;       // Q15 weights
};

__device__ __forceinline__ ColTap col_tap(float sxs, int w, float x, uintptr_t base_mod4)
{
    const float fx = fminf(fmaxf(fmaf(x + 0.5f, sxs, -0.5f), 0.0f), (float)(w - 1));
    float wx;
    const int xlo = floor_frac(fx, wx);
    const uint32_t w1 = (uint32_t)__float_as_int(fmaf(wx, 32768.0f, kTwo23)) - 0x4B000000u;   // round(wx 2^15)
    ColTap t;
    t.wq = (32768u - w1) | (w1 << 16);
    const int b = 3 * xlo;
    const int mis = (int)((base_mod4 + (uintptr_t)b) & 3u);
    t.aoff = b - mis;
    t.sh = 8u * (uint32_t)mis;
    return t;
}

// Horizontal lerp of one source row with a column's taps: three aligned
// 4-byte loads hold the 6 tap bytes.
__device__ __forceinline__ void row_lerp_col(const uint8_t *row, const ColTap &c, uint32_t (&t)[3])
{
    const uint32_t *q = reinterpret_cast<const uint32_t *>(row + c.aoff);
    const uint32_t w0 = __ldg(q), w1 = __ldg(q + 1), w2 = __ldg(q + 2);
    const uint32_t lo = __funnelshift_r(w0, w1, c.sh), hi = __funnelshift_r(w1, w2, c.sh);
    const uint32_t rg = __byte_perm(lo, hi, 0x4130u);  // [Lr Rr Lg Rg]
    const uint32_t bb = __byte_perm(lo, hi, 0x5252u);  // [Lb Rb . .]
    t[0] = __dp2a_lo(c.wq, rg, 0u);
    t[1] = __dp2a_hi(c.wq, rg, 0u);
    t[2] = __dp2a_lo(c.wq, bb, 0u);
}

__global__ void __launch_bounds__(1024) crops_cols_kernel(const ArrayGeom g, const CropArgs a)
{
    const int n = blockIdx.y;
    if (a.count && n >= *a.count) return;
    const rt_crop cr = a.crops[n];
    const CamGeom &cg = g.cam[cr.cam];
    const int S = a.S;
    const float sxs = (float)cr.w / (float)S, sys = (float)cr.h / (float)S;
    const size_t plane = (size_t)S * S;
    __half *out = a.out + (size_t)n * 3 * plane;
    const uint8_t *base = cg.rgb + (size_t)cr.y0 * cg.rgb_pitch + 3 * cr.x0;
    // rows start on 16 bytes: a row's byte alignment is the window base's
    const uintptr_t bmod = reinterpret_cast<uintptr_t>(base) & 3u;
    const float kScale = 1.0f / (255.0f * 32768.0f);
    const int ox = 2 * (int)threadIdx.x;
    const bool two = ox + 1 < S;
    const float fox = int_f(ox);
    const ColTap c0 = col_tap(sxs, cr.w, fox, bmod);
    const ColTap c1 = col_tap(sxs, cr.w, fox + 1.0f, bmod);
    // two rows per round: both rows' tap loads are in flight together
    const int step = (int)gridDim.x;
    for (int oy0 = blockIdx.x; oy0 < S; oy0 += 2 * step) {
        const bool has_b = oy0 + step < S;
        float s0[2], s1[2];
        const uint8_t *ra[2], *rb[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int oy = h == 0 || !has_b ? oy0 : oy0 + step;
            const float fy = fminf(fmaxf(fmaf(int_f(oy) + 0.5f, sys, -0.5f), 0.0f), (float)(cr.h - 1));
            float wy;
            const int ylo = floor_frac(fy, wy), yhi = min(ylo + 1, cr.h - 1);
            s1[h] = wy * kScale;
            s0[h] = kScale - s1[h];
            ra[h] = base + (size_t)ylo * cg.rgb_pitch;
            rb[h] = base + (size_t)yhi * cg.rgb_pitch;
        }
        uint32_t t[2][2][3], b[2][2][3];   // [row][pixel][channel]
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            row_lerp_col(ra[h], c0, t[h][0]);
            row_lerp_col(rb[h], c0, b[h][0]);
            if (two) {
                row_lerp_col(ra[h], c1, t[h][1]);
                row_lerp_col(rb[h], c1, b[h][1]);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !has_b) break;
            const int oy = oy0 + h * step;
            float v0[3], v1[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) v0[c] = fmaf(int_f((int)b[h][0][c]), s1[h], int_f((int)t[h][0][c]) * s0[h]);
            const size_t o = (size_t)oy * S + ox;
            if (two) {
#pragma unroll
                for (int c = 0; c < 3; ++c) v1[c] = fmaf(int_f((int)b[h][1][c]), s1[h], int_f((int)t[h][1][c]) * s0[h]);
                if ((S & 1) == 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        *reinterpret_cast<__half2 *>(out + c * plane + o) = __floats2half2_rn(v0[c], v1[c]);
                    continue;
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) out[c * plane + o + 1] = __float2half_rn(v1[c]);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) out[c * plane + o] = __float2half_rn(v0[c]);
        }
    }
}

}  // namespace

cudaError_t launch_crops(const ArrayGeom &g, const CropArgs &a, int threads, int max_grid, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    const int hp = (a.S + 1) / 2;
    if (hp <= 1024) {
        // column-stationary: one CTA of hp threads per group of rows
        dim3 grid(a.S < max_grid ? a.S : max_grid, a.n);
        crops_cols_kernel<<<grid, hp, 0, s>>>(g, a);
        return cudaGetLastError();
    }
    const int pairs = a.S * hp;
    const int per = (pairs + threads - 1) / threads;
    dim3 grid(per < max_grid ? per : max_grid, a.n);
    crops_kernel<<<grid, threads, 0, s>>>(g, a);
    return cudaGetLastError();
}

}  // namespace rt
