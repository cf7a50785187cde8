// Synthetic frame sets painted on the device, for the learned surrogate's
// training and evaluation arrays (no counterpart in the paper: its video is
// not available).  One thread per 2 x 2 pixel block of a camera computes the
// four pixels' RGB, encodes the block's four luma samples and its chroma pair
// (NV12: BT.709 limited range, chroma from the block's mean RGB) or four
// 12-bit mono samples.  The scene is deterministic in (parameters, key).
#include <cmath>

#include "rt_internal.cuh"

namespace rt {

namespace {

constexpr float kTwoPi = 6.283185307179586f;
constexpr float kKr = 0.2126f, kKb = 0.0722f, kKg = 1.0f - kKr - kKb;

// Counter-based random bits: the SplitMix64 output function (Steele, Lea,
// Flood, OOPSLA 2014) of a 64-bit counter.
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// A standard normal variate from the counter (Box-Muller on two 24-bit uniforms).
__device__ __forceinline__ float gauss(uint64_t ctr)
{
    const uint64_t r = mix64(ctr);
    const float u1 = ((float)(uint32_t)(r >> 40) + 0.5f) * (1.0f / 16777216.0f);
    const float u2 = (float)(uint32_t)((r >> 8) & 0xFFFFFFu) * (1.0f / 16777216.0f);
    return sqrtf(-2.0f * __logf(u1)) * __cosf(kTwoPi * u2);
}

// Radiance in [0, 255] of channel c at panorama column u and normalised row vn.
__device__ __forceinline__ void panorama(const float *p, float u, float vn, float out[3])
{
    const float horizon = 0.40f + 0.03f * __sinf(kTwoPi * u / (2900.0f + 900.0f * p[0]) + 6.28f * p[1]);
    const float t = fminf(vn / 0.4f, 1.0f);
    const float wave = __sinf(kTwoPi * u / (1700.0f + 600.0f * p[2]) + 6.28f * p[3]) *
                       __cosf(kTwoPi * vn * (3.0f + p[4]) + 6.28f * p[5]);
    const float slow = __sinf(kTwoPi * u / (5300.0f + 1500.0f * p[6]) + 6.28f * p[7]);
    const float sky[3] = {110.0f + 20.0f * p[8], 150.0f + 15.0f * p[9], 205.0f + 10.0f * p[10]};
    const float gnd[3] = {95.0f + 20.0f * p[11], 105.0f + 15.0f * p[12], 70.0f + 15.0f * p[13]};
    const bool is_sky = vn < horizon;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        out[c] = is_sky ? sky[c] + 35.0f * t + 12.0f * slow : gnd[c] + 25.0f * wave + 20.0f * (vn - 0.4f) + 10.0f * slow;
}

__global__ void __launch_bounds__(256) synth_kernel(const SynthArgs a)
{
    const uint32_t total = a.block_base[a.K];
    for (uint32_t bi = blockIdx.x * blockDim.x + threadIdx.x; bi < total; bi += gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < a.K && a.block_base[k + 1] <= bi) ++k;
        const uint32_t local = bi - a.block_base[k];
        const int bw = a.W[k] / 2;
        const int by = (int)(local / (uint32_t)bw), bx = (int)(local % (uint32_t)bw);
        float rgb[4][3];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int x = 2 * bx + (q & 1), y = 2 * by + (q >> 1);
            float r[3];
            panorama(a.ph, a.x0[k] + (float)x, ((float)y + 0.5f) / (float)a.H[k], r);
            const uint64_t ctr = ((((uint64_t)a.key_hi << 32) | a.key_lo) * 0x100000001B3ull) ^
                                 (((uint64_t)k << 58) | ((uint64_t)y << 32) | ((uint64_t)x << 4));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float v = r[c] * a.gain[k][c] + a.noise * gauss(ctr + (uint64_t)c);
                rgb[q][c] = fminf(fmaxf(rintf(v), 0.0f), 255.0f);
            }
        }
        if (a.fmt[k] == RT_NV12) {
            uint8_t *yp = a.y[k] + (size_t)(2 * by) * a.y_pitch[k] + 2 * bx;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float yn = (kKr * rgb[q][0] + kKg * rgb[q][1] + kKb * rgb[q][2]) / 255.0f;
                yp[(size_t)(q >> 1) * a.y_pitch[k] + (q & 1)] = (uint8_t)fminf(fmaxf(rintf(16.0f + 219.0f * yn), 0.0f), 255.0f);
            }
            float m[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) m[c] = (rgb[0][c] + rgb[1][c] + rgb[2][c] + rgb[3][c]) * (0.25f / 255.0f);
            const float ym = kKr * m[0] + kKg * m[1] + kKb * m[2];
            const float cb = 128.0f + 224.0f * (m[2] - ym) / (2.0f * (1.0f - kKb));
            const float cr = 128.0f + 224.0f * (m[0] - ym) / (2.0f * (1.0f - kKr));
            uint8_t *uvp = a.uv[k] + (size_t)by * a.uv_pitch[k] + 2 * bx;
            uvp[0] = (uint8_t)fminf(fmaxf(rintf(cb), 0.0f), 255.0f);
            uvp[1] = (uint8_t)fminf(fmaxf(rintf(cr), 0.0f), 255.0f);
        } else {
            const float top = (float)((1 << a.bits[k]) - 1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float lum = kKr * rgb[q][0] + kKg * rgb[q][1] + kKb * rgb[q][2];
                const float v = fminf(fmaxf(rintf(lum / 255.0f * top), 0.0f), top);
                uint16_t *row = reinterpret_cast<uint16_t *>(a.y[k] + (size_t)(2 * by + (q >> 1)) * a.y_pitch[k]);
                row[2 * bx + (q & 1)] = (uint16_t)v;
            }
        }
    }
}

}  // namespace

cudaError_t launch_synth(const SynthArgs &a, cudaStream_t s)
{
    const uint32_t total = a.block_base[a.K];
    const int grid = (int)std::min<uint32_t>((total + 255) / 256, 4096u);
    synth_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rt
