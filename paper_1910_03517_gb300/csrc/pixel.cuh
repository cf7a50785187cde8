// Per-pixel arithmetic shared by the conversion kernels (pass A and pass B).
//
// Colour conversion (ITU-R BT.709 / BT.601 limited range, Q8 integers):
//   v_c = clamp(floor(N_c / 256), 0, 255),
//   N_R = 298 (Y-16) + c_rv (V-128) + 128
//   N_G = 298 (Y-16) - c_gu (U-128) - c_gv (V-128) + 128
//   N_B = 298 (Y-16) + c_bu (U-128) + 128
// evaluated without integer ALU work: with z = (N - 127.5) / 65280,
//   v = round_to_nearest(255 * saturate(z)),
// because (N - 127.5)/256 lies at least 0.5/256 away from every half
// integer, and the float error of z (a few ulp of numbers <= 2, < 1e-6)
// times 255 stays far below that margin.  255*z is rounded to an integer by
// adding 2^23 in one FMA; the float's bit pattern is then 0x4B000000 + v.
// Downstream code works on that bit pattern ("vbits") directly: an
// application t = a * v + c becomes t = a * vbits + (c - a * 0x4B000000)
// modulo 2^32, exact whenever the true t fits in 32 bits.
#pragma once
#include <cstdint>

#include "rt_internal.cuh"

namespace rt {

constexpr uint32_t kMagicBits = 0x4B000000u;   // bits of 2^23
constexpr float kMagic = 8388608.0f;           // 2^23

// Host only: the constants travel to the kernels in ArrayGeom::conv.
inline ConvConsts conv_consts(int matrix)
{
    // integer coefficients of the standard (round(256 k 255/219 or 255/224))
    const int cy = 298;
    const int crv = matrix == RT_BT601 ? 409 : 459;
    const int cgu = matrix == RT_BT601 ? 100 : 55;
    const int cgv = matrix == RT_BT601 ? 208 : 136;
    const int cbu = matrix == RT_BT601 ? 516 : 541;
    const double inv = 1.0 / 65280.0;
    ConvConsts k;
    k.ky = (float)(cy * inv);
    // constant part: -cy*16 + 128 - 127.5 - c*128 for each chroma term
    k.krv = (float)(crv * inv);
    k.c_r0 = (float)((-cy * 16.0 + 0.5 - crv * 128.0) * inv);
    k.kgu = (float)(-cgu * inv);
    k.kgv = (float)(-cgv * inv);
    k.c_g0 = (float)((-cy * 16.0 + 0.5 + cgu * 128.0 + cgv * 128.0) * inv);
    k.kbu = (float)(cbu * inv);
    k.c_b0 = (float)((-cy * 16.0 + 0.5 - cbu * 128.0) * inv);
    return k;
}

#ifdef __CUDACC__
// byte i (0..3) of w as a float, via the 2^23 bit trick (one PRMT + FADD)
__device__ __forceinline__ float byte_f(uint32_t w, int i)
{
    return __uint_as_float(__byte_perm(w, kMagicBits, 0x7440u | (uint32_t)i)) - kMagic;
}

// z -> bit pattern 0x4B000000 + round(255 * saturate(z))
__device__ __forceinline__ uint32_t zbits(float yf, float ky, float cz)
{
    float z = __saturatef(fmaf(yf, ky, cz));
    return __float_as_uint(fmaf(z, 255.0f, kMagic));
}

// 8-bit value of a mono sample: min(255, v >> shift), as vbits
__device__ __forceinline__ uint32_t mono_bits(uint32_t v16, int shift)
{
    uint32_t v = v16 >> shift;
    return (v > 255u ? 255u : v) + kMagicBits;
}

// Block index of row y for B blocks over H rows: the largest j with
// floor(j H / B) <= y, i.e. floor(((y + 1) B - 1) / H).
__device__ __forceinline__ int block_of_row(int y, int H, int B)
{
    return B == 1 ? 0 : (int)(((y + 1) * B - 1) / H);
}

// Insert byte 2 of t at byte position pos (0..3) of w.
__device__ __forceinline__ uint32_t put_byte2(uint32_t w, uint32_t t, int pos)
{
    uint32_t sel = 0x7654u;                      // keep w's bytes
    sel = (sel & ~(0xFu << (4 * pos))) | (2u << (4 * pos));
    return __byte_perm(t, w, sel) ;
}
#endif

}  // namespace rt
