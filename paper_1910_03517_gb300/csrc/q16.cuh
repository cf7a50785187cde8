// Q16 quantisation of a smoothed map value (S4): round half away from zero
// of 65536 v, computed from the bits of v (no FP64 instruction; GB300's FP64
// pipe is narrow).  Valid for |v| < 2^15.
#pragma once
#include <cstdint>

namespace rt {

__device__ __forceinline__ int32_t q16_round(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 2047) - 1023;
    const unsigned long long mant = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = 36 - ex;                       // 65536 |v| = mant 2^-sh
    int32_t q;
    if (sh >= 64) q = 0;
    else if (sh <= 0) q = (int32_t)(mant << -sh);
    else q = (int32_t)((mant + (1ull << (sh - 1))) >> sh);
    return (b >> 63) ? -q : q;
}

}  // namespace rt
