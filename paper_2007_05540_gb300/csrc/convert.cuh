// Conversions between IEEE-754 binary64 and binary32 done on the integer pipes.  On GB300
// the hardware double <-> float conversion runs at the (reduced) FP64 rate, about one
// result per SM and clock, which makes it the bottleneck of kernels that convert every
// operand element; these bit-level versions run several times faster.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace heff {

// Rows of the split-precision operand arrays (hi and lo halves of every element): the row
// is cut into K blocks of KB elements (64 bytes of one half), and each K block of hi values
// is followed by the same K block of lo values, so a row of ld columns takes 2 ld elements
// and one 128-byte row of a TMA box carries both halves of a K block.  Column c of a row
// sits at element c + KB floor(c / KB); its lo half is KB elements further on.
template <int KB>
__host__ __device__ __forceinline__ int64_t split_col(int64_t c) {
    return c + (c & ~(int64_t)(KB - 1));
}

// binary64 -> binary32, round to nearest even.  Results below the normal binary32 range
// (|x| < 2^-126) become a zero of the same sign (no subnormal results); values above it
// round to infinity; infinities stay infinite and NaNs stay NaN.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32);
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);                  // binary64 biased exponent
    const uint64_t m = b & 0x000fffffffffffffull;             // 52 fraction bits
    if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x00400000u : 0u));
    const int ef = e - 1023 + 127;                             // binary32 biased exponent
    if (ef <= 0) return __uint_as_float(sign);
    if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
    uint32_t bits = ((uint32_t)ef << 23) | (uint32_t)(m >> 29);   // keep the top 23 fraction bits
    const uint32_t rem = (uint32_t)(m & 0x1fffffffu);             // the 29 bits dropped
    bits += (rem > 0x10000000u) || (rem == 0x10000000u && (bits & 1u));   // a carry may round up the exponent
    return __uint_as_float(sign | (bits < 0x7f800000u ? bits : 0x7f800000u));
}

// binary32 -> binary64 (exact for every normal value and zero; binary32 subnormals, which
// the producers above never create, become zero).
__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    const uint32_t e = (u >> 23) & 0xffu;
    const uint64_t m = (uint64_t)(u & 0x007fffffu) << 29;
    if (e == 0) return __longlong_as_double((long long)sign);
    const uint64_t ed = e == 0xffu ? 0x7ffull : (uint64_t)e - 127 + 1023;
    return __longlong_as_double((long long)(sign | (ed << 52) | m));
}

}  // namespace heff
