// gadi_bits.cuh -- FP64 -> FP32 and FP32 -> FP64 conversions done with
// integer operations on the IEEE-754 bit patterns.
//
// On this GPU FP64 arithmetic and FP32 <-> FP64 conversions issue at about
// two per clock per SM, a small fraction of the integer and FP32 rates. The
// demotion of the residual (Alg. 1 step 2: r^ = fl_r(2^-e r)) is evaluated
// at every neighbour a stencil row reads; it starts from a round-to-odd FP32
// copy of r written once per row by the residual pass, and needs only FP32
// work after that. The update (Alg. 1 step 4) promotes the inner solution
// to FP64 exactly. Both give the same bits as the FP64 multiply and IEEE
// round-to-nearest-even conversion they replace.
//
// Plain C++ on the host as well (no CUDA intrinsics outside __CUDA_ARCH__),
// so the routines can be checked on the CPU against a library conversion.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define GADI_HD __host__ __device__ __forceinline__
#else
#define GADI_HD inline
#endif

namespace gadi {

GADI_HD uint64_t bits_of(double x)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

GADI_HD double double_of(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    std::memcpy(&x, &b, sizeof x);
    return x;
#endif
}

GADI_HD uint32_t bits_of(float x)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(x);
#else
    uint32_t b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

GADI_HD int clz32(uint32_t v)
{
#if defined(__CUDA_ARCH__)
    return __clz((int)v);
#else
    return v ? __builtin_clz(v) : 32;
#endif
}

// FP32 bits of x rounded to odd: the significand is truncated to 24 bits
// and its last bit set when anything nonzero was dropped. Rounding this
// value to FP16 (round to nearest even, also after an exact scaling by a
// power of two) gives the same result as rounding x directly, because 24 >=
// 11 + 2 (round-to-odd double rounding). Magnitudes below the FP32 normal
// range give a signed zero (x = 0) or a signed smallest subnormal; at or
// above 2^128 a signed infinity; NaN stays NaN.
GADI_HD uint32_t float_bits_round_odd(double x)
{
    const uint64_t b = bits_of(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int ex = (int)((b >> 52) & 0x7ffu);
    const uint64_t mant = b & 0xFFFFFFFFFFFFFull;
    if (ex == 0x7ff) return sign | 0x7f800000u | (mant ? 0x400000u : 0u);
    const int E = ex - 1023;
    if (E > 127) return sign | 0x7f800000u;
    if (E < -126) return sign | ((ex | mant) ? 1u : 0u);
    const uint32_t m = (uint32_t)(mant >> 29);
    const uint32_t sticky = (mant & ((1ull << 29) - 1)) ? 1u : 0u;
    return sign | ((uint32_t)(E + 127) << 23) | m | sticky;
}

// The FP64 value of an FP32 value (exact)
GADI_HD double double_of_float(float f)
{
    const uint32_t b = bits_of(f);
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    const uint32_t E = (b >> 23) & 0xffu;
    uint32_t m = b & 0x7fffffu;
    if (E == 255) return double_of(sign | 0x7ff0000000000000ull | ((uint64_t)m << 29));
    if (E == 0) {
        if (m == 0) return double_of(sign);
        const int lz = clz32(m) - 8;               // leading bit to position 23
        m = (m << lz) & 0x7fffffu;
        return double_of(sign | ((uint64_t)(1023 - 126 - lz) << 52) | ((uint64_t)m << 29));
    }
    return double_of(sign | ((uint64_t)(E + 896) << 52) | ((uint64_t)m << 29));
}

}  // namespace gadi
