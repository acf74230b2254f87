// Conversions between IEEE-754 binary64 and binary32 as integer operations
// on the bit patterns.  GB300 issues the hardware conversion instructions to
// its FP64 unit, where each costs the slot of an FP64 fused multiply-add
// (about 1.6 lanes per SM and clock, measured); these use the integer pipe.
//
// Written from the two formats:
//   binary64: sign 1 | exponent 11, bias 1023 | fraction 52
//   binary32: sign 1 | exponent 8,  bias 127  | fraction 23
// A binary32 exponent e corresponds to the binary64 exponent e + 896.
//
// Behaviour, and where it differs from the hardware conversions:
//   hx_f64_to_f32: round to nearest, ties to even; overflow gives a signed
//     infinity, NaN a quiet NaN.  Magnitudes below 2^-126 (the smallest
//     normal binary32) give a zero of the same sign, so no subnormal is made.
//   hx_f32_to_f64: exact; a subnormal binary32 gives a zero of the same sign.
// Host and device share the code; a host test checks it against the C casts.
#pragma once
#include <stdint.h>
#include <string.h>
#if !defined(__cplusplus)
#include <stdbool.h>
#endif

#if defined(__CUDACC__)
#define HX_FPC_HD __host__ __device__ __forceinline__
#else
#define HX_FPC_HD static inline
#endif

HX_FPC_HD uint64_t hx_bits_f64(double x) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    return u;
#endif
}

HX_FPC_HD double hx_f64_from_bits(uint64_t u) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, sizeof x);
    return x;
#endif
}

HX_FPC_HD uint32_t hx_bits_f32(float x) {
#if defined(__CUDA_ARCH__)
    return (uint32_t)__float_as_uint(x);
#else
    uint32_t u;
    memcpy(&u, &x, sizeof u);
    return u;
#endif
}

HX_FPC_HD float hx_f32_from_bits(uint32_t u) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float x;
    memcpy(&x, &u, sizeof x);
    return x;
#endif
}

// binary64 -> binary32, round to nearest with ties to even.
HX_FPC_HD float hx_f64_to_f32(double x) {
    const uint64_t u = hx_bits_f64(x);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;            // binary32 biased exponent
    const uint32_t frac = ((hi & 0xfffffu) << 3) | (lo >> 29);  // the 23 kept fraction bits
    const uint32_t rest = lo & 0x1fffffffu;                     // the 29 dropped ones; half is bit 28
    // Exponent and fraction side by side: a carry out of the fraction
    // increments the exponent, and from the largest finite value it gives
    // the infinity pattern.
    uint32_t b = ((uint32_t)e << 23) + frac;
    b += (uint32_t)((rest > 0x10000000u) | ((rest == 0x10000000u) & frac));
    const bool is_nan = ((hi & 0x7ff00000u) == 0x7ff00000u) && (((hi & 0xfffffu) | lo) != 0u);
    b = e <= 0 ? 0u : (e >= 255 ? (is_nan ? 0x7fc00000u : 0x7f800000u) : b);
    return hx_f32_from_bits(sign | b);
}

// binary32 -> binary64, exact.
HX_FPC_HD double hx_f32_to_f64(float f) {
    const uint32_t u = hx_bits_f32(f);
    const uint32_t sign = u & 0x80000000u, e = (u >> 23) & 0xffu, frac = u & 0x7fffffu;
    const uint32_t e64 = e == 0u ? 0u : (e == 255u ? 0x7ffu : e + 896u);
    const uint32_t hi = sign | (e64 << 20) | (e == 0u ? 0u : frac >> 3);
    const uint32_t lo = e == 0u ? 0u : frac << 29;
    return hx_f64_from_bits(((uint64_t)hi << 32) | lo);
}
