// The scaled residual sigma = q + (a_1 + ... + a_M) / M - u of FP64 operands
// (M = 2d neighbours, section 2.2's unscaled stencil divided by 2d),
// evaluated without the FP64 pipe, which on GB300 issues 2 instructions per
// clock per SM: M sigma = M q + sum a_i - M u is summed exactly in 128-bit
// two's-complement fixed point on the integer pipe (every operand aligned to
// the largest exponent; an operand more than 113 binary places below it
// loses its lowest bits, a relative error below 2^-113 of the largest), then
// divided by M in the integers (a shift, and an exact division by 3) and
// rounded to a double-float: relative error about 2^-48 of sigma itself,
// where an FP64 evaluation errs by about 2^-53 of the operands.  Zero,
// subnormal, infinite or NaN operands, and
// results outside the float exponent range, report ok = false (the caller
// then evaluates in FP64).  Host-compilable (its test uses binary128).
#pragma once

#include <cstdint>

#include "df.cuh"

namespace gmg {
namespace fx {

using i128 = __int128;
using u128 = unsigned __int128;

__host__ __device__ __forceinline__ int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}
__host__ __device__ __forceinline__ int bitlen(u128 t) {
    const uint64_t hi = (uint64_t)(t >> 64), lo = (uint64_t)t;
    return hi ? 128 - clz64(hi) : 64 - clz64(lo);
}
__host__ __device__ __forceinline__ float u32_to_float(uint32_t x) {  // round to nearest
#ifdef __CUDA_ARCH__
    return __uint2float_rn(x);
#else
    return (float)x;
#endif
}
// floor(t / 3): t = hi 2^64 + lo; hi = 3 qh + rh; rh 2^64 + lo = 3 rh K +
// (rh + lo) with 2^64 = 3 K + 1 (a carry out of rh + lo adds another 3 K + 1)
__host__ __device__ __forceinline__ u128 div3(u128 t) {
    constexpr uint64_t K = 6148914691236517205ull;
    const uint64_t hi = (uint64_t)(t >> 64), lo = (uint64_t)t;
    const uint64_t qh = hi / 3, rh = hi - 3 * qh;
    const uint64_t s = lo + rh;
    const uint64_t ql = s < lo ? rh * K + K + (s + 1) / 3 : rh * K + s / 3;
    return ((u128)qh << 64) | ql;
}
// 2^k as a float for -126 <= k <= 127
__host__ __device__ __forceinline__ float pow2f(int k) {
    return cvt::bits_f((uint32_t)(k + 127) << 23);
}

template <int M>
__host__ __device__ __forceinline__ df32 sigma(const double (&a)[M], double q, double u, bool& ok) {
    constexpr int NV = M + 2;
    uint64_t b[NV];
#pragma unroll
    for (int i = 0; i < M; ++i) b[i] = cvt::d_bits(a[i]);
    b[M] = cvt::d_bits(q);
    b[M + 1] = cvt::d_bits(u);
    int emax = 0;
    bool special = false;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int e = (int)(b[i] >> 52) & 0x7ff;
        special |= e == 0x7ff || (e == 0 && (b[i] << 1) != 0);
        emax = e > emax ? e : emax;
    }
    ok = !special;
    if (special || emax == 0) return df32(0.f, 0.f);
    // operand i as a signed integer in units of 2^(emax - 1135): its 53-bit
    // significand shifted left by e - emax + 60 (<= 60; the sum of the
    // 3M+1 weighted operands stays below 2^120)
    i128 acc = 0;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int e = (int)(b[i] >> 52) & 0x7ff;
        const uint64_t m = (b[i] & 0xfffffffffffffull) | 0x10000000000000ull;
        const int sh = e - emax + 60;
        i128 v = 0;
        if (e != 0) {
            if (sh >= 0)
                v = (i128)((u128)m << sh);
            else if (sh > -53)
                v = (i128)(m >> (-sh));
        }
        if (b[i] >> 63) v = -v;
        acc += i < M ? v : i == M ? v * M : -(v * M);
    }
    // sigma = (M sigma) / M on the magnitude (truncating, below 2^-113 of the
    // largest operand), then rounded to a double-float
    const bool neg = acc < 0;
    u128 t = neg ? (u128)(-acc) : (u128)acc;
    t = M == 6 ? div3(t >> 1) : t >> 2;
    if (t == 0) return df32(0.f, 0.f);
    const int L = bitlen(t);
    const u128 tn = t << (128 - L);               // leading bit at 127
    const uint32_t hi_i = (uint32_t)(tn >> 104);  // 24 bits, leading bit set
    const uint32_t lo32 = (uint32_t)(tn >> 72);   // the next 32 bits
    // sigma ~= hi_i 2^(k+24) + lo32 2^(k-8), k = L - 48 + emax - 1135; the
    // low part rounded to 24 bits, the bits below it (2^-56 relative) dropped
    const int k = L - 48 + emax - 1135;
    if (k + 24 + 23 > 127 || k + 24 + 23 < -126) {  // the high part outside the normal range
        ok = false;
        return df32(0.f, 0.f);
    }
    const float hf = cvt::bits_f(((uint32_t)(k + 24 + 23 + 127) << 23) | (hi_i & 0x7fffffu));
    // the low part: exact scaling, then (below 2^-126) one rounding into the
    // subnormal range
    const float lf = k - 8 >= -126 ? u32_to_float(lo32) * pow2f(k - 8)
                                   : u32_to_float(lo32) * pow2f(k - 8 + 64) * pow2f(-64);
    const df32 r = dw::fast_two_sum(hf, lf);
    return neg ? df32(-r.hi, -r.lo) : r;
}

}  // namespace fx
}  // namespace gmg
