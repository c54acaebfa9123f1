// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2 -- about 48 significant bits in the
// storage (8 bytes) of one double, computed on the FP32 pipe, which on GB300
// issues 64 times as many instructions per clock as the FP64 pipe.
//
// Building blocks (u = 2^-24, the FP32 unit roundoff):
//   TwoSum (Knuth; 6 adds): s + e = a + b exactly.
//   Fast2Sum (Dekker 1971; 3 adds, |a| >= |b|): s + e = a + b exactly.
//   Double-word + double-word: the accurate double-word addition of Joldes,
//     Muller & Popescu, "Tight and rigorous error bounds for basic building
//     blocks of double-word arithmetic", ACM TOMS 44(2), 2017 (two TwoSums,
//     two Fast2Sums; relative error a few u^2), 20 adds.
//   Double-word x double-word: the fma-based product of the same paper (the
//     exact high product by one fma, the cross terms by two more; relative
//     error a few u^2), 2 multiplies, 3 fmas, 4 adds.
// Every operation is an explicit round-to-nearest intrinsic (namespace rn)
// so that the compiler cannot contract an add with a preceding multiply into
// an fma, which would break the exactness of TwoSum / Fast2Sum.  The header
// also compiles as host C++ (for its tests).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cmath>
#include <cstring>

namespace gmg {
// ---------------------------------------------------------- conversions
// float <-> double conversions by the IEEE 754 binary32 / binary64 bit
// layouts, on the integer pipe: on GB300 the hardware conversions issue on
// the FP64 pipe, which the FP64 residual kernels already saturate.  Both are
// exact re-implementations of the casts (checked against them on the host,
// tests/test_df_host.py); rare operands take the cast itself.
namespace cvt {
__host__ __device__ __forceinline__ uint32_t f_bits(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return b;
#endif
}
__host__ __device__ __forceinline__ float bits_f(uint32_t b) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    std::memcpy(&f, &b, 4);
    return f;
#endif
}
__host__ __device__ __forceinline__ uint64_t d_bits(double d) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t b;
    std::memcpy(&b, &d, 8);
    return b;
#endif
}
__host__ __device__ __forceinline__ double bits_d(uint64_t b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double d;
    std::memcpy(&d, &b, 8);
    return d;
#endif
}

// (double)f, exactly: a normal binary32 number's exponent field is rebiased
// by 1023 - 127 and its 23 fraction bits move up by 29; zero, subnormal,
// infinite and NaN operands take the cast.
__host__ __device__ __forceinline__ double widen(float f) {
    const uint32_t b = f_bits(f);
    const uint32_t a = b & 0x7fffffffu;
    if (a - 0x00800000u >= 0x7f000000u) return (double)f;  // not a normal number
    return bits_d((((uint64_t)a) << 29) + ((uint64_t)(1023 - 127) << 52) +
                  ((uint64_t)(b >> 31) << 63));
}
__host__ __device__ __forceinline__ float int_to_float(int32_t r) {
#ifdef __CUDA_ARCH__
    return __int2float_rn(r);
#else
    return (float)r;
#endif
}

// hi = (float)x and lo = (float)(x - hi), exactly: hi is x's 24 leading
// significand bits rounded to nearest even (the carry of a round-up runs
// into the exponent field, as the format intends); x - hi is the signed
// remainder of the 29 lower bits in units of x's last place, which converts
// to float with one rounding and is scaled by a power of two.  Exponents
// outside [2^-74, 2^126) (where the scaled remainder could be subnormal, or
// hi overflow) and zero, subnormal, infinite and NaN operands take the casts.
struct split_t {
    float hi, lo;
};
__host__ __device__ __forceinline__ split_t split(double x) {
    const uint64_t b = d_bits(x);
    const uint32_t ex = (uint32_t)(b >> 52) & 0x7ffu;
    if (ex - 949u > 1149u - 949u) {
        const float h = (float)x;
        return split_t{h, (float)(x - (double)h)};
    }
    const uint32_t rem = (uint32_t)b & 0x1fffffffu;  // the 29 bits below hi
    uint32_t hb = ((uint32_t)(b >> 63) << 31) | ((ex - (1023 - 127)) << 23) |
                  ((uint32_t)(b >> 29) & 0x7fffffu);
    const uint32_t up = rem > 0x10000000u || (rem == 0x10000000u && (hb & 1u)) ? 1u : 0u;
    hb += up;
    int32_t r = (int32_t)rem - (up ? 0x20000000 : 0);
    if (b >> 63) r = -r;
    const float scale = bits_f((ex - (1075 - 127)) << 23);  // 2^(ex - 1075)
    return split_t{bits_f(hb), int_to_float(r) * scale};
}
}  // namespace cvt

// Round-to-nearest float operations that the compiler may not fuse or
// reorder: the device intrinsics, or on the host (tests only, built with
// -ffp-contract=off) the plain operators.
namespace rn {
__host__ __device__ __forceinline__ float add(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
__host__ __device__ __forceinline__ float sub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
__host__ __device__ __forceinline__ float mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
__host__ __device__ __forceinline__ float fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}
}  // namespace rn

// The type and its operators live in a namespace of their own: argument-
// dependent lookup finds them for df32 operands, while unqualified calls
// such as fma(double, double, double) elsewhere in gmg still reach the
// standard overloads.
namespace dw {

struct __align__(8) df32 {
    float hi, lo;
    df32() = default;
    __host__ __device__ constexpr df32(float h, float l) : hi(h), lo(l) {}
    // nearest split of a double: hi = RN(x), lo = RN(x - hi) (x - hi is
    // exact in double precision); by integer operations (cvt::split)
    __host__ __device__ explicit df32(double x) {
        const cvt::split_t t = cvt::split(x);
        hi = t.hi;
        lo = t.lo;
    }
    __host__ __device__ explicit df32(int x) : df32((double)x) {}
    __host__ __device__ explicit operator double() const {
        return cvt::widen(hi) + cvt::widen(lo);
    }
};

__host__ __device__ __forceinline__ df32 two_sum(float a, float b) {
    const float s = rn::add(a, b);
    const float bb = rn::sub(s, a);
    const float e = rn::add(rn::sub(a, rn::sub(s, bb)), rn::sub(b, bb));
    return df32(s, e);
}

__host__ __device__ __forceinline__ df32 fast_two_sum(float a, float b) {
    const float s = rn::add(a, b);
    return df32(s, rn::sub(b, rn::sub(s, a)));
}

__host__ __device__ __forceinline__ df32 operator+(df32 x, df32 y) {
    const df32 s = two_sum(x.hi, y.hi);
    const df32 t = two_sum(x.lo, y.lo);
    const df32 v = fast_two_sum(s.hi, rn::add(s.lo, t.hi));
    return fast_two_sum(v.hi, rn::add(t.lo, v.lo));
}

__host__ __device__ __forceinline__ df32 operator-(df32 x) { return df32(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ df32 operator-(df32 x, df32 y) { return x + (-y); }
__host__ __device__ __forceinline__ df32& operator+=(df32& x, df32 y) { return x = x + y; }

__host__ __device__ __forceinline__ df32 operator*(df32 x, df32 y) {
    const float ch = rn::mul(x.hi, y.hi);
    const float cl1 = rn::fma(x.hi, y.hi, -ch);
    const float tl0 = rn::mul(x.lo, y.lo);
    const float tl1 = rn::fma(x.hi, y.lo, tl0);
    const float cl2 = rn::fma(x.lo, y.hi, tl1);
    const float cl3 = rn::add(cl1, cl2);
    return fast_two_sum(ch, cl3);
}

// a * b + c as one product and one sum (not fused: two roundings to double-
// word precision)
__host__ __device__ __forceinline__ df32 fma(df32 a, df32 b, df32 c) { return a * b + c; }

// x + y when both may be of any size and sign: TwoSum of the high parts, the
// low parts and the error added in FP32, TwoSum to renormalise (14 adds;
// absolute error a few u^2 (|x| + |y|), no precondition on the operands).
__host__ __device__ __forceinline__ df32 add_fast(df32 x, df32 y) {
    const df32 s = two_sum(x.hi, y.hi);
    return two_sum(s.hi, rn::add(s.lo, rn::add(x.lo, y.lo)));
}

// Sums of the 2d neighbours in the pair tree ((a + b) + (c + d)) + (e + f)
// (2D: (a + b) + (c + d)), compensated: the high parts added by TwoSum, each
// rounding error and every low part accumulated in FP32, TwoSum at the end.
// 46 (30) adds instead of 100 (60) for the same tree of double-word sums;
// absolute error about 11 u^2 times the sum of magnitudes.
__host__ __device__ __forceinline__ df32 sum4(df32 a, df32 b, df32 c, df32 d) {
    const df32 ab = two_sum(a.hi, b.hi);
    const df32 cd = two_sum(c.hi, d.hi);
    const df32 t = two_sum(ab.hi, cd.hi);
    float e = rn::add(ab.lo, rn::add(a.lo, b.lo));
    e = rn::add(e, rn::add(cd.lo, rn::add(c.lo, d.lo)));
    e = rn::add(e, t.lo);
    return two_sum(t.hi, e);
}
__host__ __device__ __forceinline__ df32 sum6(df32 a, df32 b, df32 c, df32 d, df32 e_, df32 f) {
    const df32 ab = two_sum(a.hi, b.hi);
    const df32 cd = two_sum(c.hi, d.hi);
    const df32 ef = two_sum(e_.hi, f.hi);
    const df32 t = two_sum(ab.hi, cd.hi);
    const df32 v = two_sum(t.hi, ef.hi);
    float e = rn::add(ab.lo, rn::add(a.lo, b.lo));
    e = rn::add(e, rn::add(cd.lo, rn::add(c.lo, d.lo)));
    e = rn::add(e, rn::add(ef.lo, rn::add(e_.lo, f.lo)));
    e = rn::add(e, t.lo);
    e = rn::add(e, v.lo);
    return two_sum(v.hi, e);
}

// 1/6 as the triple-float c0 + c1 + c2 (about 72 bits): a double-float
// constant alone is off by 9e-16 relative, a bias that the coarse solve
// would amplify wherever a residual is formed.
constexpr float kSixth0 = 0x1.555556p-3f;     // fl32(1/6)
constexpr float kSixth1 = -0x1.555556p-28f;   // fl32(1/6 - c0)
constexpr float kSixth2 = 0x1.555556p-53f;    // fl32(1/6 - c0 - c1)
// s / 6 (relative error about 2 u^2, unbiased)
__host__ __device__ __forceinline__ df32 sixth(df32 s) {
    const float p = rn::mul(kSixth0, s.hi);
    const float pe = rn::fma(kSixth0, s.hi, -p);
    const float t = rn::fma(kSixth0, s.lo, rn::fma(kSixth1, s.hi, rn::mul(kSixth2, s.hi)));
    return fast_two_sum(p, rn::add(pe, t));
}
// s / 4, exact
__host__ __device__ __forceinline__ df32 quarter(df32 s) {
    return df32(rn::mul(0.25f, s.hi), rn::mul(0.25f, s.lo));
}

// ------------------------------------------------------------ triple-float
// A Gauss-Seidel value formed to about 70 bits, for the one place where a
// double-float value enters an FP64 iterate and its own rounding would stay
// behind as residual: q + s / (2d) with s the sum of 2d double-float values
// and q double-float, returned as t0 + t1 + t2 (t2 ~ u^2 |t0|).  Error-free
// transformations (TwoSum, the fma product error) at the first two levels,
// plain FP32 sums at the third; relative error about 2^-65.
struct tf32 {
    float t0, t1, t2;
};

// s = x[0] + ... + x[m-1] (m <= 6 double-float terms) as a triple-float.
template <int M>
__host__ __device__ __forceinline__ tf32 sum_tf(const df32 (&x)[M]) {
    // level 0: the high parts, the TwoSum errors go one level down
    float s = x[0].hi, err0[M - 1];
#pragma unroll
    for (int i = 1; i < M; ++i) {
        const df32 t = two_sum(s, x[i].hi);
        s = t.hi;
        err0[i - 1] = t.lo;
    }
    // level 1: the low parts and the level-0 errors
    float t = x[0].lo, r = 0.f;
#pragma unroll
    for (int i = 1; i < M; ++i) {
        const df32 a = two_sum(t, x[i].lo);
        t = a.hi;
        r = rn::add(r, a.lo);
    }
#pragma unroll
    for (int i = 0; i < M - 1; ++i) {
        const df32 a = two_sum(t, err0[i]);
        t = a.hi;
        r = rn::add(r, a.lo);
    }
    return tf32{s, t, r};
}

// q + s * c with c = c0 + c1 + c2 (a triple-float constant; c1 = c2 = 0 for
// a power of two), as a triple-float.
__host__ __device__ __forceinline__ tf32 fma_tf(tf32 s, float c0, float c1, float c2, df32 q) {
    // level 0 product and its exact error
    const float p0 = rn::mul(c0, s.t0);
    const float pe0 = rn::fma(c0, s.t0, -p0);
    // level 1 terms: c0 t1, c1 t0 (each with its exact error), pe0
    const float a = rn::mul(c0, s.t1);
    const float ae = rn::fma(c0, s.t1, -a);
    const float b = rn::mul(c1, s.t0);
    const float be = rn::fma(c1, s.t0, -b);
    const df32 m1 = two_sum(pe0, a);
    const df32 m2 = two_sum(m1.hi, b);
    // level 2 terms
    float w = rn::add(rn::add(ae, be), rn::add(m1.lo, m2.lo));
    w = rn::add(w, rn::fma(c0, s.t2, rn::fma(c1, s.t1, rn::mul(c2, s.t0))));
    // + q
    const df32 z0 = two_sum(p0, q.hi);
    const df32 z1 = two_sum(m2.hi, q.lo);
    const df32 z2 = two_sum(z1.hi, z0.lo);
    return tf32{z0.hi, z2.hi, rn::add(w, rn::add(z1.lo, z2.lo))};
}

// the triple-float value in FP64 (one rounding at the end)
__host__ __device__ __forceinline__ double tf_to_double(tf32 v) {
    return (cvt::widen(v.t0) + cvt::widen(v.t1)) + cvt::widen(v.t2);
}

}  // namespace dw
using dw::df32;
using dw::kSixth0;
using dw::kSixth1;
using dw::kSixth2;
using dw::tf32;
}  // namespace gmg
