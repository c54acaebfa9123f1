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
// Every operation is an explicit round-to-nearest intrinsic so that the
// compiler cannot contract an add with a preceding multiply into an fma,
// which would break the exactness of TwoSum / Fast2Sum.
#pragma once

#include <cuda_runtime.h>

namespace gmg {
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
    // exact in double precision)
    __host__ __device__ explicit df32(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit df32(int x) : df32((double)x) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df32 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df32(s, e);
}

__device__ __forceinline__ df32 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df32(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df32 operator+(df32 x, df32 y) {
    const df32 s = two_sum(x.hi, y.hi);
    const df32 t = two_sum(x.lo, y.lo);
    const df32 v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ df32 operator-(df32 x) { return df32(-x.hi, -x.lo); }
__device__ __forceinline__ df32 operator-(df32 x, df32 y) { return x + (-y); }
__device__ __forceinline__ df32& operator+=(df32& x, df32 y) { return x = x + y; }

__device__ __forceinline__ df32 operator*(df32 x, df32 y) {
    const float ch = __fmul_rn(x.hi, y.hi);
    const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
    const float tl0 = __fmul_rn(x.lo, y.lo);
    const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    const float cl3 = __fadd_rn(cl1, cl2);
    return fast_two_sum(ch, cl3);
}

// a * b + c as one product and one sum (not fused: two roundings to double-
// word precision)
__device__ __forceinline__ df32 fma(df32 a, df32 b, df32 c) { return a * b + c; }

// x + y when both may be of any size and sign: TwoSum of the high parts, the
// low parts and the error added in FP32, TwoSum to renormalise (14 adds;
// absolute error a few u^2 (|x| + |y|), no precondition on the operands).
__device__ __forceinline__ df32 add_fast(df32 x, df32 y) {
    const df32 s = two_sum(x.hi, y.hi);
    return two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

// Sums of the 2d neighbours in the pair tree ((a + b) + (c + d)) + (e + f)
// (2D: (a + b) + (c + d)), compensated: the high parts added by TwoSum, each
// rounding error and every low part accumulated in FP32, TwoSum at the end.
// 46 (30) adds instead of 100 (60) for the same tree of double-word sums;
// absolute error about 11 u^2 times the sum of magnitudes.
__device__ __forceinline__ df32 sum4(df32 a, df32 b, df32 c, df32 d) {
    const df32 ab = two_sum(a.hi, b.hi);
    const df32 cd = two_sum(c.hi, d.hi);
    const df32 t = two_sum(ab.hi, cd.hi);
    float e = __fadd_rn(ab.lo, __fadd_rn(a.lo, b.lo));
    e = __fadd_rn(e, __fadd_rn(cd.lo, __fadd_rn(c.lo, d.lo)));
    e = __fadd_rn(e, t.lo);
    return two_sum(t.hi, e);
}
__device__ __forceinline__ df32 sum6(df32 a, df32 b, df32 c, df32 d, df32 e_, df32 f) {
    const df32 ab = two_sum(a.hi, b.hi);
    const df32 cd = two_sum(c.hi, d.hi);
    const df32 ef = two_sum(e_.hi, f.hi);
    const df32 t = two_sum(ab.hi, cd.hi);
    const df32 v = two_sum(t.hi, ef.hi);
    float e = __fadd_rn(ab.lo, __fadd_rn(a.lo, b.lo));
    e = __fadd_rn(e, __fadd_rn(cd.lo, __fadd_rn(c.lo, d.lo)));
    e = __fadd_rn(e, __fadd_rn(ef.lo, __fadd_rn(e_.lo, f.lo)));
    e = __fadd_rn(e, t.lo);
    e = __fadd_rn(e, v.lo);
    return two_sum(v.hi, e);
}

// 1/6 as the triple-float c0 + c1 + c2 (about 72 bits): a double-float
// constant alone is off by 9e-16 relative, a bias that the coarse solve
// would amplify wherever a residual is formed.
constexpr float kSixth0 = 0x1.555556p-3f;     // fl32(1/6)
constexpr float kSixth1 = -0x1.555556p-28f;   // fl32(1/6 - c0)
constexpr float kSixth2 = 0x1.555556p-53f;    // fl32(1/6 - c0 - c1)
// s / 6 (relative error about 2 u^2, unbiased)
__device__ __forceinline__ df32 sixth(df32 s) {
    const float p = __fmul_rn(kSixth0, s.hi);
    const float pe = __fmaf_rn(kSixth0, s.hi, -p);
    const float t = __fmaf_rn(kSixth0, s.lo, __fmaf_rn(kSixth1, s.hi, __fmul_rn(kSixth2, s.hi)));
    return fast_two_sum(p, __fadd_rn(pe, t));
}
// s / 4, exact
__device__ __forceinline__ df32 quarter(df32 s) {
    return df32(__fmul_rn(0.25f, s.hi), __fmul_rn(0.25f, s.lo));
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
__device__ __forceinline__ tf32 sum_tf(const df32 (&x)[M]) {
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
        r = __fadd_rn(r, a.lo);
    }
#pragma unroll
    for (int i = 0; i < M - 1; ++i) {
        const df32 a = two_sum(t, err0[i]);
        t = a.hi;
        r = __fadd_rn(r, a.lo);
    }
    return tf32{s, t, r};
}

// q + s * c with c = c0 + c1 + c2 (a triple-float constant; c1 = c2 = 0 for
// a power of two), as a triple-float.
__device__ __forceinline__ tf32 fma_tf(tf32 s, float c0, float c1, float c2, df32 q) {
    // level 0 product and its exact error
    const float p0 = __fmul_rn(c0, s.t0);
    const float pe0 = __fmaf_rn(c0, s.t0, -p0);
    // level 1 terms: c0 t1, c1 t0 (each with its exact error), pe0
    const float a = __fmul_rn(c0, s.t1);
    const float ae = __fmaf_rn(c0, s.t1, -a);
    const float b = __fmul_rn(c1, s.t0);
    const float be = __fmaf_rn(c1, s.t0, -b);
    const df32 m1 = two_sum(pe0, a);
    const df32 m2 = two_sum(m1.hi, b);
    // level 2 terms
    float w = __fadd_rn(__fadd_rn(ae, be), __fadd_rn(m1.lo, m2.lo));
    w = __fadd_rn(w, __fmaf_rn(c0, s.t2, __fmaf_rn(c1, s.t1, __fmul_rn(c2, s.t0))));
    // + q
    const df32 z0 = two_sum(p0, q.hi);
    const df32 z1 = two_sum(m2.hi, q.lo);
    const df32 z2 = two_sum(z1.hi, z0.lo);
    return tf32{z0.hi, z2.hi, __fadd_rn(w, __fadd_rn(z1.lo, z2.lo))};
}

// the triple-float value in FP64 (one rounding at the end)
__device__ __forceinline__ double tf_to_double(tf32 v) {
    return ((double)v.t0 + (double)v.t1) + (double)v.t2;
}

}  // namespace dw
using dw::df32;
using dw::kSixth0;
using dw::kSixth1;
using dw::kSixth2;
using dw::tf32;
}  // namespace gmg
