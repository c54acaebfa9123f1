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

}  // namespace dw
using dw::df32;
}  // namespace gmg
