// Level kernels of the V-cycle (Algorithm 1), templated on the storage type
// T (double, float, __nv_bfloat16, df32) with arithmetic in C = double for
// double storage, double-float for df32 storage (df.cuh) and float
// otherwise.
//
// Scaled variables: with the unscaled 5/7-point operator A' (section 2.2)
// and b = h^2 f, each level stores q = b / (2d); the Gauss-Seidel value of a
// node is q + c * (sum of its 2d neighbours), c = 1/(2d), and the scaled
// residual is sigma = q + c * sum - u = (b - A'u) / (2d).  Full weighting of
// b_{l+1} = 4 FW(b - A'u) then reads q_{l+1} = 4 FW(sigma): every transfer
// weight is a power of two.
//
// Instruction counts per node (what bounds the FP64 instantiation on GB300,
// whose FP64 pipe issues 2 instructions/clock/SM):
//   red-black half sweep   5 add + 1 fma per updated node (FP64 3D diagonal
//                          walkers: 4 + 1/kWalk add + 1 fma)
//   residual               5 add + 1 fma + 1 add
//   restriction            red nodes only after a black half sweep (the black
//                          residual is zero in exact arithmetic): 13 ops per
//                          coarse node in 3D
//   prolongation+correct   per coarse cell, pair/quad/octet sums shared by
//                          its 2^d fine nodes: 2.5 ops per fine node in 3D
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "df.cuh"
#include "gmg_internal.cuh"

namespace gmg {
namespace lk {

// x / d for 32-bit unsigned x and a fixed divisor d >= 1 by one multiply-high
// and shifts: the round-up method of Granlund & Montgomery, "Division by
// invariant integers using multiplication" (PLDI 1994, Fig. 4.1), with
// l = ceil(log2 d) and mag = floor(2^32 (2^l - d) / d) + 1 (< 2^32).
struct FastDiv {
    uint32_t d, mag;
    int l;
};
inline FastDiv fastdiv_make(uint32_t d) {
    FastDiv f{d, 0u, 0};
    while ((1ull << f.l) < d) ++f.l;
    f.mag = (uint32_t)((((1ull << f.l) - d) << 32) / d + 1);
    return f;
}
__device__ inline uint32_t fastdiv(uint32_t x, const FastDiv& f) {
    if (f.l == 0) return x;  // d = 1
    const uint32_t t = __umulhi(x, f.mag);
    return (t + ((x - t) >> 1)) >> (f.l - 1);
}

template <typename T>
struct Num;
template <>
struct Num<double> {
    using C = double;
    __device__ static double ld(double v) { return v; }
    __device__ static double st(double v) { return v; }
};
template <>
struct Num<float> {
    using C = float;
    __device__ static float ld(float v) { return v; }
    __device__ static float st(float v) { return v; }
};
template <>
struct Num<__nv_bfloat16> {
    using C = float;
    __device__ static float ld(__nv_bfloat16 v) {  // exact: BF16 = FP32's upper half
        return __uint_as_float((uint32_t)__bfloat16_as_ushort(v) << 16);
    }
    __device__ static __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};
template <>
struct Num<df32> {
    using C = df32;
    __device__ static df32 ld(df32 v) { return v; }
    __device__ static df32 st(df32 v) { return v; }
};

// The Gauss-Seidel value q + c * s, c = 1/(2d), of a node whose
// neighbours sum to s.  In 3D c = 1/6 is not a
// binary number: fma with c = fl(1/6) = (1/6)(1 - 5.6e-17) biases every
// product by the same relative amount.  In a residual of the full iterate u
// (level 0) that bias is a smooth field of size 5.6e-17 |u|, which the coarse
// solve amplifies by 1/lambda_min -- 3e-12 |u| at n = 512, above the 1e-12
// per-cycle agreement with a correctly rounded evaluation.  EXACT (FP64 3D
// only) carries 1/6 as the double-double kSixthHi + kSixthLo: one more fma,
// an unbiased result.  The black half sweep right before a red-only residual
// uses the same expression, so the black residual stays exactly zero.
constexpr double kSixthHi = 0x1.5555555555555p-3;   // fl(1/6)
constexpr double kSixthLo = 0x1.5555555555555p-57;  // fl(1/6 - kSixthHi) = fl(2^-55 / 3)
// Double-float (C = df32): always unbiased -- s / 6 with a triple-float 1/6
// (df.cuh, sixth), s / 4 exactly -- then q added (add_fast); c is not used.
template <int DIM, bool EXACT, typename C>
__device__ inline C gs_value(C c, C s, C q) {
    if constexpr (std::is_same<C, df32>::value)
        return add_fast(DIM == 3 ? sixth(s) : quarter(s), q);
    else if constexpr (EXACT && DIM == 3 && std::is_same<C, double>::value)
        return fma(c, s, fma(kSixthLo, s, q));
    else
        return fma(c, s, q);
}

__host__ __device__ inline int64_t sy_of(int n) { return (int64_t)n + 1; }
template <int DIM>
__host__ __device__ inline int64_t sz_of(int n) {
    return DIM == 3 ? ((int64_t)n + 1) * (n + 1) : 0;
}

struct RowLaunch {
    dim3 grid, block;
};

// x threads along a row (32..128), rows j over blockIdx.x, planes k over
// blockIdx.y (3D).
inline RowLaunch row_launch(int d, int n, int xcount) {
    int bx = 32;
    while (bx < xcount && bx < 128) bx *= 2;
    const int by = 256 / bx;
    RowLaunch L;
    L.block = dim3(bx, by, 1);
    L.grid = dim3((unsigned)((n - 1 + by - 1) / by), d == 3 ? (unsigned)(n - 1) : 1u, 1);
    return L;
}

// Sum of the 2d axis neighbours as a pair tree: 2D (x- + x+) + (y- + y+),
// 3D ((x- + x+) + (y- + z-)) + (y+ + z+) -- the same 2d-1 adds as a chain,
// dependency depth 3.  In 3D the (y+ + z+) pair of node (i, j, k) is the
// (y- + z-) pair of node (i, j+1, k+1), a node of the same colour, which
// lets k_rb_half3_walk form each pair once for two nodes.  xm, xp: offsets
// of the x-1 and x+1 neighbours (-1, +1 in the dense layout).
template <int DIM, typename T>
__device__ inline typename Num<T>::C nbr_sum_x(const T* u, int64_t p, int64_t xm, int64_t xp,
                                               int64_t sy, int64_t sz) {
    using N = Num<T>;
    if constexpr (std::is_same<T, df32>::value) {  // same tree, compensated (df.cuh)
        if (DIM == 3)
            return sum6(u[p + xm], u[p + xp], u[p - sy], u[p - sz], u[p + sy], u[p + sz]);
        return sum4(u[p + xm], u[p + xp], u[p - sy], u[p + sy]);
    }
    const auto sx = N::ld(u[p + xm]) + N::ld(u[p + xp]);
    if (DIM == 3) {
        const auto lo = N::ld(u[p - sy]) + N::ld(u[p - sz]);
        const auto hi = N::ld(u[p + sy]) + N::ld(u[p + sz]);
        return (sx + lo) + hi;
    }
    return sx + (N::ld(u[p - sy]) + N::ld(u[p + sy]));
}
template <int DIM, typename T>
__device__ inline typename Num<T>::C nbr_sum(const T* u, int64_t p, int64_t sy, int64_t sz) {
    return nbr_sum_x<DIM>(u, p, -1, 1, sy, sz);
}

// Offset of node x = i within its row, and of its x-1 / x+1 neighbours
// relative to it, for the dense (SPLIT = false) and colour-split layouts.
template <bool SPLIT>
__host__ __device__ inline int64_t xo(const Lay& L, int i) {
    return SPLIT ? ((i & 1) ? L.he + (i >> 1) : (i >> 1)) : i;
}
// The same for a layout known only at run time (he = 0: dense): the coarse
// level of a transfer may be dense under a colour-split fine level.
__host__ __device__ inline int64_t xo_any(const Lay& L, int i) {
    return L.he ? xo<true>(L, i) : i;
}
template <bool SPLIT>
__device__ inline void xnb(const Lay& L, int i, int64_t& xm, int64_t& xp) {
    if (!SPLIT) {
        xm = -1;
        xp = 1;
    } else if (i & 1) {
        xm = -L.he;
        xp = 1 - L.he;
    } else {
        xm = L.he - 1;
        xp = L.he;
    }
}

// One colour of red-black Gauss-Seidel: nodes with (i+j+k) % 2 == color.
template <int DIM, bool SPLIT, typename T, bool EXACT = false>
__global__ void __launch_bounds__(256) k_rb_half(T* __restrict__ u, const T* __restrict__ q, Lay L,
                                                 int color) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = DIM == 3 ? C(1.0 / 6.0) : C(0.25);
    const int n = L.n;
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    if (j >= n) return;
    const int64_t row = k * L.sz + j * L.sy;
    const int i0 = 1 + ((1 + j + k + color) & 1);
    int64_t xm, xp;
    xnb<SPLIT>(L, i0, xm, xp);  // every node of the loop has i0's parity
    for (int i = i0 + 2 * threadIdx.x; i < n; i += 2 * blockDim.x) {
        const int64_t p = row + xo<SPLIT>(L, i);
        u[p] = N::st(
            gs_value<DIM, EXACT>(c, nbr_sum_x<DIM>(u, p, xm, xp, L.sy, L.sz), N::ld(q[p])));
    }
}

// V consecutive elements of a colour-split half row (16-byte aligned: V = 4
// for FP32, 8 for BF16) as V values of the compute type.
__device__ inline void ldv(const float* p, float* v) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}
// BF16 is the upper half of an FP32 bit pattern: each value is widened
// exactly by one shift or mask on the integer pipe.
__device__ inline void ldv(const __nv_bfloat16* p, float* v) {
    const uint4 a = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        v[2 * h] = __uint_as_float(w[h] << 16);
        v[2 * h + 1] = __uint_as_float(w[h] & 0xffff0000u);
    }
}
__device__ inline void stv(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ inline void stv(__nv_bfloat16* p, const float* v) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h)
        *reinterpret_cast<__nv_bfloat162*>(&w[h]) = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}
template <typename T>
__host__ __device__ constexpr int vec_of() {
    return 16 / (int)sizeof(T);
}

// One colour of red-black Gauss-Seidel on a colour-split level (FP32 / BF16
// storage), V = 16 bytes of nodes per thread: work item w = (row (j, k),
// group g) holds the nodes of the colour at half-row positions V g .. V g +
// V-1, whose q, y/z neighbours (same half of the neighbouring rows) and
// result are one 16-byte vector each, and whose x neighbours are V+1
// consecutive entries of the row's other half.  Same operands in the same
// order as nbr_sum_x: the results equal k_rb_half's bit for bit.  G = groups
// per half row.
// RES: the scaled residual of the colour's nodes (sigma = value - u) into
// res instead of the new values into u (the red-only residual after a black half
// sweep; the same expression as k_residual).
template <int DIM, typename T, bool RES = false>
__global__ void __launch_bounds__(256, sizeof(T) == 2 ? 8 : 1) k_rb_half_vec(T* __restrict__ u, const T* __restrict__ q,
                                                     Lay L, int color, FastDiv fG, FastDiv fm,
                                                     uint32_t items, T* __restrict__ res = nullptr) {
    using N = Num<T>;
    constexpr int V = vec_of<T>();
    const float c = DIM == 3 ? 1.f / 6.f : 0.25f;
    const int n = L.n;
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= items) return;
    // work item w = (row r, group g), row r = (j-1) + (k-1)(n-1): divisions
    // by multiply-high (the counts stay below 2^32)
    const uint32_t r = fastdiv(w, fG);
    const int g = (int)(w - r * fG.d);
    const uint32_t kk = DIM == 3 ? fastdiv(r, fm) : 0;
    const int j = (int)(r - kk * fm.d) + 1, k = DIM == 3 ? (int)kk + 1 : 0;
    const int par = (color + j + k) & 1;  // x parity of the colour in this row
    const int x0 = 2 * V * g + par;       // x of the group's first node
    if (x0 > n - 1) return;
    const int64_t row = k * L.sz + j * L.sy;
    const int64_t base = row + (par ? L.he : 0) + V * g;
    // other half: x-1 / x+1 of node t are entries t-1+par / t+par of it
    const int64_t ob = row + (par ? 0 : L.he) + V * g;
    float xo[V + 1];  // other-half entries V g - 1 + par .. V g + V - 1 + par
    {
        // compile-time indices only: a runtime index would put xo on the stack
        float v[V];
        ldv(u + ob, v);
        const float edge = par ? N::ld(u[ob + V]) : g > 0 ? N::ld(u[ob - 1]) : 0.f;  // g == 0: x = 0
#pragma unroll
        for (int t = 0; t <= V; ++t) {
            const float a = t < V ? v[t] : edge;      // par = 1: xo[t] = v[t]
            const float b = t > 0 ? v[t - 1] : edge;  // par = 0: xo[t] = v[t - 1]
            xo[t] = par ? a : b;
        }
    }
    float qv[V], ym[V], yp[V], zm[V], zp[V], out[V];
    ldv(q + base, qv);
    ldv(u + base - L.sy, ym);
    ldv(u + base + L.sy, yp);
    if (DIM == 3) {
        ldv(u + base - L.sz, zm);
        ldv(u + base + L.sz, zp);
    }
#pragma unroll
    for (int t = 0; t < V; ++t) {
        const float sx = xo[t] + xo[t + 1];
        if (DIM == 3) {
            const float lo = ym[t] + zm[t];
            const float hi = yp[t] + zp[t];
            out[t] = fmaf(c, (sx + lo) + hi, qv[t]);
        } else {
            out[t] = fmaf(c, sx + (ym[t] + yp[t]), qv[t]);
        }
    }
    T* dst = u;
    if constexpr (RES) {
        float own[V];
        ldv(u + base, own);
#pragma unroll
        for (int t = 0; t < V; ++t) out[t] = out[t] - own[t];
        dst = res;
    }
    if (x0 >= 1 && x0 + 2 * (V - 1) <= n - 1) {
        stv(dst + base, out);
    } else {
#pragma unroll
        for (int t = 0; t < V; ++t) {
            const int x = x0 + 2 * t;
            if (x >= 1 && x <= n - 1) dst[base + t] = N::st(out[t]);
        }
    }
}

// Double-float nodes per thread of the colour-split half sweep.
#ifndef GMG_DF_VEC
#define GMG_DF_VEC 2
#endif
constexpr int kDfVec = GMG_DF_VEC;

// Two double-float nodes = one 16-byte vector of a colour-split half row.
__device__ inline void ldv2(const df32* p, df32& a, df32& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = df32(v.x, v.y);
    b = df32(v.z, v.w);
}
__device__ inline void stv2(df32* p, df32 a, df32 b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.hi, a.lo, b.hi, b.lo);
}

// k_rb_half_vec for double-float storage: V (2 or 4) nodes of the colour per
// thread (V/2 16-byte vectors per operand row), the x neighbours the V+1
// consecutive entries of the row's other half.  Same operands in the same
// order as nbr_sum_x on the dense layout (its compensated sum, gs_value).
template <int V>
__device__ __forceinline__ void ldvn(const df32* p, df32 (&v)[V]) {
#pragma unroll
    for (int h = 0; h < V / 2; ++h) ldv2(p + 2 * h, v[2 * h], v[2 * h + 1]);
}
// One work item w of the colour-split double-float half sweep: the colour's
// Gauss-Seidel values out[] at its V nodes, from row offset base on (x of
// the first node x0).  False when the item lies past the row's end.
template <int DIM, int V>
__device__ __forceinline__ bool vec_df_item(const df32* __restrict__ u,
                                            const df32* __restrict__ q, const Lay& L, int color,
                                            FastDiv fG, FastDiv fm, uint32_t w, int64_t& base,
                                            int& x0, df32 (&out)[V]) {
    const df32 c = DIM == 3 ? df32(1.0 / 6.0) : df32(0.25);
    const int n = L.n;
    const uint32_t r = fastdiv(w, fG);
    const int g = (int)(w - r * fG.d);
    const uint32_t kk = DIM == 3 ? fastdiv(r, fm) : 0;
    const int j = (int)(r - kk * fm.d) + 1, k = DIM == 3 ? (int)kk + 1 : 0;
    const int par = (color + j + k) & 1;
    x0 = 2 * V * g + par;
    if (x0 > n - 1) return false;
    const int64_t row = k * L.sz + j * L.sy;
    base = row + (par ? L.he : 0) + V * g;
    const int64_t ob = row + (par ? 0 : L.he) + V * g;
    df32 xo[V + 1];
    {
        // entries V g - 1 + par .. V g + V - 1 + par of the other half, with
        // compile-time indices only (a runtime index would put xo on the stack)
        df32 v[V];
        ldvn(u + ob, v);
        const df32 edge = par ? u[ob + V] : g > 0 ? u[ob - 1] : df32(0.f, 0.f);  // g == 0: x = 0
#pragma unroll
        for (int t = 0; t <= V; ++t) {
            const df32 a = t < V ? v[t] : edge;       // par = 1: xo[t] = v[t]
            const df32 b = t > 0 ? v[t - 1] : edge;   // par = 0: xo[t] = v[t - 1]
            xo[t] = par ? a : b;
        }
    }
    df32 qv[V], ym[V], yp[V], zm[V], zp[V];
    ldvn(q + base, qv);
    ldvn(u + base - L.sy, ym);
    ldvn(u + base + L.sy, yp);
    if (DIM == 3) {
        ldvn(u + base - L.sz, zm);
        ldvn(u + base + L.sz, zp);
    }
#pragma unroll
    for (int t = 0; t < V; ++t) {
        const df32 sum = DIM == 3 ? sum6(xo[t], xo[t + 1], ym[t], zm[t], yp[t], zp[t])
                                  : sum4(xo[t], xo[t + 1], ym[t], yp[t]);
        out[t] = gs_value<DIM, true>(c, sum, qv[t]);
    }
    return true;
}

// Store V double-float values of one work item (one 16-byte vector per two
// nodes where the whole group is interior, node by node at the row's ends).
template <int V>
__device__ __forceinline__ void vec_df_store(df32* __restrict__ dst, int64_t base, int x0, int n,
                                             const df32 (&out)[V]) {
    if (x0 >= 1 && x0 + 2 * (V - 1) <= n - 1) {
#pragma unroll
        for (int h = 0; h < V / 2; ++h) stv2(dst + base + 2 * h, out[2 * h], out[2 * h + 1]);
    } else {
#pragma unroll
        for (int t = 0; t < V; ++t) {
            const int x = x0 + 2 * t;
            if (x >= 1 && x <= n - 1) dst[base + t] = out[t];
        }
    }
}

// skip (may be NULL): the launch does nothing while *skip is nonzero (a
// kernel of a captured step that the step's device-side plan leaves out).
template <int DIM, int V, bool RES = false>
__global__ void __launch_bounds__(256) k_rb_half_vec_df(df32* __restrict__ u,
                                                        const df32* __restrict__ q, Lay L,
                                                        int color, FastDiv fG, FastDiv fm,
                                                        uint32_t items,
                                                        df32* __restrict__ res = nullptr,
                                                        const int* __restrict__ skip = nullptr) {
    static_assert(V == 2 || V == 4, "V nodes of 8 bytes per thread: one or two 16-byte vectors");
    if (skip && *skip) return;
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= items) return;
    int64_t base;
    int x0;
    df32 out[V];
    if (!vec_df_item<DIM, V>(u, q, L, color, fG, fm, w, base, x0, out)) return;
    df32* dst = u;
    if constexpr (RES) {  // sigma = value - u, as k_residual
        df32 own[V];
        ldvn(u + base, own);
#pragma unroll
        for (int t = 0; t < V; ++t) out[t] = out[t] - own[t];
        dst = res;
    }
    vec_df_store<V>(dst, base, x0, L.n, out);
}

// The red half sweep that opens the next cycle, with the stopping-test norm
// of the current iterate folded in: after a black half sweep the residual
// vanishes on the black nodes, and on a red node it is the change the red
// update makes (sigma = value - u).  Writes u = value and r = sigma on the
// red nodes, and per block the sum of sigma^2 (double-float, then FP64
// across the block in a fixed order) to partial[blockIdx.x].  Grid-stride
// over the work items with a fixed grid (one wave: kAheadCtasPerSm CTAs of
// 256 threads per SM), so the partials' count and order do not depend on
// timing.
// k_red_restore_df undoes the update from r.
constexpr int kAheadCtasPerSm = 6;
template <int DIM, int V>
__global__ void __launch_bounds__(256, kAheadCtasPerSm) k_red_ahead_df(df32* __restrict__ u,
                                                      const df32* __restrict__ q,
                                                      df32* __restrict__ r, Lay L, FastDiv fG,
                                                      FastDiv fm, uint32_t items,
                                                      double* __restrict__ partial,
                                                      const int* __restrict__ skip) {
    __shared__ double warp_sums[8];
    if (skip && *skip) return;
    df32 acc2(0.f, 0.f);
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < items;
         w += gridDim.x * blockDim.x) {
        int64_t base;
        int x0;
        df32 out[V];
        if (!vec_df_item<DIM, V>(u, q, L, 0, fG, fm, w, base, x0, out)) continue;
        df32 own[V], sig[V];
        ldvn(u + base, own);
#pragma unroll
        for (int t = 0; t < V; ++t) {
            sig[t] = out[t] - own[t];
            const int x = x0 + 2 * t;
            if (x >= 1 && x <= L.n - 1) acc2 = acc2 + sig[t] * sig[t];
        }
        vec_df_store<V>(u, base, x0, L.n, out);
        vec_df_store<V>(r, base, x0, L.n, sig);
    }
    double acc = (double)acc2;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += warp_sums[k];
        partial[blockIdx.x] = s;
    }
}

// Undo k_red_ahead_df: u -= r on the red nodes, while *flag is nonzero.
// Grid-stride over the work items with a small grid: the launch runs once
// per solve and returns at once in every other cycle.
template <int DIM, int V>
__global__ void __launch_bounds__(256) k_red_restore_df(df32* __restrict__ u,
                                                        const df32* __restrict__ r, Lay L,
                                                        FastDiv fG, FastDiv fm, uint32_t items,
                                                        const int* __restrict__ flag) {
    if (!*flag) return;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < items;
         w += gridDim.x * blockDim.x) {
        const uint32_t rr = fastdiv(w, fG);
        const int g = (int)(w - rr * fG.d);
        const uint32_t kk = DIM == 3 ? fastdiv(rr, fm) : 0;
        const int j = (int)(rr - kk * fm.d) + 1, k = DIM == 3 ? (int)kk + 1 : 0;
        const int par = (j + k) & 1;
        const int x0 = 2 * V * g + par;
        if (x0 > L.n - 1) continue;
        const int64_t base = k * L.sz + j * L.sy + (par ? L.he : 0) + V * g;
        df32 v[V], d[V];
        ldvn(u + base, v);
        ldvn(r + base, d);
#pragma unroll
        for (int t = 0; t < V; ++t) v[t] = v[t] - d[t];
        vec_df_store<V>(u, base, x0, L.n, v);
    }
}

// 3D red-black half sweep by diagonal walkers.  The (n-1)^2 interior rows
// (j, k) form n-1 cyclic diagonals k-1 = (j-1+line) mod (n-1); a walker
// (one threadIdx.y) takes kWalk consecutive rows (j, k) -> (j+1, k+1) of one
// diagonal, one red node per x thread and row, and carries the (y+ + z+)
// pair of each node over as the (y- + z-) pair of the next: 4 adds + 1 fma
// per node instead of 5 + 1.  Where the diagonal wraps (k: n-1 -> 1) the
// colour's x offset flips and the pair is formed afresh.  Walkers are
// numbered segment-major, so the CTAs resident at one time sweep a slab of
// consecutive j.  Red nodes read only black ones, so the node order does not
// matter; the operands and their order are nbr_sum's (a + b == b + a), so
// the result equals k_rb_half's bit for bit.
// 256 threads, at least 4 CTAs per SM (<= 64 registers): the FP64 pipe needs
// the warps more than each thread needs registers.
template <typename T, bool EXACT = false>
__global__ void __launch_bounds__(256, 4) k_rb_half3_walk(T* __restrict__ u, const T* __restrict__ q,
                                                          int n, int color, int segs) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = C(1.0 / 6.0);
    const int m = n - 1;
    const int64_t w = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
    if (w >= (int64_t)m * segs) return;
    const int seg = (int)(w / m), line = (int)(w % m);
    int j = 1 + seg * kWalk;
    const int jend = min(j + kWalk, n);
    int k = 1 + (j - 1 + line) % m;
    const int64_t sy = sy_of(n), sz = sz_of<3>(n);
    while (j < jend) {
        const int run = min(jend - j, n - k);  // rows before k passes n-1
        const int i = 1 + ((1 + j + k + color) & 1) + 2 * (int)threadIdx.x;
        if (i < n) {
            // every black operand of the run is loaded before the first store
            // (the compiler cannot reorder loads across stores to u)
            const int64_t p0 = (int64_t)k * sz + (int64_t)j * sy + i, dp = sy + sz;
            C xm[kWalk], xp[kWalk], yp[kWalk], zp[kWalk], qv[kWalk];
            const C ym0 = N::ld(u[p0 - sy]), zm0 = N::ld(u[p0 - sz]);
#pragma unroll
            for (int r = 0; r < kWalk; ++r) {
                if (r < run) {
                    const int64_t p = p0 + r * dp;
                    xm[r] = N::ld(u[p - 1]);
                    xp[r] = N::ld(u[p + 1]);
                    yp[r] = N::ld(u[p + sy]);
                    zp[r] = N::ld(u[p + sz]);
                    qv[r] = N::ld(q[p]);
                }
            }
            C lo = ym0 + zm0;
#pragma unroll
            for (int r = 0; r < kWalk; ++r) {
                if (r < run) {
                    const C hi = yp[r] + zp[r];
                    u[p0 + r * dp] =
                        N::st(gs_value<3, EXACT>(c, ((xm[r] + xp[r]) + lo) + hi, qv[r]));
                    lo = hi;
                }
            }
        }
        j += run;
        k = 1;  // either the diagonal wrapped or j reached jend
    }
}

// Walker w of the diagonal decomposition above (colour `color`): calls
// f(p, sum, i, j, k) for each of its nodes p = (i, j, k) with
// sum = nbr_sum<3>(u, p) (the same operands in the same order), forming each
// (y- + z-) pair once per run.  For kernels that do not write u (residual,
// norms).
template <typename T, class F>
__device__ inline void walk_nodes(const T* __restrict__ u, int n, int color, int64_t w, int segs,
                                  F&& f) {
    using N = Num<T>;
    using C = typename N::C;
    const int m = n - 1;
    const int seg = (int)(w / m), line = (int)(w % m);
    int j = 1 + seg * kWalk;
    const int jend = min(j + kWalk, n);
    int k = 1 + (j - 1 + line) % m;
    const int64_t sy = sy_of(n), sz = sz_of<3>(n);
    while (j < jend) {
        const int run = min(jend - j, n - k);
        const int i = 1 + ((1 + j + k + color) & 1) + 2 * (int)threadIdx.x;
        if (i < n) {
            int64_t p = (int64_t)k * sz + (int64_t)j * sy + i;
            C lo = N::ld(u[p - sy]) + N::ld(u[p - sz]);
#pragma unroll 1  // rolled: no spills at 64 registers, and faster than unrolled
            for (int r = 0; r < run; ++r, p += sy + sz) {
                const C sx = N::ld(u[p - 1]) + N::ld(u[p + 1]);
                const C hi = N::ld(u[p + sy]) + N::ld(u[p + sz]);
                f(p, (sx + lo) + hi, i, j + r, k + r);
                lo = hi;
            }
        }
        j += run;
        k = 1;
    }
}

// Red-only residual (after a black half sweep) by diagonal walkers: sigma
// at the red nodes, equal to k_residual<3, true>'s bit for bit.
template <typename T, bool EXACT = false>
__global__ void __launch_bounds__(256, 4) k_residual3_walk(const T* __restrict__ u,
                                                           const T* __restrict__ q,
                                                           T* __restrict__ r, int n, int segs) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = C(1.0 / 6.0);
    const int64_t w = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
    if (w >= (int64_t)(n - 1) * segs) return;
    walk_nodes(u, n, 0, w, segs, [&](int64_t p, C sum, int, int, int) {
        r[p] = N::st(gs_value<3, EXACT>(c, sum, N::ld(q[p])) - N::ld(u[p]));
    });
}

// Launch shape of the walker kernels for a 3D level n (128 <= n <= 512):
// block (bx, 256/bx) with bx >= n/2 x threads, walkers and CTAs.
struct WalkLaunch {
    dim3 block;
    int segs;
    int64_t walkers;
    unsigned blocks;
};
inline WalkLaunch walk_launch(int n) {
    WalkLaunch L;
    int bx = 32;
    while (bx < n / 2) bx *= 2;
    L.block = dim3(bx, 256 / bx, 1);
    L.segs = (n - 1 + kWalk - 1) / kWalk;
    L.walkers = (int64_t)(n - 1) * L.segs;
    L.blocks = (unsigned)((L.walkers + L.block.y - 1) / L.block.y);
    return L;
}
// From n = 128 up (at n = 64 the 126 walker CTAs leave SMs idle and the row
// kernels are faster).
inline bool walk_applies(int d, int n, size_t elem) {
    return elem == sizeof(double) && d == 3 && n >= 128 && n <= 512 && rb_walk_enabled();
}

// Weighted Jacobi: u_out = u + omega * sigma, all nodes from u_in.
template <int DIM, bool SPLIT, typename T>
__global__ void __launch_bounds__(256) k_wj(const T* __restrict__ u, T* __restrict__ uo,
                                            const T* __restrict__ q, Lay L, double omega_d) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = DIM == 3 ? C(1.0 / 6.0) : C(0.25);
    const C omega = C(omega_d);
    const int n = L.n;
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    if (j >= n) return;
    const int64_t row = k * L.sz + j * L.sy;
    for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
        const int64_t p = row + xo<SPLIT>(L, i);
        int64_t xm, xp;
        xnb<SPLIT>(L, i, xm, xp);
        const C up = N::ld(u[p]);
        const C sig =
            gs_value<DIM, false>(c, nbr_sum_x<DIM>(u, p, xm, xp, L.sy, L.sz), N::ld(q[p])) - up;
        uo[p] = N::st(fma(omega, sig, up));
    }
}

// sigma on all interior nodes, or on red nodes only (black entries of r are
// never written and never read in that mode).
template <int DIM, bool RED_ONLY, bool SPLIT, typename T, bool EXACT = false>
__global__ void __launch_bounds__(256) k_residual(const T* __restrict__ u, const T* __restrict__ q,
                                                  T* __restrict__ r, Lay L) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = DIM == 3 ? C(1.0 / 6.0) : C(0.25);
    const int n = L.n;
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    if (j >= n) return;
    const int64_t row = k * L.sz + j * L.sy;
    const int step = RED_ONLY ? 2 : 1;
    const int i0 = RED_ONLY ? 1 + ((1 + j + k) & 1) : 1;
    for (int i = i0 + step * threadIdx.x; i < n; i += step * blockDim.x) {
        const int64_t p = row + xo<SPLIT>(L, i);
        int64_t xm, xp;
        xnb<SPLIT>(L, i, xm, xp);
        r[p] = N::st(
            gs_value<DIM, EXACT>(c, nbr_sum_x<DIM>(u, p, xm, xp, L.sy, L.sz), N::ld(q[p])) -
            N::ld(u[p]));
    }
}

// q_c = 4 FW(sigma) at every coarse interior node; u_c = 0 (a fresh coarse
// iterate) or u_c = q_c when the coarse grid has its single unknown (exact
// solve u = b/(2d)).  With RED_ONLY the black-node terms (faces and corners
// in 3D, faces in 2D) are zero and skipped.  F: fine layout, Cl: coarse.
template <int DIM, bool RED_ONLY, bool SPLIT, typename T>
__global__ void __launch_bounds__(256) k_restrict(const T* __restrict__ r, T* __restrict__ qc,
                                                  T* __restrict__ uc, Lay F, Lay Cl, int exact) {
    using N = Num<T>;
    using C = typename N::C;
    const int nc = Cl.n;
    const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int J = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int K = DIM == 3 ? blockIdx.z + 1 : 0;
    if (I >= nc || J >= nc) return;
    const int64_t sy = F.sy, sz = F.sz;
    const int64_t p = (2 * K) * sz + (2 * J) * sy + xo<SPLIT>(F, 2 * I);
    int64_t xm, xp;  // fine x-1, x+1 of the (even) centre 2I
    xnb<SPLIT>(F, 2 * I, xm, xp);
    auto R = [&](int64_t o) { return N::ld(r[p + o]); };
    C v;
    if (DIM == 3) {
        C e = R(xm - sy) + R(xp - sy);
        e += R(xm + sy);
        e += R(xp + sy);
        e += R(xm - sz);
        e += R(xp - sz);
        e += R(-sy - sz);
        e += R(sy - sz);
        e += R(xm + sz);
        e += R(xp + sz);
        e += R(-sy + sz);
        e += R(sy + sz);
        if (RED_ONLY) {
            v = fma(C(0.125), e, C(0.5) * R(0));
        } else {
            C fc = R(xm) + R(xp);
            fc += R(-sy);
            fc += R(sy);
            fc += R(-sz);
            fc += R(sz);
            C co = R(xm - sy - sz) + R(xp - sy - sz);
            co += R(xm + sy - sz);
            co += R(xp + sy - sz);
            co += R(xm - sy + sz);
            co += R(xp - sy + sz);
            co += R(xm + sy + sz);
            co += R(xp + sy + sz);
            v = fma(C(0.0625), co, fma(C(0.125), e, fma(C(0.25), fc, C(0.5) * R(0))));
        }
    } else {
        C co = R(xm - sy) + R(xp - sy);
        co += R(xm + sy);
        co += R(xp + sy);
        if (RED_ONLY) {
            v = fma(C(0.25), co, R(0));
        } else {
            C fc = R(xm) + R(xp);
            fc += R(-sy);
            fc += R(sy);
            v = fma(C(0.25), co, fma(C(0.5), fc, R(0)));
        }
    }
    const int64_t P = (int64_t)K * Cl.sz + (int64_t)J * Cl.sy + xo_any(Cl, I);
    qc[P] = N::st(v);
    uc[P] = exact ? N::st(v) : N::st(C(0));
}

// u += P u_c, one thread per coarse cell (I,J,K) in [0, nc-1]^d updating
// the fine nodes (2I+a, 2J+b, 2K+c), a,b,c in {0,1}, that are interior.
// BLACK_ONLY: only the black fine nodes (a+b+c odd) are corrected.  Used
// where a red half sweep comes next: it overwrites every red node from its
// black neighbours without reading the old red value, so the red
// corrections would never be seen (13 instead of 20 ops per cell in 3D).
// Cl: coarse layout, F: fine layout.
template <int DIM, bool BLACK_ONLY, bool SPLIT, typename T>
__global__ void __launch_bounds__(256) k_prolong_add(const T* __restrict__ uc, T* __restrict__ u,
                                                     Lay Cl, Lay F) {
    using N = Num<T>;
    using C = typename N::C;
    const int nc = Cl.n;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = DIM == 3 ? blockIdx.z : 0;
    if (I >= nc || J >= nc) return;
    const int64_t sy = F.sy, sz = F.sz, cy = Cl.sy, cz = Cl.sz;
    const int64_t Pr = K * cz + J * cy;
    const int64_t P = Pr + xo_any(Cl, I), P1 = Pr + xo_any(Cl, I + 1);  // x = I, I+1
    const int64_t pr = (2 * K) * sz + (2 * J) * sy;
    const int64_t p = pr + xo<SPLIT>(F, 2 * I), p1 = pr + xo<SPLIT>(F, 2 * I + 1);  // x = 2I, 2I+1
    const C c000 = N::ld(uc[P]), c100 = N::ld(uc[P1]), c010 = N::ld(uc[P + cy]),
            c110 = N::ld(uc[P1 + cy]);
    const C x00 = c000 + c100;
    const C x10 = c010 + c110;
    const C y00 = c000 + c010;
    const C qxy = x00 + x10;
    auto add = [&](int64_t o, C w, C v) { u[o] = N::st(fma(w, v, N::ld(u[o]))); };
    if (DIM == 2) {
        if (!BLACK_ONLY && I > 0 && J > 0) u[p] = N::st(N::ld(u[p]) + c000);
        if (J > 0) add(p1, C(0.5), x00);
        if (I > 0) add(p + sy, C(0.5), y00);
        if (!BLACK_ONLY) add(p1 + sy, C(0.25), qxy);
    } else {
        const C c001 = N::ld(uc[P + cz]), c101 = N::ld(uc[P1 + cz]),
                c011 = N::ld(uc[P + cy + cz]), c111 = N::ld(uc[P1 + cy + cz]);
        const C x01 = c001 + c101;
        const C x11 = c011 + c111;
        const C y01 = c001 + c011;
        const C z00 = c000 + c001;
        const C qxz = x00 + x01;
        const C qyz = y00 + y01;
        const C oct = qxy + (x01 + x11);
        if (K > 0) {
            if (!BLACK_ONLY && I > 0 && J > 0) u[p] = N::st(N::ld(u[p]) + c000);
            if (J > 0) add(p1, C(0.5), x00);
            if (I > 0) add(p + sy, C(0.5), y00);
            if (!BLACK_ONLY) add(p1 + sy, C(0.25), qxy);
        }
        if (I > 0 && J > 0) add(p + sz, C(0.5), z00);
        if (!BLACK_ONLY && J > 0) add(p1 + sz, C(0.25), qxz);
        if (!BLACK_ONLY && I > 0) add(p + sy + sz, C(0.25), qyz);
        add(p1 + sy + sz, C(0.125), oct);
    }
}

// ------------------------------------------- z-walking transfers (3D, dense,
// fine n >= 128).  A thread takes a few coarse nodes / cells (I, J, K..)
// along z and carries what two neighbours along z share.

constexpr int kZWalk = 4;  // restriction

// Red-only full weighting (after a black half sweep only the red fine nodes
// carry sigma): per coarse node the centre and the twelve red fine nodes two
// of whose offsets are +-1.  The four of an odd fine plane 2K+1 (offsets
// (+-1, 0) and (0, +-1) in it) belong to coarse nodes K and K+1: their sum is
// formed once.  8 adds + 2 multiplies per node instead of 11 + 2; the same
// terms and weights as k_restrict<3, true>, summed in another order.
template <typename T>
__global__ void __launch_bounds__(256) k_restrict3_zwalk(const T* __restrict__ r,
                                                         T* __restrict__ qc, T* __restrict__ uc,
                                                         int n) {
    using N = Num<T>;
    using C = typename N::C;
    const int nc = n / 2;
    const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int J = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int K0 = 1 + (int)blockIdx.z * kZWalk;
    if (I >= nc || J >= nc) return;
    const int64_t sy = sy_of(n), sz = sz_of<3>(n);
    const int64_t cy = sy_of(nc), cz = sz_of<3>(nc);
    auto R = [&](int64_t o) { return N::ld(r[o]); };
    // the four red fine nodes of odd plane z around column (2I, 2J)
    auto odd_plane = [&](int64_t o) { return ((R(o - 1) + R(o + 1)) + R(o - sy)) + R(o + sy); };
    int64_t p = (int64_t)(2 * K0) * sz + (int64_t)(2 * J) * sy + 2 * I;
    int64_t P = (int64_t)K0 * cz + (int64_t)J * cy + I;
    C below = odd_plane(p - sz);
    const int Kend = min(K0 + kZWalk, nc);
    for (int K = K0; K < Kend; ++K, p += 2 * sz, P += cz) {
        const C in_plane = ((R(p - 1 - sy) + R(p + 1 - sy)) + R(p - 1 + sy)) + R(p + 1 + sy);
        const C above = odd_plane(p + sz);
        const C v = fma(C(0.125), (in_plane + below) + above, C(0.5) * R(p));
        qc[P] = N::st(v);
        uc[P] = N::st(C(0));
        below = above;
    }
}

// Black-only trilinear prolongation (a red half sweep comes next): a thread
// takes KZ cells (I, J, K..) along z; the coarse values of plane K+1 and
// their x-pair and face sums are the next cell's plane-K ones.  The operands
// and their order are k_prolong_add<3, true>'s, so the result is the same
// bit for bit.  The corrections are formed first (coarse values only), then
// every fine operand is loaded, then the fine nodes are updated: no load
// waits behind a store.  KZ = 2 at 4 CTAs per SM (64 registers) beats both
// the one-cell kernel and KZ = 4 (fewer adds, but 80 registers).
template <typename T, int KZ>
__global__ void __launch_bounds__(256, 4) k_prolong3_zwalk(const T* __restrict__ uc,
                                                           T* __restrict__ u, int nc) {
    using N = Num<T>;
    using C = typename N::C;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K0 = (int)blockIdx.z * KZ;
    if (I >= nc || J >= nc) return;
    const int n = 2 * nc;
    const int64_t sy = sy_of(n), sz = sz_of<3>(n);
    const int64_t cy = sy_of(nc), cz = sz_of<3>(nc);
    const int64_t P = (int64_t)K0 * cz + (int64_t)J * cy + I;
    const int64_t p = (int64_t)(2 * K0) * sz + (int64_t)(2 * J) * sy + 2 * I;
    const int run = min(KZ, nc - K0);
    C cx[KZ], cyv[KZ], czv[KZ], co[KZ];
    {
        C c00 = N::ld(uc[P]), c01 = N::ld(uc[P + cy]);
        C x0 = c00 + N::ld(uc[P + 1]);
        C face = x0 + (c01 + N::ld(uc[P + 1 + cy]));
#pragma unroll
        for (int t = 0; t < KZ; ++t) {
            if (t < run) {
                const int64_t Q = P + (t + 1) * cz;
                const C d00 = N::ld(uc[Q]), d10 = N::ld(uc[Q + 1]);
                const C d01 = N::ld(uc[Q + cy]), d11 = N::ld(uc[Q + 1 + cy]);
                const C x1 = d00 + d10;
                const C face1 = x1 + (d01 + d11);
                cx[t] = x0;
                cyv[t] = c00 + c01;
                czv[t] = c00 + d00;
                co[t] = face + face1;
                c00 = d00;
                c01 = d01;
                x0 = x1;
                face = face1;
            }
        }
    }
    const bool ex = J > 0, ey = I > 0, ez = I > 0 && J > 0;
    C fx[KZ], fy[KZ], fz[KZ], fo[KZ];
#pragma unroll
    for (int t = 0; t < KZ; ++t) {
        if (t < run) {
            const int64_t pt = p + 2 * t * sz;
            const bool kin = K0 + t > 0;
            fx[t] = kin && ex ? N::ld(u[pt + 1]) : C(0);
            fy[t] = kin && ey ? N::ld(u[pt + sy]) : C(0);
            fz[t] = ez ? N::ld(u[pt + sz]) : C(0);
            fo[t] = N::ld(u[pt + 1 + sy + sz]);
        }
    }
#pragma unroll
    for (int t = 0; t < KZ; ++t) {
        if (t < run) {
            const int64_t pt = p + 2 * t * sz;
            const bool kin = K0 + t > 0;
            if (kin && ex) u[pt + 1] = N::st(fma(C(0.5), cx[t], fx[t]));
            if (kin && ey) u[pt + sy] = N::st(fma(C(0.5), cyv[t], fy[t]));
            if (ez) u[pt + sz] = N::st(fma(C(0.5), czv[t], fz[t]));
            u[pt + 1 + sy + sz] = N::st(fma(C(0.125), co[t], fo[t]));
        }
    }
}

inline bool zwalk_applies(int d, const Lay& F) { return d == 3 && !F.he && F.n >= 128; }

// ------------------------------------------- the paper's own variant
// (dense levels).  Multi-colour Gauss-Seidel: the nodes of colour
// (i&1) + 2(j&1) + 4(k&1) = color, one thread per node of the colour's rows.
template <int DIM, typename T>
__global__ void __launch_bounds__(256) k_mc_sweep(T* __restrict__ u, const T* __restrict__ q,
                                                  Lay L, int color) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = DIM == 3 ? C(1.0 / 6.0) : C(0.25);
    const int n = L.n;
    const int cx = color & 1, cy = (color >> 1) & 1, cz = (color >> 2) & 1;
    // rows j = jb, jb+2, ... with j = cy (mod 2), j >= 1; planes likewise
    const int j = (cy ? 1 : 2) + 2 * (int)(blockIdx.x * blockDim.y + threadIdx.y);
    const int k = DIM == 3 ? (cz ? 1 : 2) + 2 * (int)blockIdx.y : 0;
    if (j >= n || (DIM == 3 && k >= n)) return;
    const int64_t row = k * L.sz + j * L.sy;
    for (int i = (cx ? 1 : 2) + 2 * threadIdx.x; i < n; i += 2 * blockDim.x) {
        const int64_t p = row + i;
        u[p] = N::st(fma(c, nbr_sum<DIM>(u, p, L.sy, L.sz), N::ld(q[p])));
    }
}

// The paper's restriction (eq. Restriction2d, 15-point analogue in 3D),
// q_c = 4 R(sigma) with weight 1/2^d at the centre 2I and 1/2^(d+1) at
// 2I +- delta, delta in {0,1}^d nonzero: the transpose of the diagonal
// prolongation over 2^d.  u_c = 0, or u_c = q_c on the one-unknown grid.
template <int DIM, typename T>
__global__ void __launch_bounds__(256) k_restrict_paper(const T* __restrict__ r,
                                                        T* __restrict__ qc, T* __restrict__ uc,
                                                        Lay F, Lay Cl, int exact) {
    using N = Num<T>;
    using C = typename N::C;
    const int nc = Cl.n;
    const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int J = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int K = DIM == 3 ? blockIdx.z + 1 : 0;
    if (I >= nc || J >= nc) return;
    const int64_t sy = F.sy, sz = F.sz;
    const int64_t p = (2 * K) * sz + (2 * J) * sy + 2 * I;
    auto R = [&](int64_t o) { return N::ld(r[p + o]); };
    // pair sums over +-delta, delta = x, y, xy (2D) and z, xz, yz, xyz (3D)
    C s = (R(-1) + R(1)) + (R(-sy) + R(sy));
    s += R(-1 - sy) + R(1 + sy);
    C v;
    if (DIM == 3) {
        C t = (R(-sz) + R(sz)) + (R(-1 - sz) + R(1 + sz));
        t += (R(-sy - sz) + R(sy + sz)) + (R(-1 - sy - sz) + R(1 + sy + sz));
        v = fma(C(0.25), s + t, C(0.5) * R(0));  // 4 x (1/16, 1/8)
    } else {
        v = fma(C(0.5), s, R(0));  // 4 x (1/8, 1/4)
    }
    const int64_t P = (int64_t)K * Cl.sz + (int64_t)J * Cl.sy + I;
    qc[P] = N::st(v);
    uc[P] = exact ? N::st(v) : N::st(C(0));
}

// The paper's prolongation (eq. Prolongation2d, 3D analogue), u += P u_c:
// one thread per coarse cell (I,J,K) in [0, nc-1]^d; fine node 2I + delta
// gets u_c(I) (delta = 0) or (u_c(I) + u_c(I + delta)) / 2.
template <int DIM, typename T>
__global__ void __launch_bounds__(256) k_prolong_paper(const T* __restrict__ uc,
                                                       T* __restrict__ u, Lay Cl, Lay F) {
    using N = Num<T>;
    using C = typename N::C;
    const int nc = Cl.n;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = DIM == 3 ? blockIdx.z : 0;
    if (I >= nc || J >= nc) return;
    const int64_t sy = F.sy, sz = F.sz, cy = Cl.sy, cz = Cl.sz;
    const int64_t P = K * cz + J * cy + I;
    const int64_t p = (2 * K) * sz + (2 * J) * sy + 2 * I;
    const C c0 = N::ld(uc[P]);
    auto add = [&](int64_t o, int64_t co) {
        u[p + o] = N::st(fma(C(0.5), c0 + N::ld(uc[P + co]), N::ld(u[p + o])));
    };
    const int kz = DIM == 3 ? 2 : 1;
    for (int dz = 0; dz < kz; ++dz) {
        if (DIM == 3 && dz == 0 && K == 0) continue;  // plane 2K = 0 is boundary
        const int64_t oz = dz * sz, coz = dz * cz;
        if (dz == 0) {
            if (I > 0 && J > 0) u[p] = N::st(N::ld(u[p]) + c0);
        } else if (I > 0 && J > 0) {
            add(oz, coz);
        }
        if (J > 0) add(oz + 1, coz + 1);
        if (I > 0) add(oz + sy, coz + cy);
        add(oz + 1 + sy, coz + 1 + cy);
    }
}

// ------------------------------------------------------------- launchers

// FP64 3D dense levels with 128 <= n <= 512 use the diagonal walkers (one red
// node per x thread and row, 256 threads) for the half sweeps and the
// red-only residual unless GMG_RB_WALK=0 (same results bit for bit).
template <typename T>
void rb_half(int d, const Lay& L, T* u, const T* q, int color, cudaStream_t s, bool exact) {
    const int n = L.n;
    constexpr bool kFp64 = std::is_same<T, double>::value;
    exact = exact && kFp64 && d == 3;
    if (L.he == 0 && walk_applies(d, n, sizeof(T))) {
        const WalkLaunch W = walk_launch(n);
        if (exact)
            k_rb_half3_walk<T, kFp64><<<W.blocks, W.block, 0, s>>>(u, q, n, color, W.segs);
        else
            k_rb_half3_walk<T><<<W.blocks, W.block, 0, s>>>(u, q, n, color, W.segs);
        return;
    }
    if (exact) {
        RowLaunch R = row_launch(d, n, n / 2);
        k_rb_half<3, false, T, kFp64><<<R.grid, R.block, 0, s>>>(u, q, L, color);
        return;
    }
    if constexpr (std::is_same<T, float>::value || std::is_same<T, __nv_bfloat16>::value) {
        if (L.he) {
            constexpr int V = vec_of<T>();
            const int G = (n / 2 + 1 + V - 1) / V;
            const int64_t items = (int64_t)G * (d == 3 ? (int64_t)(n - 1) * (n - 1) : n - 1);
            const unsigned blocks = (unsigned)((items + 255) / 256);
            const FastDiv fG = fastdiv_make((uint32_t)G), fm = fastdiv_make((uint32_t)(n - 1));
            if (d == 3)
                k_rb_half_vec<3, T><<<blocks, 256, 0, s>>>(u, q, L, color, fG, fm, (uint32_t)items);
            else
                k_rb_half_vec<2, T><<<blocks, 256, 0, s>>>(u, q, L, color, fG, fm, (uint32_t)items);
            return;
        }
    }
    if constexpr (std::is_same<T, df32>::value) {
        if (L.he) {
            constexpr int V = kDfVec;
            const int G = (n / 2 + 1 + V - 1) / V;
            const int64_t items = (int64_t)G * (d == 3 ? (int64_t)(n - 1) * (n - 1) : n - 1);
            const unsigned blocks = (unsigned)((items + 255) / 256);
            const FastDiv fG = fastdiv_make((uint32_t)G), fm = fastdiv_make((uint32_t)(n - 1));
            if (d == 3)
                k_rb_half_vec_df<3, V><<<blocks, 256, 0, s>>>(u, q, L, color, fG, fm,
                                                              (uint32_t)items);
            else
                k_rb_half_vec_df<2, V><<<blocks, 256, 0, s>>>(u, q, L, color, fG, fm,
                                                              (uint32_t)items);
            return;
        }
    }
    RowLaunch R = row_launch(d, n, n / 2);
    if (d == 3) {
        if (L.he)
            k_rb_half<3, true, T><<<R.grid, R.block, 0, s>>>(u, q, L, color);
        else
            k_rb_half<3, false, T><<<R.grid, R.block, 0, s>>>(u, q, L, color);
    } else {
        if (L.he)
            k_rb_half<2, true, T><<<R.grid, R.block, 0, s>>>(u, q, L, color);
        else
            k_rb_half<2, false, T><<<R.grid, R.block, 0, s>>>(u, q, L, color);
    }
}

template <typename T>
void wj_sweep(int d, const Lay& L, const T* u_in, T* u_out, const T* q, double omega,
              cudaStream_t s) {
    RowLaunch R = row_launch(d, L.n, L.n);
    if (d == 3) {
        if (L.he)
            k_wj<3, true, T><<<R.grid, R.block, 0, s>>>(u_in, u_out, q, L, omega);
        else
            k_wj<3, false, T><<<R.grid, R.block, 0, s>>>(u_in, u_out, q, L, omega);
    } else {
        if (L.he)
            k_wj<2, true, T><<<R.grid, R.block, 0, s>>>(u_in, u_out, q, L, omega);
        else
            k_wj<2, false, T><<<R.grid, R.block, 0, s>>>(u_in, u_out, q, L, omega);
    }
}

template <int DIM, bool SPLIT, typename T, bool EXACT = false>
void residual_rows(const Lay& L, const T* u, const T* q, T* r, bool red_only, cudaStream_t s) {
    RowLaunch R = row_launch(DIM, L.n, red_only ? L.n / 2 : L.n);
    if (red_only)
        k_residual<DIM, true, SPLIT, T, EXACT><<<R.grid, R.block, 0, s>>>(u, q, r, L);
    else
        k_residual<DIM, false, SPLIT, T, EXACT><<<R.grid, R.block, 0, s>>>(u, q, r, L);
}

template <typename T>
void residual(int d, const Lay& L, const T* u, const T* q, T* r, bool red_only, cudaStream_t s,
              bool exact) {
    const int n = L.n;
    constexpr bool kFp64 = std::is_same<T, double>::value;
    exact = exact && kFp64 && d == 3;
    if (red_only && L.he == 0 && walk_applies(d, n, sizeof(T))) {
        const WalkLaunch W = walk_launch(n);
        if (exact)
            k_residual3_walk<T, kFp64><<<W.blocks, W.block, 0, s>>>(u, q, r, n, W.segs);
        else
            k_residual3_walk<T><<<W.blocks, W.block, 0, s>>>(u, q, r, n, W.segs);
        return;
    }
    if (exact && L.he == 0) {
        residual_rows<3, false, T, kFp64>(L, u, q, r, red_only, s);
        return;
    }
    if constexpr (!kFp64) {
        // red-only on the colour-split layout: the vector half-sweep kernel's
        // residual mode (16 bytes of red nodes per operand row and thread)
        if (red_only && L.he) {
            constexpr int V = std::is_same<T, df32>::value ? kDfVec : vec_of<T>();
            const int G = (n / 2 + 1 + V - 1) / V;
            const int64_t items = (int64_t)G * (d == 3 ? (int64_t)(n - 1) * (n - 1) : n - 1);
            const unsigned blocks = (unsigned)((items + 255) / 256);
            const FastDiv fG = fastdiv_make((uint32_t)G), fm = fastdiv_make((uint32_t)(n - 1));
            T* uu = const_cast<T*>(u);  // read only in this mode
            if constexpr (std::is_same<T, df32>::value) {
                if (d == 3)
                    k_rb_half_vec_df<3, V, true><<<blocks, 256, 0, s>>>(uu, q, L, 0, fG, fm,
                                                                        (uint32_t)items, r);
                else
                    k_rb_half_vec_df<2, V, true><<<blocks, 256, 0, s>>>(uu, q, L, 0, fG, fm,
                                                                        (uint32_t)items, r);
            } else {
                if (d == 3)
                    k_rb_half_vec<3, T, true><<<blocks, 256, 0, s>>>(uu, q, L, 0, fG, fm,
                                                                     (uint32_t)items, r);
                else
                    k_rb_half_vec<2, T, true><<<blocks, 256, 0, s>>>(uu, q, L, 0, fG, fm,
                                                                     (uint32_t)items, r);
            }
            return;
        }
    }
    if (d == 3) {
        if (L.he)
            residual_rows<3, true>(L, u, q, r, red_only, s);
        else
            residual_rows<3, false>(L, u, q, r, red_only, s);
    } else {
        if (L.he)
            residual_rows<2, true>(L, u, q, r, red_only, s);
        else
            residual_rows<2, false>(L, u, q, r, red_only, s);
    }
}

template <int DIM, bool SPLIT, typename T>
void restrict_grid(const Lay& F, const Lay& C, const T* r, T* qc, T* uc, bool red_only, int ex,
                   dim3 grid, dim3 block, cudaStream_t s) {
    if (red_only)
        k_restrict<DIM, true, SPLIT, T><<<grid, block, 0, s>>>(r, qc, uc, F, C, ex);
    else
        k_restrict<DIM, false, SPLIT, T><<<grid, block, 0, s>>>(r, qc, uc, F, C, ex);
}

template <typename T>
void restrict_fw(int d, const Lay& F, const Lay& C, const T* r, T* qc, T* uc, bool red_only,
                 bool exact_coarsest, cudaStream_t s) {
    const int nc = C.n;
    int bx = 32;
    while (bx < nc - 1 && bx < 128) bx *= 2;
    const int by = 256 / bx;
    dim3 block(bx, by, 1);
    dim3 grid((nc - 1 + bx - 1) / bx, (nc - 1 + by - 1) / by, d == 3 ? nc - 1 : 1);
    const int ex = exact_coarsest ? 1 : 0;
    if constexpr (std::is_same<T, double>::value) {
        if (red_only && !exact_coarsest && zwalk_applies(d, F)) {
            const dim3 gz(grid.x, grid.y, (unsigned)((nc - 1 + kZWalk - 1) / kZWalk));
            k_restrict3_zwalk<T><<<gz, block, 0, s>>>(r, qc, uc, F.n);
            return;
        }
    }
    if (d == 3) {
        if (F.he)
            restrict_grid<3, true>(F, C, r, qc, uc, red_only, ex, grid, block, s);
        else
            restrict_grid<3, false>(F, C, r, qc, uc, red_only, ex, grid, block, s);
    } else {
        if (F.he)
            restrict_grid<2, true>(F, C, r, qc, uc, red_only, ex, grid, block, s);
        else
            restrict_grid<2, false>(F, C, r, qc, uc, red_only, ex, grid, block, s);
    }
}

template <int DIM, bool SPLIT, typename T>
void prolong_grid(const Lay& C, const Lay& F, const T* uc, T* u, bool black_only, dim3 grid,
                  dim3 block, cudaStream_t s) {
    if (black_only)
        k_prolong_add<DIM, true, SPLIT, T><<<grid, block, 0, s>>>(uc, u, C, F);
    else
        k_prolong_add<DIM, false, SPLIT, T><<<grid, block, 0, s>>>(uc, u, C, F);
}

template <typename T>
void prolong_add(int d, const Lay& C, const Lay& F, const T* uc, T* u, cudaStream_t s,
                 bool black_only) {
    const int nc = C.n;
    int bx = 32;
    while (bx < nc && bx < 128) bx *= 2;
    const int by = 256 / bx;
    dim3 block(bx, by, 1);
    dim3 grid((nc + bx - 1) / bx, (nc + by - 1) / by, d == 3 ? nc : 1);
    if constexpr (std::is_same<T, double>::value) {
        if (black_only && zwalk_applies(d, F)) {
            constexpr int KZ = 2;
            const dim3 gz(grid.x, grid.y, (unsigned)((nc + KZ - 1) / KZ));
            k_prolong3_zwalk<T, KZ><<<gz, block, 0, s>>>(uc, u, nc);
            return;
        }
    }
    if (d == 3) {
        if (F.he)
            prolong_grid<3, true>(C, F, uc, u, black_only, grid, block, s);
        else
            prolong_grid<3, false>(C, F, uc, u, black_only, grid, block, s);
    } else {
        if (F.he)
            prolong_grid<2, true>(C, F, uc, u, black_only, grid, block, s);
        else
            prolong_grid<2, false>(C, F, uc, u, black_only, grid, block, s);
    }
}

template <typename T>
void mc_sweep(int d, const Lay& L, T* u, const T* q, int color, cudaStream_t s) {
    const int n = L.n;
    int bx = 32;
    while (bx < n / 2 && bx < 128) bx *= 2;
    const int by = 256 / bx;
    const int rows = n / 2;  // rows of one parity in 1..n-1 (at most n/2)
    dim3 grid((unsigned)((rows + by - 1) / by), d == 3 ? (unsigned)(n / 2) : 1u, 1);
    if (d == 3)
        k_mc_sweep<3, T><<<grid, dim3(bx, by, 1), 0, s>>>(u, q, L, color);
    else
        k_mc_sweep<2, T><<<grid, dim3(bx, by, 1), 0, s>>>(u, q, L, color);
}

template <typename T>
void restrict_paper(int d, const Lay& F, const Lay& C, const T* r, T* qc, T* uc,
                    bool exact_coarsest, cudaStream_t s) {
    const int nc = C.n;
    int bx = 32;
    while (bx < nc - 1 && bx < 128) bx *= 2;
    const int by = 256 / bx;
    dim3 block(bx, by, 1);
    dim3 grid((nc - 1 + bx - 1) / bx, (nc - 1 + by - 1) / by, d == 3 ? nc - 1 : 1);
    const int ex = exact_coarsest ? 1 : 0;
    if (d == 3)
        k_restrict_paper<3, T><<<grid, block, 0, s>>>(r, qc, uc, F, C, ex);
    else
        k_restrict_paper<2, T><<<grid, block, 0, s>>>(r, qc, uc, F, C, ex);
}

template <typename T>
void prolong_paper(int d, const Lay& C, const Lay& F, const T* uc, T* u, cudaStream_t s) {
    const int nc = C.n;
    int bx = 32;
    while (bx < nc && bx < 128) bx *= 2;
    const int by = 256 / bx;
    dim3 block(bx, by, 1);
    dim3 grid((nc + bx - 1) / bx, (nc + by - 1) / by, d == 3 ? nc : 1);
    if (d == 3)
        k_prolong_paper<3, T><<<grid, block, 0, s>>>(uc, u, C, F);
    else
        k_prolong_paper<2, T><<<grid, block, 0, s>>>(uc, u, C, F);
}

}  // namespace lk
}  // namespace gmg
