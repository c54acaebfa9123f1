// Fused leg kernels of the V-cycle (Algorithm 1) for the 3D red-black
// inner hierarchies (FP32 and double-float storage, colour-split layout):
//
//   down leg  S half sweeps (alternating colours, the last one black), the
//             red-only residual and the full-weighting restriction of it:
//             reads u and q once, writes u and the coarse right-hand side
//             (and the fresh coarse iterate u_c = 0);
//   up leg    the black-only trilinear prolongation + correction of u from
//             the coarse iterate, then S half sweeps starting with red:
//             reads the coarse iterate, u and q once, writes u.
//
// One CTA owns a CX x CY column of (x, y) nodes and a range of z planes.  It
// streams the planes through a ring in shared memory (TMA box loads, one
// plane per time step, D steps ahead) and runs every stage of the leg as a
// wavefront: at time step t stage s works on plane t - s, so when stage s
// reads planes p-1, p, p+1 they hold exactly the values the unfused kernels
// would see (stage s-1 has reached p+1 earlier in the same step, stage s+1
// reaches p-1 later in it).  In x and y the CTA loads a halo of HL / HH nodes
// around its column and recomputes the halo's values instead of exchanging
// them: stage s is exact on the loaded region shrunk by s nodes, which covers
// the column (and, for the residual and the restriction, the one extra node
// they read).  In z a CTA likewise starts S+2 planes below its range and
// runs S+1 planes past it.
//
// Every node value is formed by the same expression, with the same operands
// in the same order, as the unfused level kernels (level_kernels.cuh:
// k_rb_half_vec / k_rb_half_vec_df, k_residual, k_restrict, k_prolong_add),
// so the fused legs give the unfused cycle bit for bit.
//
// The CTA algorithm (leg_cta) is written once for a "platform" P that
// supplies the thread index, the CTA barrier and the plane loads: the CUDA
// kernel in legs.cu (TMA and mbarriers), and a sequential host emulation
// (tests/legs_host_check.cpp), which runs it with one thread and plain box
// copies.  The header therefore compiles as host C++ too.
#pragma once

#include <cstdint>

#include "df.cuh"

#if defined(__CUDACC__)
#define LEG_HD __host__ __device__ __forceinline__
#else
#define LEG_HD inline
#endif

namespace gmg {
namespace legs {

constexpr int kDown = 0, kUp = 1;
#ifndef GMG_LEG_D
#define GMG_LEG_D 2
#endif
constexpr int kD = GMG_LEG_D;  // plane batches in flight ahead of the one in use

constexpr int rup(int a, int b) { return (a + b - 1) / b * b; }
LEG_HD int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }  // floor, b > 0

// ------------------------------------------------------------ arithmetic
// The node formulas of the level kernels, per storage type.
template <typename T>
struct Ar;
template <>
struct Ar<float> {
    using C = float;
    // k_rb_half_vec: fmaf(1/6, ((x- + x+) + (y- + z-)) + (y+ + z+), q)
    static LEG_HD float gs(float xm, float xp, float ym, float zm, float yp, float zp, float q) {
        const float sx = rn::add(xm, xp);
        const float lo = rn::add(ym, zm);
        const float hi = rn::add(yp, zp);
        return rn::fma(1.f / 6.f, rn::add(rn::add(sx, lo), hi), q);
    }
    static LEG_HD float sub(float a, float b) { return rn::sub(a, b); }
    static LEG_HD float add(float a, float b) { return rn::add(a, b); }
    static LEG_HD float mul(float a, float b) { return rn::mul(a, b); }
    static LEG_HD float fma(float a, float b, float c) { return rn::fma(a, b, c); }
    static LEG_HD float cst(double v) { return (float)v; }
};
template <>
struct Ar<df32> {
    using C = df32;
    // k_rb_half_vec_df: add_fast(sixth(sum6(x-, x+, y-, z-, y+, z+)), q)
    static LEG_HD df32 gs(df32 xm, df32 xp, df32 ym, df32 zm, df32 yp, df32 zp, df32 q) {
        return dw::add_fast(dw::sixth(dw::sum6(xm, xp, ym, zm, yp, zp)), q);
    }
    static LEG_HD df32 sub(df32 a, df32 b) { return a - b; }
    static LEG_HD df32 add(df32 a, df32 b) { return a + b; }
    static LEG_HD df32 mul(df32 a, df32 b) { return a * b; }
    static LEG_HD df32 fma(df32 a, df32 b, df32 c) { return dw::fma(a, b, c); }
    static LEG_HD df32 cst(double v) { return df32(v); }
};

// ------------------------------------------------------------ geometry
// Tile geometry of a leg kernel.  x positions of a region row are stored as
// two half rows of BXH entries (even x, odd x: the colour-split layout of
// the level arrays); V entries (16 bytes) form a group.  A box starts at an
// even x that is a multiple of 2V, so that both half rows start on a 16-byte
// boundary in global memory (a TMA requirement).
template <typename T, int MODE, int S>
struct Geo {
    static constexpr int es = (int)sizeof(T);
    static constexpr int V = 16 / es;
    static constexpr bool DOWN = MODE == kDown;
    static constexpr int D = kD;
    // halo below / above the column (x and y); the up leg's prolongation
    // leaves the region's outermost rows uncorrected, one more row each side
    static constexpr int HL = DOWN ? S + 2 : S + 1;
    static constexpr int HH = DOWN ? S + 1 : S + 1;
    static constexpr int CX = es == 4 ? 64 : 32;   // column width (x), a multiple of 4V
    static constexpr int PADL = rup(HL, 2 * V);
    static constexpr int PADR = rup(PADL + CX + HH, 2 * V) - PADL - CX;
    static constexpr int BXH = (PADL + CX + PADR) / 2;  // entries per half row
    static constexpr int GH = BXH / V;                   // groups per half row
    // planes held: u (S+2+D), q (S+1+D down, S+D up), sigma (3, down)
    static constexpr int RU = S + 2 + D;
    static constexpr int RQ = DOWN ? S + 1 + D : S + D;
    static constexpr int RS = DOWN ? 3 : 0;
    static constexpr int RC = DOWN ? 0 : 4;  // coarse planes (up leg)
#ifndef GMG_LEG_SMEM_KB
#define GMG_LEG_SMEM_KB 224
#endif
    static constexpr int kBudget = GMG_LEG_SMEM_KB * 1024;
    // rows CY (even) from the shared-memory budget
    static constexpr int half_bytes(int by) { return rup(by * BXH * es, 128); }
    static constexpr int by_of(int cy) { return cy + HL + HH; }
    // coarse box (up leg): coarse x I in [xs/2 - OFFC, ...), rows J in [ys_c, ys_c + BYC)
    static constexpr int OFFC = ((PADL / 2) % (2 * V) == 0) ? 0 : 2 * V - (PADL / 2) % (2 * V);
    static constexpr int bxhc() { return rup((OFFC + BXH + 2 + 1) / 2, V); }
    static constexpr int byc_of(int by) { return by / 2 + 3; }
    static constexpr int bytes_of(int cy) {
        return (RU + RQ + RS) * 2 * half_bytes(by_of(cy)) +
               RC * 2 * rup(byc_of(by_of(cy)) * bxhc() * es, 128);
    }
    static constexpr int cy_fit() {
        int cy = 2;
        while (bytes_of(cy + 2) + 256 <= kBudget) cy += 2;
        return cy;
    }
    static constexpr int CY = cy_fit();
    static constexpr int BY = by_of(CY);
    static constexpr int HALF = half_bytes(BY) / es;  // elements per half-plane buffer
    static constexpr int PLANE = 2 * HALF;            // elements per plane slot
    static constexpr int BXHC = bxhc();
    static constexpr int BYC = byc_of(BY);
    static constexpr int HALFC = rup(BYC * BXHC * es, 128) / es;
    static constexpr int PLANEC = 2 * HALFC;
    static constexpr int SMEM = (RU + RQ + RS) * PLANE * es + RC * PLANEC * es + 256;
#ifndef GMG_LEG_NT
    static constexpr int NT = rup(GH * (BY - 2), 32);  // threads: one item each per stage
#else
    static constexpr int NT = GMG_LEG_NT;
#endif
    static_assert(CX % (4 * V) == 0 && BXH % V == 0, "group alignment");
    static_assert(OFFC % 2 == 0, "coarse x parity follows the fine group's");
    static_assert(CY % 2 == 0 && CY >= 4, "tile rows");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Level layout (colour-split: even x at x/2, odd x at he + (x-1)/2).
struct LayS {
    int n, he;
    int64_t sy, sz;
};

template <typename T>
struct LegArgs {
    LayS F, Cl;        // fine level, coarse level
    int zseg;          // planes per CTA: coarse planes (down), fine planes (up)
    const T* u_in;     // fine iterate read (the loads go through the platform)
    T* u_out;          // fine iterate written (a different array: other CTAs read u_in)
    T* qc;             // down: coarse right-hand side written
    T* uc;             // down: coarse iterate written (0)
};

// ------------------------------------------------------------ vector moves
// V consecutive entries (16 bytes) of shared or global memory.
template <typename T, int V>
LEG_HD void vld(const T* p, typename Ar<T>::C (&v)[V]) {
#if defined(__CUDA_ARCH__)
    const float4 a = *reinterpret_cast<const float4*>(p);
    if constexpr (V == 4) {
        v[0] = a.x;
        v[1] = a.y;
        v[2] = a.z;
        v[3] = a.w;
    } else {
        v[0] = df32(a.x, a.y);
        v[1] = df32(a.z, a.w);
    }
#else
    for (int t = 0; t < V; ++t) v[t] = p[t];
#endif
}
template <typename T, int V>
LEG_HD void vst(T* p, const typename Ar<T>::C (&v)[V]) {
#if defined(__CUDA_ARCH__)
    if constexpr (V == 4)
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else
        *reinterpret_cast<float4*>(p) = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
#else
    for (int t = 0; t < V; ++t) p[t] = v[t];
#endif
}

// ------------------------------------------------------------ the CTA
// Platform P:
//   static constexpr bool kHost               true: one host thread plays every thread
//   int tid(), nt();  void sync();           threads and CTA barrier
//   void fence_async();                      generic -> async proxy fence (before slot reuse)
//   void load_u(T* dst, int xh, int y, int z), load_q(...), load_c(...):
//        one half-row box (BXH x BY, or BXHC x BYC for the coarse level)
//        whose first entry is half-row index xh (global, within the row:
//        0.. for the even half, he.. for the odd half), row y, plane z;
//        out-of-range rows / planes / entries read as 0
//   void begin(int bar, int fine_boxes, int coarse_boxes)   the next loads form
//        one batch, signalled on barrier bar (called before them)
//   bool wait(int bar, int parity)           the batch has landed (false: gave up)
//   void drain(int t, int zhi, int zlo)      before leaving after a failed wait:
//        waits (bounded) for the batches still in flight
//   void* host_scratch(size_t bytes)         host only: storage for every thread's registers
// Returns false if a wait gave up (the CTA then stops; the caller records it).
template <typename T, int MODE, int S, class P>
LEG_HD bool leg_cta(P& pl, const LegArgs<T>& a, int bx, int by, int bz, T* smem) {
    using G = Geo<T, MODE, S>;
    using A = Ar<T>;
    using Cx = typename A::C;
    constexpr int V = G::V, BXH = G::BXH, GH = G::GH, BY = G::BY, HALF = G::HALF;
    constexpr int D = G::D;
    constexpr bool DOWN = G::DOWN;
    const int n = a.F.n, nc = a.Cl.n;
    const int x0 = G::CX * bx, y0 = G::CY * by;
    const int xs = x0 - G::PADL, ys = y0 - G::HL;
    const int tid = pl.tid(), nt = pl.nt();

    // z ranges: planes loaded [zlo, zhi], written [wlo, whi), steps [zlo, tend]
    int zlo, zhi, tend, wlo, whi, K0 = 0, K1 = 0;
    if (DOWN) {
        K0 = 1 + a.zseg * bz;
        K1 = K0 + a.zseg < nc ? K0 + a.zseg : nc;
        if (K0 >= K1) return true;
        wlo = 2 * K0 - 1;
        whi = K1 == nc ? n : 2 * K1 - 1;
        zlo = 2 * K0 - 2 - S;
        zhi = 2 * K1 + S;
        tend = 2 * K1 + S;
    } else {
        wlo = 1 + a.zseg * bz;
        whi = wlo + a.zseg < n ? wlo + a.zseg : n;
        if (wlo >= whi) return true;
        zlo = wlo - S;
        zhi = whi - 1 + S;
        tend = whi - 1 + S;
    }
    if (zlo < 0) zlo = 0;
    if (zhi > n) zhi = n;
    const int pmin = zlo + 1 > 1 ? zlo + 1 : 1;      // planes a stage may update
    const int pmax = zhi - 1 < n - 1 ? zhi - 1 : n - 1;

    T* su = smem;                         // RU plane slots
    T* sq = su + G::RU * G::PLANE;        // RQ
    T* ss = sq + G::RQ * G::PLANE;        // RS (sigma, down)
    T* scn = ss + G::RS * G::PLANE;       // RC coarse slots (up)
    auto uslot = [&](int p) { return su + (p % G::RU) * G::PLANE; };
    auto qslot = [&](int p) { return sq + (p % G::RQ) * G::PLANE; };
    auto sslot = [&](int p) { return ss + (p % 3) * G::PLANE; };
    auto cslot = [&](int K) { return scn + (G::RC ? K % (G::RC ? G::RC : 1) : 0) * G::PLANEC; };
    const int xh0 = xs / 2;  // first half-row entry of the region (both halves)
    // coarse box origin (up leg)
    const int xsc = xh0 - G::OFFC;  // first coarse x of the box (a multiple of 2V)
    const int ysc = fdiv(ys, 2);

    // ---- batch L: u plane L, q plane L-1, coarse planes up to floor(L/2) + (L odd)
    int kc_next = fdiv(zlo, 2);  // next coarse plane to load (up leg)
    auto issue = [&](int L) {
        if (tid == 0) {
            pl.fence_async();  // the slots it refills were written through the generic proxy
            const int bar = (L - zlo) % (D + 1);
            const bool wq = L - 1 >= zlo;
            int kmax = -1;
            if (!DOWN) {
                kmax = fdiv(L, 2) + (L & 1);
                if (kmax > nc) kmax = nc;
            }
            const int ncp = kmax >= kc_next ? kmax - kc_next + 1 : 0;
            pl.begin(bar, wq ? 4 : 2, 2 * ncp);  // boxes of the fine and the coarse level
            T* du = uslot(L);
            pl.load_u(du, xh0, ys, L);
            pl.load_u(du + HALF, a.F.he + xh0, ys, L);
            if (wq) {
                T* dq = qslot(L - 1);
                pl.load_q(dq, xh0, ys, L - 1);
                pl.load_q(dq + HALF, a.F.he + xh0, ys, L - 1);
            }
            for (; kc_next <= kmax; ++kc_next) {
                T* dc = cslot(kc_next);
                pl.load_c(dc, xsc / 2, ysc, kc_next);
                pl.load_c(dc + G::HALFC, a.Cl.he + xsc / 2, ysc, kc_next);
            }
        }
    };

    // ---- every thread owns one item of every stage: region row ri = 1 + t / GH
    // (rows 1 .. BY-2) and group gi = t % GH of the colour's half row.  The
    // device computes its item once; the host emulation (P::kHost) runs the
    // stage for every thread index in turn.
    struct Item {
        int ri, yi, offi, xf0, gi;
        bool act, full0, full1;
    };
    auto make_item = [&](int t) {
        Item it;
        const int gi = t % GH;
        it.ri = 1 + t / GH;
        it.gi = gi;
        it.yi = ys + it.ri;
        it.act = t < GH * (BY - 2) && it.yi >= 1 && it.yi <= n - 1;
        it.offi = it.ri * BXH + V * gi;  // item offset within a half-plane buffer
        // the group lies inside the interior for the half of x parity 0 / 1
        it.xf0 = xs + 2 * V * gi;
        it.full0 = it.xf0 >= 1 && it.xf0 + 2 * (V - 1) <= n - 1;
        it.full1 = it.xf0 + 1 >= 1 && it.xf0 + 1 + 2 * (V - 1) <= n - 1;
        return it;
    };
    const Item mine = make_item(tid);
    // Register blocking along z.  At step t every stage of a thread works on
    // the same half row (x parity par) of its item: stage s on plane t - s
    // with colour c_s, and c_s + (t - s) has the parity of c_1 + t - 1.  So
    // the item's z neighbours on planes p -+ 1 are the thread's own stage
    // s-1 values of two steps ago and of this step, and its x neighbours on
    // plane p are its own stage s-1 values of the previous step (the other
    // half row) plus one entry of the neighbouring group.  Per stage the
    // thread keeps out[s] of this step (C), the previous (A) and the one
    // before (B); shared memory carries only what other threads need: the
    // y neighbours (rows ri -+ 1) and the edge entry.  No stage of a step
    // reads what another thread wrote in the same step, so the stages of a
    // step run without barriers.
    struct Regs {
        Cx A[S + 1][V], B[S + 1][V], C[S + 1][V];
    };
    Regs mine_regs;
    Regs* host_regs = nullptr;
    if constexpr (P::kHost)
        host_regs = reinterpret_cast<Regs*>(pl.host_scratch(G::NT * sizeof(Regs)));
    auto each = [&](auto&& f) {
        if constexpr (P::kHost) {
            for (int t = 0; t < G::NT; ++t) f(make_item(t), host_regs[t]);
        } else {
            f(mine, mine_regs);
        }
    };
    const int c1 = DOWN ? ((S - 1) & 1) ^ 1 : 0;  // colour of stage 1
    each([&](const Item&, Regs& R) {
#pragma unroll
        for (int s = 0; s <= S; ++s)
#pragma unroll
            for (int v = 0; v < V; ++v) R.A[s][v] = R.B[s][v] = R.C[s][v] = A::cst(0.0);
    });

    // One stage of the item on plane p, own half row `par`: the Gauss-Seidel
    // values (uo given: the scaled residual of uo) from x neighbours xr (this
    // item's other-half values) and the neighbouring group's edge entry, y
    // neighbours from shared memory, z neighbours zm, zp; nodes outside the
    // interior get 0 (their value in every level array).  The result goes to
    // dst (a plane slot) and to out.
    auto stage = [&](const Item& it, int par, const T* cur, const T* qs, T* dst, const Cx (&xr)[V],
                     const Cx (&zm)[V], const Cx (&zp)[V], const Cx* uo, Cx (&out)[V]) {
        const int ho = par ? HALF : 0, hx = par ? 0 : HALF;
        const T* own = cur + ho + it.offi;
        const T* oth = cur + hx + it.offi;
        const Cx edge = par ? oth[V] : oth[-1];
        Cx xo[V + 1], ym[V], yp[V], qv[V];
#pragma unroll
        for (int t = 0; t <= V; ++t) {
            const Cx e1 = t < V ? xr[t] : edge;       // par = 1: xo[t] = xr[t]
            const Cx e0 = t > 0 ? xr[t - 1] : edge;   // par = 0: xo[t] = xr[t-1]
            xo[t] = par ? e1 : e0;
        }
        vld<T, V>(own - BXH, ym);
        vld<T, V>(own + BXH, yp);
        vld<T, V>(qs + ho + it.offi, qv);
#pragma unroll
        for (int t = 0; t < V; ++t) {
            const Cx g = A::gs(xo[t], xo[t + 1], ym[t], zm[t], yp[t], zp[t], qv[t]);
            out[t] = uo ? A::sub(g, uo[t]) : g;
        }
        if (!(par ? it.full1 : it.full0)) {
            const int xf = it.xf0 + par;
#pragma unroll
            for (int t = 0; t < V; ++t) {
                const int x = xf + 2 * t;
                if (x < 1 || x > n - 1) out[t] = A::cst(0.0);
            }
        }
        vst<T, V>(dst + ho + it.offi, out);
    };

    // ---- coarse plane K: q_c = 4 FW(sigma) on the column's coarse nodes
    // (k_restrict, red only: the 12 red edge nodes and the centre, same order)
    auto restrict_plane = [&](int K) {
        constexpr int CI = G::CX / 2, CJ = G::CY / 2, QI = G::CX / 4;
        const T* s0 = sslot(2 * K - 1);
        const T* s1 = sslot(2 * K);
        const T* s2 = sslot(2 * K + 1);
        const int items = CI * CJ;
        for (int w = tid; w < items; w += nt) {
            const int jl = w / CI, rem = w % CI;
            const int I = x0 / 2 + 2 * (rem % QI) + rem / QI;
            const int J = y0 / 2 + jl;
            if (I < 1 || I > nc - 1 || J < 1 || J > nc - 1) continue;
            // the centre (2I, 2J) in the even half; x -+ 1 in the odd half at c - 1, c
            const int c = (2 * J - ys) * BXH + (I - xh0);
            const int o = HALF + c;
            Cx e = A::add(s1[o - 1 - BXH], s1[o - BXH]);
            e = A::add(e, s1[o - 1 + BXH]);
            e = A::add(e, s1[o + BXH]);
            e = A::add(e, s0[o - 1]);
            e = A::add(e, s0[o]);
            e = A::add(e, s0[c - BXH]);
            e = A::add(e, s0[c + BXH]);
            e = A::add(e, s2[o - 1]);
            e = A::add(e, s2[o]);
            e = A::add(e, s2[c - BXH]);
            e = A::add(e, s2[c + BXH]);
            const Cx vq = A::fma(A::cst(0.125), e, A::mul(A::cst(0.5), s1[c]));
            const int64_t pc = (int64_t)K * a.Cl.sz + (int64_t)J * a.Cl.sy +
                               ((I & 1) ? a.Cl.he + (I >> 1) : (I >> 1));
            a.qc[pc] = vq;
            a.uc[pc] = A::cst(0.0);
        }
    };

    // ---- the column's part of plane p into u_out
    auto write_out = [&](int p) {
        constexpr int GC = G::CX / (2 * V);  // groups per half row of the column
        const T* cur = uslot(p);
        const int items = G::CY * 2 * GC;
        const int64_t pz = (int64_t)p * a.F.sz;
        for (int w = tid; w < items; w += nt) {
            const int rl = w / (2 * GC), rem = w % (2 * GC);
            const int hf = rem / GC, g = rem % GC;
            const int y = y0 + rl;
            if (y < 1 || y > n - 1) continue;
            const int h = G::PADL / 2 + V * g;
            Cx v[V];
            vld<T, V>(cur + (hf ? HALF : 0) + (G::HL + rl) * BXH + h, v);
            vst<T, V>(a.u_out + pz + (int64_t)y * a.F.sy + (hf ? a.F.he : 0) + xh0 + h, v);
        }
    };

    // ---- up leg: the black nodes of the item's half row on plane t (par:
    // their x parity) corrected by P e_c (k_prolong_add, BLACK_ONLY: the
    // same sums in the same order); nodes outside the interior get 0
    auto prolong_item = [&](const Item& it, int par, int t, Cx (&u)[V]) {
        const int K = t >> 1;
        const int b = (G::OFFC + V * it.gi) >> 1;  // coarse half entry of I0 (OFFC, V gi even)
        // coarse value at I = I0 + i (i >= 0) in row pointer r: even I in the
        // even half, odd I in the odd half
        auto cv = [&](const T* r, int i) -> Cx {
            return (i & 1) ? r[G::HALFC + b + ((i - 1) >> 1)] : r[b + (i >> 1)];
        };
        auto row = [&](int Kp, int J) { return cslot(Kp) + (J - ysc) * G::BXHC; };
        const int xf = it.xf0 + par;
        if ((t & 1) == 0) {
            if (par) {  // (2I+1, 2J, 2K): x00, J = y/2
                const T* r = row(K, it.yi >> 1);
#pragma unroll
                for (int i = 0; i < V; ++i)
                    u[i] = A::fma(A::cst(0.5), A::add(cv(r, i), cv(r, i + 1)), u[i]);
            } else {    // (2I, 2J+1, 2K): y00, J = (y-1)/2
                const T* r0 = row(K, (it.yi - 1) >> 1);
                const T* r1 = r0 + G::BXHC;
#pragma unroll
                for (int i = 0; i < V; ++i)
                    u[i] = A::fma(A::cst(0.5), A::add(cv(r0, i), cv(r1, i)), u[i]);
            }
        } else if (!par) {  // (2I, 2J, 2K+1): z00, J = y/2
            const T* r0 = row(K, it.yi >> 1);
            const T* r1 = row(K + 1, it.yi >> 1);
#pragma unroll
            for (int i = 0; i < V; ++i)
                u[i] = A::fma(A::cst(0.5), A::add(cv(r0, i), cv(r1, i)), u[i]);
        } else {            // (2I+1, 2J+1, 2K+1): octet, J = (y-1)/2
            const T* r00 = row(K, (it.yi - 1) >> 1);
            const T* r10 = r00 + G::BXHC;
            const T* r01 = row(K + 1, (it.yi - 1) >> 1);
            const T* r11 = r01 + G::BXHC;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const Cx x00 = A::add(cv(r00, i), cv(r00, i + 1));
                const Cx x10 = A::add(cv(r10, i), cv(r10, i + 1));
                const Cx qxy = A::add(x00, x10);
                const Cx x01 = A::add(cv(r01, i), cv(r01, i + 1));
                const Cx x11 = A::add(cv(r11, i), cv(r11, i + 1));
                u[i] = A::fma(A::cst(0.125), A::add(qxy, A::add(x01, x11)), u[i]);
            }
        }
        if (!(par ? it.full1 : it.full0)) {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const int x = xf + 2 * i;
                if (x < 1 || x > n - 1) u[i] = A::cst(0.0);
            }
        }
    };

    // ---------------------------------------------------------------- run
    for (int L = zlo; L < zlo + D && L <= zhi; ++L) issue(L);
    for (int t = zlo; t <= tend; ++t) {
        if (t + D <= zhi) issue(t + D);
        if (t <= zhi) {
            if (!pl.wait((t - zlo) % (D + 1), ((t - zlo) / (D + 1)) & 1)) {
                pl.drain(t, zhi, zlo);
                return false;
            }
        } else {
            pl.sync();
        }
        const int pr = t - S - 1;  // the residual's plane (down leg)
        const int iu = t % G::RU, iq = t % G::RQ;  // slots of plane t (t >= 0)
        each([&](const Item& it, Regs& R) {
            if (!it.act) return;
            const int par = (c1 + it.yi + t - 1) & 1;
            // stage 0: the loaded plane t (up leg: its black half row, which is
            // this item's, plus the prolongation of the coarse correction)
            if (t <= zhi) {
                T* ld = uslot(t) + (par ? HALF : 0) + it.offi;
                vld<T, V>(ld, R.C[0]);
                if (!DOWN && t >= 1 && t <= n - 1) {
                    prolong_item(it, par, t, R.C[0]);
                    vst<T, V>(ld, R.C[0]);
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) R.C[0][v] = A::cst(0.0);
            }
#pragma unroll
            for (int s = 1; s <= S; ++s) {
                const int p = t - s;
                if (p >= pmin && p <= pmax) {
                    T* cur = su + (iu >= s ? iu - s : iu - s + G::RU) * G::PLANE;
                    const T* qs = sq + (iq >= s ? iq - s : iq - s + G::RQ) * G::PLANE;
                    stage(it, par, cur, qs, cur, R.A[s - 1], R.B[s - 1], R.C[s - 1], nullptr,
                          R.C[s]);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) R.C[s][v] = A::cst(0.0);
                }
            }
            if (DOWN && pr >= pmin && pr <= pmax && it.ri >= G::HL - 1 &&
                it.ri <= G::HL + G::CY - 1) {
                // red residual of plane t-S-1: black x neighbours (stage S of the
                // previous step), black z neighbours (stage S), own red value
                // (stage S-1 of two steps ago)
                Cx sig[V];
                stage(it, par, uslot(pr), qslot(pr), sslot(pr), R.A[S], R.B[S], R.C[S],
                      R.B[S - 1], sig);
            }
#pragma unroll
            for (int s = 0; s <= S; ++s)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    R.B[s][v] = R.A[s][v];
                    R.A[s][v] = R.C[s][v];
                }
        });
        pl.sync();
        {
            const int p = t - S;
            if (p >= wlo && p < whi && p >= 1 && p <= n - 1) write_out(p);
        }
        if (DOWN && pr >= 3 && (pr & 1)) {
            const int K = (pr - 1) / 2;
            if (K >= K0 && K < K1) restrict_plane(K);
        }
    }
    return true;
}

}  // namespace legs
}  // namespace gmg
