// Host emulation of the fused leg kernels (csrc/legs.cuh): the CTA
// algorithm runs with one thread, plain box copies for the TMA loads (rows,
// planes and entries outside the array read as 0, as the tensor maps make
// them) and no barriers, CTA after CTA, reading u_in and writing u_out.  The
// result is compared bit for bit with the unfused sequence written as plain
// loops over the colour-split level arrays: S half sweeps, the red-only
// residual and the full-weighting restriction (down leg), or the black-only
// prolongation and S half sweeps (up leg).  Every shared-memory and global
// access of the emulation is bounds-checked.  Prints one line per case,
// "<case> <mismatches> <bad accesses>", and exits 0.
#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "legs.cuh"

using gmg::df32;
using namespace gmg::legs;

namespace {

long g_bad = 0;

LayS split_lay(int n) {
    LayS L;
    L.n = n;
    L.he = (n / 2 + 1 + 7) / 8 * 8;
    L.sy = L.he + (n / 2 + 7) / 8 * 8;
    L.sz = L.sy * (n + 1);
    return L;
}
int64_t elems(const LayS& L) { return L.sz * (L.n + 1); }
int64_t at(const LayS& L, int x, int y, int z) {
    return (int64_t)z * L.sz + (int64_t)y * L.sy + ((x & 1) ? L.he + (x >> 1) : (x >> 1));
}

template <typename T>
bool same(const T& a, const T& b) {
    return std::memcmp(&a, &b, sizeof(T)) == 0;
}

template <typename T>
T rnd(std::mt19937_64& g) {
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    if constexpr (sizeof(T) == 4)
        return (float)U(g);
    else
        return df32(U(g));
}

// ---------------------------------------------------------------- unfused
template <typename T>
void half_ref(const LayS& L, T* u, const T* q, int c) {
    using A = Ar<T>;
    const int n = L.n;
    for (int z = 1; z < n; ++z)
        for (int y = 1; y < n; ++y)
            for (int x = 1; x < n; ++x) {
                if (((x + y + z) & 1) != c) continue;
                u[at(L, x, y, z)] =
                    A::gs(u[at(L, x - 1, y, z)], u[at(L, x + 1, y, z)], u[at(L, x, y - 1, z)],
                          u[at(L, x, y, z - 1)], u[at(L, x, y + 1, z)], u[at(L, x, y, z + 1)],
                          q[at(L, x, y, z)]);
            }
}
template <typename T>
void residual_ref(const LayS& L, const T* u, const T* q, T* r) {
    using A = Ar<T>;
    const int n = L.n;
    for (int z = 1; z < n; ++z)
        for (int y = 1; y < n; ++y)
            for (int x = 1; x < n; ++x) {
                if (((x + y + z) & 1) != 0) continue;
                r[at(L, x, y, z)] = A::sub(
                    A::gs(u[at(L, x - 1, y, z)], u[at(L, x + 1, y, z)], u[at(L, x, y - 1, z)],
                          u[at(L, x, y, z - 1)], u[at(L, x, y + 1, z)], u[at(L, x, y, z + 1)],
                          q[at(L, x, y, z)]),
                    u[at(L, x, y, z)]);
            }
}
template <typename T>
void restrict_ref(const LayS& F, const LayS& C, const T* r, T* qc, T* uc) {
    using A = Ar<T>;
    const int nc = C.n;
    for (int K = 1; K < nc; ++K)
        for (int J = 1; J < nc; ++J)
            for (int I = 1; I < nc; ++I) {
                const int x = 2 * I, y = 2 * J, z = 2 * K;
                auto R = [&](int a, int b, int c) { return r[at(F, x + a, y + b, z + c)]; };
                auto e = A::add(R(-1, -1, 0), R(1, -1, 0));
                e = A::add(e, R(-1, 1, 0));
                e = A::add(e, R(1, 1, 0));
                e = A::add(e, R(-1, 0, -1));
                e = A::add(e, R(1, 0, -1));
                e = A::add(e, R(0, -1, -1));
                e = A::add(e, R(0, 1, -1));
                e = A::add(e, R(-1, 0, 1));
                e = A::add(e, R(1, 0, 1));
                e = A::add(e, R(0, -1, 1));
                e = A::add(e, R(0, 1, 1));
                qc[at(C, I, J, K)] = A::fma(A::cst(0.125), e, A::mul(A::cst(0.5), R(0, 0, 0)));
                uc[at(C, I, J, K)] = A::cst(0.0);
            }
}
template <typename T>
void prolong_ref(const LayS& C, const LayS& F, const T* uc, T* u) {
    using A = Ar<T>;
    const int nc = C.n;
    // k_prolong_add with BLACK_ONLY, cell by cell
    for (int K = 0; K < nc; ++K)
        for (int J = 0; J < nc; ++J)
            for (int I = 0; I < nc; ++I) {
                auto c = [&](int a, int b, int d) { return uc[at(C, I + a, J + b, K + d)]; };
                const auto c000 = c(0, 0, 0), c100 = c(1, 0, 0), c010 = c(0, 1, 0),
                           c110 = c(1, 1, 0), c001 = c(0, 0, 1), c101 = c(1, 0, 1),
                           c011 = c(0, 1, 1), c111 = c(1, 1, 1);
                const auto x00 = A::add(c000, c100), x10 = A::add(c010, c110);
                const auto y00 = A::add(c000, c010), qxy = A::add(x00, x10);
                const auto x01 = A::add(c001, c101), x11 = A::add(c011, c111);
                const auto z00 = A::add(c000, c001);
                const auto oct = A::add(qxy, A::add(x01, x11));
                auto add = [&](int x, int y, int z, double w, decltype(x00) v) {
                    T& d = u[at(F, x, y, z)];
                    d = A::fma(A::cst(w), v, d);
                };
                const int x = 2 * I, y = 2 * J, z = 2 * K;
                if (K > 0) {
                    if (J > 0) add(x + 1, y, z, 0.5, x00);
                    if (I > 0) add(x, y + 1, z, 0.5, y00);
                }
                if (I > 0 && J > 0) add(x, y, z + 1, 0.5, z00);
                add(x + 1, y + 1, z + 1, 0.125, oct);
            }
}

// ---------------------------------------------------------------- emulation
template <typename T, int MODE, int S>
struct HostP {
    using G = Geo<T, MODE, S>;
    static constexpr bool kHost = true;
    const T* uin;
    const T* q;
    const T* ec;
    LayS F, Cl;
    const T* smem_lo;
    const T* smem_hi;
    int tid() const { return 0; }
    int nt() const { return 1; }
    void sync() {}
    void fence_async() {}
    void begin(int, int, int) {}
    bool wait(int, int) { return true; }
    void drain(int, int, int) {}
    std::vector<unsigned char> scratch;
    void* host_scratch(size_t bytes) {
        scratch.assign(bytes, 0);
        return scratch.data();
    }
    void check(const T* p, int count) {
        if (p < smem_lo || p + count > smem_hi) ++g_bad;
    }
    void box(T* dst, const T* src, const LayS& L, int bx, int by, int xh, int y, int z) {
        check(dst, bx * by);
        for (int r = 0; r < by; ++r)
            for (int e = 0; e < bx; ++e) {
                const int yy = y + r, ee = xh + e;
                const bool in = z >= 0 && z <= L.n && yy >= 0 && yy <= L.n && ee >= 0 && ee < L.sy;
                if ((ee * (int)sizeof(T)) % 16 != 0 && e == 0) ++g_bad;  // TMA x alignment
                dst[r * bx + e] = in ? src[(int64_t)z * L.sz + (int64_t)yy * L.sy + ee] : T{};
            }
    }
    void load_u(T* dst, int xh, int y, int z) { box(dst, uin, F, G::BXH, G::BY, xh, y, z); }
    void load_q(T* dst, int xh, int y, int z) { box(dst, q, F, G::BXH, G::BY, xh, y, z); }
    void load_c(T* dst, int xh, int y, int z) { box(dst, ec, Cl, G::BXHC, G::BYC, xh, y, z); }
};

template <typename T, int MODE, int S>
long run_case(int n, int nseg, uint64_t seed) {
    using G = Geo<T, MODE, S>;
    std::mt19937_64 g(seed);
    const LayS F = split_lay(n), C = split_lay(n / 2);
    std::vector<T> u(elems(F)), q(elems(F)), ec(elems(C)), qc(elems(C)), uc(elems(C));
    // random interior values, zero boundaries (padding entries random too:
    // they must never matter)
    for (auto& v : u) v = rnd<T>(g);
    for (auto& v : q) v = rnd<T>(g);
    for (auto& v : ec) v = rnd<T>(g);
    auto zero_bd = [](const LayS& L, std::vector<T>& a) {
        for (int z = 0; z <= L.n; ++z)
            for (int y = 0; y <= L.n; ++y)
                for (int x = 0; x <= L.n; ++x)
                    if (x == 0 || y == 0 || z == 0 || x == L.n || y == L.n || z == L.n)
                        a[at(L, x, y, z)] = T{};
    };
    zero_bd(F, u);
    zero_bd(C, ec);
    // reference
    std::vector<T> ur = u, qcr(elems(C)), ucr(elems(C)), r(elems(F));
    for (auto& v : qcr) v = T{};
    for (auto& v : ucr) v = T{};
    for (auto& v : qc) v = T{};
    for (auto& v : uc) v = T{};
    if (MODE == kDown) {
        for (int s = 1; s <= S; ++s) half_ref(F, ur.data(), q.data(), ((S - s) & 1) ^ 1);
        residual_ref(F, ur.data(), q.data(), r.data());
        restrict_ref(F, C, r.data(), qcr.data(), ucr.data());
    } else {
        prolong_ref(C, F, ec.data(), ur.data());
        for (int s = 1; s <= S; ++s) half_ref(F, ur.data(), q.data(), (s - 1) & 1);
    }
    // emulation
    std::vector<T> uo = u;  // u_out starts as a copy (boundaries)
    std::vector<T> smem((G::SMEM - 256) / sizeof(T));
    HostP<T, MODE, S> pl;
    pl.uin = u.data();
    pl.q = q.data();
    pl.ec = ec.data();
    pl.F = F;
    pl.Cl = C;
    pl.smem_lo = smem.data();
    pl.smem_hi = smem.data() + (G::SMEM - 256) / sizeof(T);
    LegArgs<T> a{};
    a.F = F;
    a.Cl = C;
    a.u_in = u.data();
    a.u_out = uo.data();
    a.qc = qc.data();
    a.uc = uc.data();
    const int planes = MODE == kDown ? C.n - 1 : n - 1;
    a.zseg = (planes + nseg - 1) / nseg;
    const int tx = n / G::CX, ty = (n + G::CY - 1) / G::CY, tz = (planes + a.zseg - 1) / a.zseg;
    for (int bz = 0; bz < tz; ++bz)
        for (int by = 0; by < ty; ++by)
            for (int bx = 0; bx < tx; ++bx) {
                for (auto& v : smem) v = rnd<T>(g);  // stale shared memory must not matter
                leg_cta<T, MODE, S>(pl, a, bx, by, bz, smem.data());
            }
    long bad = 0;
    for (int z = 0; z <= n; ++z)
        for (int y = 0; y <= n; ++y)
            for (int x = 0; x <= n; ++x)
                if (!same(uo[at(F, x, y, z)], ur[at(F, x, y, z)])) ++bad;
    if (MODE == kDown) {
        const int nc = C.n;
        for (int z = 1; z < nc; ++z)
            for (int y = 1; y < nc; ++y)
                for (int x = 1; x < nc; ++x) {
                    if (!same(qc[at(C, x, y, z)], qcr[at(C, x, y, z)])) ++bad;
                    if (!same(uc[at(C, x, y, z)], ucr[at(C, x, y, z)])) ++bad;
                }
    }
    return bad;
}

template <typename T, int MODE, int S>
void report(const char* tname, int n, int nseg) {
    g_bad = 0;
    const long mism = run_case<T, MODE, S>(n, nseg, 1000 + 17 * n + 5 * S + MODE + nseg);
    std::printf("%s_%s_S%d_n%d_seg%d %ld %ld\n", tname, MODE == kDown ? "down" : "up", S, n, nseg,
                mism, g_bad);
    std::fflush(stdout);
}

}  // namespace

int main() {
    // single-float path: columns of 64, grids 128 (two columns) and 256
    report<float, kDown, 4>("f32", 128, 3);
    report<float, kDown, 3>("f32", 128, 1);
    report<float, kDown, 2>("f32", 128, 5);
    report<float, kUp, 4>("f32", 128, 3);
    report<float, kUp, 3>("f32", 128, 7);
    report<float, kUp, 2>("f32", 128, 1);
    report<float, kDown, 4>("f32", 256, 4);
    report<float, kUp, 4>("f32", 256, 4);
    // double-float path: columns of 32
    report<df32, kDown, 3>("df", 64, 2);
    report<df32, kDown, 4>("df", 64, 1);
    report<df32, kDown, 2>("df", 64, 3);
    report<df32, kUp, 3>("df", 64, 4);
    report<df32, kUp, 4>("df", 64, 1);
    report<df32, kUp, 2>("df", 64, 2);
    report<df32, kDown, 3>("df", 128, 5);
    report<df32, kUp, 3>("df", 128, 6);
    return 0;
}
