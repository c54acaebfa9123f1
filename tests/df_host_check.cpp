// Host build of the library's double-float arithmetic (csrc/df.cuh) checked
// against exact references: the C casts for the integer-pipe conversions,
// and binary128 (__float128, 113-bit significand) sums and products for the
// double-word and triple-float operations.  Prints one line per check,
// "<name> <cases> <failures> <worst error in units of u^2 or the bound>",
// and exits 0; tests/test_df_host.py reads the lines.
#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "df.cuh"

using gmg::df32;
using gmg::tf32;
using Q = __float128;

namespace {

constexpr double kU2 = 1.0 / 281474976710656.0;  // u^2 = 2^-48, u = 2^-24

std::mt19937_64 rng(12345);

uint64_t dbits(double d) {
    uint64_t b;
    std::memcpy(&b, &d, 8);
    return b;
}
uint32_t fbits(float f) {
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return b;
}
bool same_float(float a, float b) { return (std::isnan(a) && std::isnan(b)) || fbits(a) == fbits(b); }
bool same_double(double a, double b) {
    return (std::isnan(a) && std::isnan(b)) || dbits(a) == dbits(b);
}

// a normalised double-float near magnitude 2^e with random sign
df32 rand_df(int e) {
    std::uniform_real_distribution<double> m(1.0, 2.0);
    const double x = std::ldexp(m(rng), e) * (rng() & 1 ? -1.0 : 1.0);
    return df32(x);
}
Q qv(df32 a) { return (Q)a.hi + (Q)a.lo; }
Q qv(tf32 a) { return (Q)a.t0 + (Q)a.t1 + (Q)a.t2; }
double dq(Q x) { return (double)(x < 0 ? -x : x); }

void report(const char* name, long cases, long fails, double worst) {
    std::printf("%s %ld %ld %.6g\n", name, cases, fails, worst);
}

void check_widen() {
    long cases = 0, fails = 0;
    // every 61st bit pattern, and the neighbourhood of each class boundary
    auto one = [&](uint32_t b) {
        float f;
        std::memcpy(&f, &b, 4);
        ++cases;
        if (!same_double(gmg::cvt::widen(f), (double)f)) ++fails;
    };
    for (uint64_t b = 0; b <= 0xffffffffull; b += 61) one((uint32_t)b);
    for (uint32_t edge : {0x0u, 0x1u, 0x7fffffu, 0x800000u, 0x800001u, 0x7f7fffffu, 0x7f800000u,
                          0x7f800001u, 0x7fc00000u, 0x3f800000u})
        for (uint32_t s : {0x0u, 0x80000000u})
            for (int d = -2; d <= 2; ++d) one((edge | s) + (uint32_t)d);
    report("widen", cases, fails, 0.0);
}

void check_split() {
    long cases = 0, fails = 0;
    auto one = [&](double x) {
        ++cases;
        const gmg::cvt::split_t t = gmg::cvt::split(x);
        const float h = (float)x;
        const float l = (float)(x - (double)h);
        if (!same_float(t.hi, h) || (!std::isinf(h) && !same_float(t.lo, l))) ++fails;
    };
    std::uniform_int_distribution<int> ex(-1080, 1030);
    std::uniform_real_distribution<double> m(1.0, 2.0);
    for (int i = 0; i < 2000000; ++i) one(std::ldexp(m(rng), ex(rng)) * (i & 1 ? -1.0 : 1.0));
    // the fast path's exponent band and its edges, with ties and round-up carries
    for (int e : {-75, -74, -73, -60, 0, 1, 100, 125, 126, 127, 128}) {
        for (int i = 0; i < 20000; ++i) {
            uint64_t b = dbits(std::ldexp(m(rng), e));
            if (i % 4 == 1) b = (b & ~0x1fffffffull) | 0x10000000ull;  // exact tie
            if (i % 4 == 2) b |= 0x000fffffe0000000ull;                 // carry into the exponent
            double x;
            std::memcpy(&x, &b, 8);
            one(i & 8 ? -x : x);
        }
    }
    const double specials[] = {0.0, -0.0, 5e-324, -5e-324, 1e-310, 1.0, -1.0,
                               3.4028234663852886e38, 3.4028235677973366e38, 1e39,
                               (double)INFINITY, -(double)INFINITY, (double)NAN};
    for (double x : specials) one(x);
    report("split", cases, fails, 0.0);
}

// TwoSum / Fast2Sum are exact: the pair sums to a + b
void check_two_sum() {
    long cases = 0, fails = 0;
    std::uniform_int_distribution<int> ex(-60, 60);
    std::uniform_real_distribution<float> m(1.0f, 2.0f);
    for (int i = 0; i < 2000000; ++i) {
        const float a = std::ldexp(m(rng), ex(rng)) * (i & 1 ? -1.f : 1.f);
        const float b = std::ldexp(m(rng), ex(rng)) * (i & 2 ? -1.f : 1.f);
        const df32 s = gmg::dw::two_sum(a, b);
        ++cases;
        if ((Q)s.hi + (Q)s.lo != (Q)a + (Q)b) ++fails;
        if (std::fabs(a) >= std::fabs(b)) {
            const df32 t = gmg::dw::fast_two_sum(a, b);
            ++cases;
            if ((Q)t.hi + (Q)t.lo != (Q)a + (Q)b) ++fails;
        }
    }
    report("two_sum", cases, fails, 0.0);
}

// relative error bounds in units of u^2 (with margin over the published ones)
void check_df_ops() {
    std::uniform_int_distribution<int> ex(-40, 10), near(-3, 3);
    long cases = 0, f_add = 0, f_fast = 0, f_mul = 0, f_sum = 0, f_sixth = 0;
    double w_add = 0, w_fast = 0, w_mul = 0, w_sum = 0, w_sixth = 0;
    for (int i = 0; i < 400000; ++i) {
        const int e = ex(rng);
        const df32 x = rand_df(e), y = rand_df(e + near(rng));
        ++cases;
        // accurate addition: relative to the exact sum
        const Q xs = qv(x) + qv(y);
        if (xs != 0) {
            const double r = dq(qv(x + y) - xs) / dq(xs) / kU2;
            w_add = std::fmax(w_add, r);
            if (r > 4.0) ++f_add;
        }
        // add_fast: relative to |x| + |y|
        const double rf = dq(qv(gmg::dw::add_fast(x, y)) - xs) / (dq(qv(x)) + dq(qv(y))) / kU2;
        w_fast = std::fmax(w_fast, rf);
        if (rf > 4.0) ++f_fast;
        // product
        const Q xp = qv(x) * qv(y);
        const double rm = dq(qv(x * y) - xp) / dq(xp) / kU2;
        w_mul = std::fmax(w_mul, rm);
        if (rm > 6.0) ++f_mul;
        // compensated sums of 6 and 4 neighbours: relative to the sum of magnitudes
        df32 v[6];
        Q ex6 = 0, mag = 0;
        for (auto& t : v) {
            t = rand_df(e + near(rng));
            ex6 += qv(t);
            mag += dq(qv(t));
        }
        const double rs = dq(qv(gmg::dw::sum6(v[0], v[1], v[2], v[3], v[4], v[5])) - ex6) /
                          (double)mag / kU2;
        const Q ex4 = qv(v[0]) + qv(v[1]) + qv(v[2]) + qv(v[3]);
        const double rs4 = dq(qv(gmg::dw::sum4(v[0], v[1], v[2], v[3])) - ex4) /
                           (dq(qv(v[0])) + dq(qv(v[1])) + dq(qv(v[2])) + dq(qv(v[3]))) / kU2;
        w_sum = std::fmax(w_sum, std::fmax(rs, rs4));
        if (rs > 16.0 || rs4 > 12.0) ++f_sum;
        // s / 6 with the triple-float constant (unbiased to 2^-72)
        const double r6 = dq(qv(gmg::dw::sixth(x)) - qv(x) / 6) / dq(qv(x) / 6) / kU2;
        w_sixth = std::fmax(w_sixth, r6);
        if (r6 > 3.0) ++f_sixth;
    }
    report("df_add", cases, f_add, w_add);
    report("df_add_fast", cases, f_fast, w_fast);
    report("df_mul", cases, f_mul, w_mul);
    report("df_sum46", cases, f_sum, w_sum);
    report("df_sixth", cases, f_sixth, w_sixth);
}

// triple-float Gauss-Seidel value q + S c: error below 2^-60 (|q| + |S c|),
// and its FP64 value within one rounding of the exact one
void check_triple() {
    std::uniform_int_distribution<int> ex(-40, 10), near(-3, 3);
    long cases = 0, fails = 0, f_dbl = 0;
    double worst = 0, worst_d = 0;
    const Q sixth = (Q)1 / 6;
    for (int i = 0; i < 400000; ++i) {
        const int e = ex(rng);
        df32 v[6];
        Q s = 0;
        for (auto& t : v) {
            t = rand_df(e + near(rng));
            s += qv(t);
        }
        const df32 q = rand_df(e + near(rng) - 2);
        const bool three = i & 1;
        const tf32 st = three ? gmg::dw::sum_tf(v)
                              : gmg::dw::sum_tf(*reinterpret_cast<const df32(*)[4]>(v));
        const Q sum = three ? s : qv(v[0]) + qv(v[1]) + qv(v[2]) + qv(v[3]);
        const Q c = three ? sixth : (Q)0.25;
        const tf32 r = three ? gmg::dw::fma_tf(st, gmg::kSixth0, gmg::kSixth1, gmg::kSixth2, q)
                             : gmg::dw::fma_tf(st, 0.25f, 0.f, 0.f, q);
        const Q exact = qv(q) + sum * c;
        const double scale = dq(qv(q)) + dq(sum * c);
        const double err = dq(qv(r) - exact) / scale;
        ++cases;
        worst = std::fmax(worst, err / std::ldexp(1.0, -60));
        if (err > std::ldexp(1.0, -60)) ++fails;
        const double d = gmg::dw::tf_to_double(r);
        const double ed = dq((Q)d - exact) / scale;
        worst_d = std::fmax(worst_d, ed / std::ldexp(1.0, -52));
        if (ed > std::ldexp(1.0, -52)) ++f_dbl;
    }
    report("triple_fma", cases, fails, worst);
    report("triple_to_double", cases, f_dbl, worst_d);
}

}  // namespace

int main() {
    check_widen();
    check_split();
    check_two_sum();
    check_df_ops();
    check_triple();
    return 0;
}
