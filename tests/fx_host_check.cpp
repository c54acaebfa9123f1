// Host build of the fixed-point scaled residual (csrc/fx.cuh) against a
// binary128 (__float128) evaluation of q + (a_1 + ... + a_M)/M - u.  Cases:
// neighbours close to u (the residual a small difference of large values,
// as in a converging solve), random magnitudes over several binades, exact
// cancellation, zeros among the operands, negative values, and the
// fallback flag for special operands and results below the float range.  Prints one line per check,
// "<name> <cases> <failures> <worst relative error in units of 2^-48>".
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "fx.cuh"

using gmg::df32;
using Q = __float128;

namespace {
std::mt19937_64 rng(777);

template <int M>
Q ref(const double (&a)[M], double q, double u) {
    Q s = 0;
    for (int i = 0; i < M; ++i) s += (Q)a[i];
    return (Q)q + s / (Q)M - (Q)u;
}
Q val(df32 x) { return (Q)x.hi + (Q)x.lo; }

template <int M>
void run(const char* name, int cases, int kind) {
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    long fails = 0;
    double worst = 0;
    for (int c = 0; c < cases; ++c) {
        double a[M], q, u;
        const double scale = std::ldexp(1.0, (int)(rng() % 200) - 100);
        u = U(rng) * scale;
        if (kind == 0) {  // converging: neighbours near u, residual tiny
            const double eps = std::ldexp(1.0, -(int)(rng() % 50));
            for (int i = 0; i < M; ++i) a[i] = u * (1 + eps * U(rng));
            q = u * eps * U(rng) * 0.1;
        } else if (kind == 1) {  // random magnitudes
            for (int i = 0; i < M; ++i) a[i] = U(rng) * std::ldexp(scale, (int)(rng() % 40) - 20);
            q = U(rng) * std::ldexp(scale, (int)(rng() % 40) - 20);
        } else if (kind == 2) {  // exact cancellation: sigma = 0
            for (int i = 0; i < M; ++i) a[i] = u;
            q = 0.0;
        } else {  // zeros among the operands
            for (int i = 0; i < M; ++i) a[i] = (rng() & 1) ? 0.0 : U(rng) * scale;
            q = (rng() & 1) ? 0.0 : U(rng) * scale;
            if (rng() & 1) u = 0.0;
        }
        bool ok = true;
        const df32 s = gmg::fx::sigma<M>(a, q, u, ok);
        const Q r = ref<M>(a, q, u);
        if (!ok) {
            // the FP64 fallback is for results below the float range only
            // (and for special operands, which these cases have none of)
            const Q mag = r < 0 ? -r : r;
            if (mag > (Q)std::ldexp(1.0, -124)) ++fails;
            continue;
        }
        const Q d = val(s) - r;
        Q mag = r < 0 ? -r : r;
        double rel;
        if (mag == 0) {
            rel = val(s) == 0 ? 0.0 : 1e30;
        } else {  // in units of 2^-48 |sigma|, plus the subnormal floats' spacing
            rel = (double)(((d < 0 ? -d : d) - (Q)std::ldexp(1.0, -149)) / mag) *
                  std::ldexp(1.0, 48);
        }
        if (rel > worst) worst = rel;
        if (rel > 1.01) ++fails;
    }
    std::printf("%s %d %ld %.4g\n", name, cases, fails, worst);
}

void special() {
    long fails = 0;
    int cases = 0;
    const double bad[] = {INFINITY, -INFINITY, NAN, 4.9e-324, -1e-310};
    for (double v : bad) {
        double a[6] = {1, 2, 3, 4, 5, v};
        bool ok = true;
        gmg::fx::sigma<6>(a, 0.5, 1.0, ok);
        ++cases;
        if (ok) ++fails;
    }
    double z[6] = {0, 0, 0, 0, 0, 0};
    bool ok = false;
    const df32 s = gmg::fx::sigma<6>(z, 0.0, 0.0, ok);
    ++cases;
    if (!ok || s.hi != 0.f || s.lo != 0.f) ++fails;
    std::printf("special %d %ld 0\n", cases, fails);
}
}  // namespace

int main() {
    run<6>("converging3d", 200000, 0);
    run<6>("random3d", 200000, 1);
    run<6>("cancel3d", 20000, 2);
    run<6>("zeros3d", 50000, 3);
    run<4>("converging2d", 100000, 0);
    run<4>("random2d", 100000, 1);
    special();
    return 0;
}
