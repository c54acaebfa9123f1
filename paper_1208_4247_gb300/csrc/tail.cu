// Persistent tail: the small levels of a V-cycle in one launch of one CTA.
//
// Levels l_tail .. L-1 (the ones with n <= the tail threshold) run entirely
// in shared memory: the CTA loads q of level l_tail (just restricted from the
// level above), runs the rest of the V-cycle -- smoothing, residual,
// full-weighting restriction, exact one-unknown solve (or red-black sweeps on
// a larger coarsest grid), prolongation, smoothing -- with __syncthreads
// between the steps, and writes u of level l_tail back.  It replaces about
// 15 launches per small level, each dominated by launch latency, with one
// launch.  No waits other than __syncthreads.  The arithmetic of every step
// is the level kernels' (level_kernels.cuh), node for node.
#include "level_kernels.cuh"

namespace gmg {
namespace tail {
namespace {

using lk::Num;

template <typename T>
struct SLevel {
    int n;
    T* u;
    T* u2;  // weighted-Jacobi partner
    T* q;
    T* r;
};

template <int DIM>
__device__ inline int64_t nodes_of(int n) {
    const int64_t m = n + 1;
    return DIM == 3 ? m * m * m : m * m;
}

// interior node with linear interior index idx -> (node index, i, j, k);
// NN, the level's n, is a compile-time constant so the divisions are cheap
template <int DIM, int NN>
__device__ inline int64_t inode(int idx, int& i, int& j, int& k) {
    constexpr int m = NN - 1;
    i = idx % m + 1;
    j = (idx / m) % m + 1;
    k = DIM == 3 ? idx / (m * m) + 1 : 0;
    return ((int64_t)k * (NN + 1) + j) * (NN + 1) + i;
}

template <int DIM, int NN>
__device__ constexpr int interior_count() {
    return DIM == 3 ? (NN - 1) * (NN - 1) * (NN - 1) : (NN - 1) * (NN - 1);
}

// f.template operator()<NN>() for the level size n (a power of two, 2..64)
template <class F>
__device__ inline void dispatch_n(int n, F&& f) {
    switch (n) {
        case 2: f.template operator()<2>(); break;
        case 4: f.template operator()<4>(); break;
        case 8: f.template operator()<8>(); break;
        case 16: f.template operator()<16>(); break;
        case 32: f.template operator()<32>(); break;
        default: f.template operator()<64>(); break;
    }
}

// ex: the unbiased FP64 3D value (lk::gs_value), as the grid kernels take
// it on level 0 of a plain FP64 hierarchy
template <int DIM, typename T>
__device__ void rb_half(SLevel<T>& L, int color, bool ex = false) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = DIM == 3 ? C(1.0 / 6.0) : C(0.25);
    dispatch_n(L.n, [&]<int NN>() {
        constexpr int64_t sy = NN + 1, sz = DIM == 3 ? sy * sy : 0;
        for (int idx = threadIdx.x; idx < interior_count<DIM, NN>(); idx += blockDim.x) {
            int i, j, k;
            const int64_t p = inode<DIM, NN>(idx, i, j, k);
            if (((i + j + k) & 1) != color) continue;
            const C s = lk::nbr_sum<DIM>(L.u, p, sy, sz);
            L.u[p] = N::st(ex ? lk::gs_value<DIM, true>(c, s, N::ld(L.q[p]))
                              : lk::gs_value<DIM, false>(c, s, N::ld(L.q[p])));
        }
    });
    __syncthreads();
}

template <int DIM, typename T>
__device__ void wj_sweep(SLevel<T>& L, double omega_d) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = DIM == 3 ? C(1.0 / 6.0) : C(0.25);
    const C omega = C(omega_d);
    dispatch_n(L.n, [&]<int NN>() {
        constexpr int64_t sy = NN + 1, sz = DIM == 3 ? sy * sy : 0;
        for (int idx = threadIdx.x; idx < interior_count<DIM, NN>(); idx += blockDim.x) {
            int i, j, k;
            const int64_t p = inode<DIM, NN>(idx, i, j, k);
            const C up = N::ld(L.u[p]);
            const C sig =
                lk::gs_value<DIM, false>(c, lk::nbr_sum<DIM>(L.u, p, sy, sz), N::ld(L.q[p])) - up;
            L.u2[p] = N::st(fma(omega, sig, up));
        }
    });
    __syncthreads();
    T* t = L.u;
    L.u = L.u2;
    L.u2 = t;
}

template <int DIM, typename T>
__device__ void relax(SLevel<T>& L, int smoother, double omega, int sweeps,
                      bool exact_last = false) {
    for (int s = 0; s < sweeps; ++s) {
        if (smoother == GMG_WJACOBI) {
            wj_sweep<DIM>(L, omega);
        } else {
            rb_half<DIM>(L, 0);
            rb_half<DIM>(L, 1, exact_last && s == sweeps - 1);
        }
    }
}

template <int DIM, typename T>
__device__ void residual(SLevel<T>& L, bool red_only, bool ex = false) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = DIM == 3 ? C(1.0 / 6.0) : C(0.25);
    dispatch_n(L.n, [&]<int NN>() {
        constexpr int64_t sy = NN + 1, sz = DIM == 3 ? sy * sy : 0;
        for (int idx = threadIdx.x; idx < interior_count<DIM, NN>(); idx += blockDim.x) {
            int i, j, k;
            const int64_t p = inode<DIM, NN>(idx, i, j, k);
            if (red_only && ((i + j + k) & 1)) continue;
            const C s = lk::nbr_sum<DIM>(L.u, p, sy, sz);
            const C v = ex ? lk::gs_value<DIM, true>(c, s, N::ld(L.q[p]))
                           : lk::gs_value<DIM, false>(c, s, N::ld(L.q[p]));
            L.r[p] = N::st(v - N::ld(L.u[p]));
        }
    });
    __syncthreads();
}

template <int DIM, typename T>
__device__ void restrict_fw(SLevel<T>& F, SLevel<T>& Cl, bool red_only) {
    using N = Num<T>;
    using C = typename N::C;
    const int nc = Cl.n;
    const int64_t sy = F.n + 1, sz = DIM == 3 ? sy * sy : 0;
    const bool exact = nc == 2;
    dispatch_n(nc, [&]<int NC>() {
    for (int idx = threadIdx.x; idx < interior_count<DIM, NC>(); idx += blockDim.x) {
        int I, J, K;
        const int64_t P = inode<DIM, NC>(idx, I, J, K);
        const int64_t p = (2 * K) * sz + (2 * J) * sy + 2 * I;
        auto R = [&](int64_t o) { return N::ld(F.r[p + o]); };
        C v;
        if (DIM == 3) {
            C e = R(-1 - sy) + R(1 - sy);
            e += R(-1 + sy);
            e += R(1 + sy);
            e += R(-1 - sz);
            e += R(1 - sz);
            e += R(-sy - sz);
            e += R(sy - sz);
            e += R(-1 + sz);
            e += R(1 + sz);
            e += R(-sy + sz);
            e += R(sy + sz);
            if (red_only) {
                v = fma(C(0.125), e, C(0.5) * R(0));
            } else {
                C fc = R(-1) + R(1);
                fc += R(-sy);
                fc += R(sy);
                fc += R(-sz);
                fc += R(sz);
                C co = R(-1 - sy - sz) + R(1 - sy - sz);
                co += R(-1 + sy - sz);
                co += R(1 + sy - sz);
                co += R(-1 - sy + sz);
                co += R(1 - sy + sz);
                co += R(-1 + sy + sz);
                co += R(1 + sy + sz);
                v = fma(C(0.0625), co, fma(C(0.125), e, fma(C(0.25), fc, C(0.5) * R(0))));
            }
        } else {
            C co = R(-1 - sy) + R(1 - sy);
            co += R(-1 + sy);
            co += R(1 + sy);
            if (red_only) {
                v = fma(C(0.25), co, R(0));
            } else {
                C fc = R(-1) + R(1);
                fc += R(-sy);
                fc += R(sy);
                v = fma(C(0.25), co, fma(C(0.5), fc, R(0)));
            }
        }
        Cl.q[P] = N::st(v);
        Cl.u[P] = exact ? N::st(v) : N::st(C(0));
    }
    });
    __syncthreads();
}

template <int DIM, typename T>
__device__ void prolong_add(SLevel<T>& Cl, SLevel<T>& F) {
    using N = Num<T>;
    using C = typename N::C;
    const int nc = Cl.n;
    const int64_t sy = F.n + 1, sz = DIM == 3 ? sy * sy : 0;
    const int64_t cy = nc + 1, cz = DIM == 3 ? cy * cy : 0;
    T* u = F.u;
    const T* uc = Cl.u;
    dispatch_n(nc, [&]<int NC>() {
    constexpr int cells = DIM == 3 ? NC * NC * NC : NC * NC;
    for (int cell = threadIdx.x; cell < cells; cell += blockDim.x) {
        const int I = cell % NC, J = (cell / NC) % NC, K = DIM == 3 ? cell / (NC * NC) : 0;
        const int64_t P = K * cz + J * cy + I;
        const int64_t p = (2 * K) * sz + (2 * J) * sy + 2 * I;
        const C c000 = N::ld(uc[P]), c100 = N::ld(uc[P + 1]), c010 = N::ld(uc[P + cy]),
                c110 = N::ld(uc[P + 1 + cy]);
        const C x00 = c000 + c100;
        const C x10 = c010 + c110;
        const C y00 = c000 + c010;
        const C qxy = x00 + x10;
        auto add = [&](int64_t o, C w, C v) { u[o] = N::st(fma(w, v, N::ld(u[o]))); };
        if (DIM == 2) {
            if (I > 0 && J > 0) u[p] = N::st(N::ld(u[p]) + c000);
            if (J > 0) add(p + 1, C(0.5), x00);
            if (I > 0) add(p + sy, C(0.5), y00);
            add(p + 1 + sy, C(0.25), qxy);
        } else {
            const C c001 = N::ld(uc[P + cz]), c101 = N::ld(uc[P + 1 + cz]),
                    c011 = N::ld(uc[P + cy + cz]), c111 = N::ld(uc[P + 1 + cy + cz]);
            const C x01 = c001 + c101;
            const C x11 = c011 + c111;
            const C y01 = c001 + c011;
            const C z00 = c000 + c001;
            const C qxz = x00 + x01;
            const C qyz = y00 + y01;
            const C oct = qxy + (x01 + x11);
            if (K > 0) {
                if (I > 0 && J > 0) u[p] = N::st(N::ld(u[p]) + c000);
                if (J > 0) add(p + 1, C(0.5), x00);
                if (I > 0) add(p + sy, C(0.5), y00);
                add(p + 1 + sy, C(0.25), qxy);
            }
            const int64_t pz = p + sz;
            if (I > 0 && J > 0) add(pz, C(0.5), z00);
            if (J > 0) add(pz + 1, C(0.25), qxz);
            if (I > 0) add(pz + sy, C(0.25), qyz);
            add(pz + 1 + sy, C(0.125), oct);
        }
    }
    });
    __syncthreads();
}

// The V-cycle on levels with n = n_top, n_top/2, ..., n_top >> (levels-1).
template <int DIM, typename T>
__global__ void __launch_bounds__(1024) k_tail(T* __restrict__ u_top, const T* __restrict__ q_top,
                                               Lay top, int levels, int smoother, double omega,
                                               int nu1, int nu2, int coarse_sweeps, int exact0) {
    const int n_top = top.n;
    extern __shared__ __align__(16) unsigned char smem[];
    SLevel<T> lv[8];
    T* base = reinterpret_cast<T*>(smem);
    const bool wjac = smoother == GMG_WJACOBI;
    for (int l = 0; l < levels; ++l) {
        const int64_t m = nodes_of<DIM>(n_top >> l);
        lv[l].n = n_top >> l;
        lv[l].u = base;
        base += m;
        lv[l].u2 = nullptr;
        if (wjac) {
            lv[l].u2 = base;
            base += m;
        }
        lv[l].q = base;
        base += m;
        lv[l].r = base;
        base += m;
    }
    // zero everything (boundaries stay zero), then load q of the top level
    for (int64_t p = threadIdx.x; p < base - reinterpret_cast<T*>(smem); p += blockDim.x)
        reinterpret_cast<T*>(smem)[p] = Num<T>::st(typename Num<T>::C(0));
    __syncthreads();
    // global addressing of dense node p of the top level (top's layout)
    auto gaddr = [&](int64_t p) {
        const int m = n_top + 1;
        const int i = (int)(p % m);
        const int64_t jk = p / m;
        const int j = (int)(jk % m), k = DIM == 3 ? (int)(jk / m) : 0;
        return k * top.sz + j * top.sy + (top.he ? lk::xo<true>(top, i) : i);
    };
    for (int64_t p = threadIdx.x; p < nodes_of<DIM>(n_top); p += blockDim.x) {
        const int64_t g = gaddr(p);
        lv[0].q[p] = q_top[g];
        lv[0].u[p] = u_top[g];
    }
    __syncthreads();
    const bool red_only = smoother != GMG_WJACOBI && nu1 > 0;
    for (int l = 0; l + 1 < levels; ++l) {
        relax<DIM>(lv[l], smoother, omega, nu1, exact0 && l == 0);
        residual<DIM>(lv[l], red_only, exact0 && l == 0);
        restrict_fw<DIM>(lv[l], lv[l + 1], red_only);
    }
    SLevel<T>& B = lv[levels - 1];
    if (levels == 1) {
        relax<DIM>(B, smoother, omega, nu1);
    } else if (B.n > 2) {
        for (int s = 0; s < coarse_sweeps; ++s) {
            rb_half<DIM>(B, 0);
            rb_half<DIM>(B, 1);
        }
    }
    for (int l = levels - 2; l >= 0; --l) {
        prolong_add<DIM>(lv[l + 1], lv[l]);
        relax<DIM>(lv[l], smoother, omega, nu2);
    }
    for (int64_t p = threadIdx.x; p < nodes_of<DIM>(n_top); p += blockDim.x)
        u_top[gaddr(p)] = lv[0].u[p];
}

}  // namespace

size_t smem_bytes(int d, int n_top, int levels, int smoother, size_t elem) {
    size_t total = 0;
    for (int l = 0; l < levels; ++l) {
        const size_t m = n_top >> l;
        const size_t nodes = d == 3 ? (m + 1) * (m + 1) * (m + 1) : (m + 1) * (m + 1);
        total += nodes * (smoother == GMG_WJACOBI ? 4 : 3);
    }
    return total * elem;
}

template <typename T>
cudaError_t launch(int d, const Lay& top, int levels, T* u_top, const T* q_top, int smoother,
                   double omega, int nu1, int nu2, int coarse_sweeps, cudaStream_t s,
                   bool exact_top) {
    const int exact0 = exact_top && std::is_same<T, double>::value && d == 3 ? 1 : 0;
    const size_t bytes = smem_bytes(d, top.n, levels, smoother, sizeof(T));
    cudaError_t e;
    if (d == 3) {
        e = cudaFuncSetAttribute(k_tail<3, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
        if (e != cudaSuccess) return e;
        k_tail<3, T><<<1, 1024, bytes, s>>>(u_top, q_top, top, levels, smoother, omega, nu1, nu2,
                                            coarse_sweeps, exact0);
    } else {
        e = cudaFuncSetAttribute(k_tail<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
        if (e != cudaSuccess) return e;
        k_tail<2, T><<<1, 1024, bytes, s>>>(u_top, q_top, top, levels, smoother, omega, nu1, nu2,
                                            coarse_sweeps, exact0);
    }
    return cudaGetLastError();
}

template cudaError_t launch<double>(int, const Lay&, int, double*, const double*, int, double,
                                    int, int, int, cudaStream_t, bool);
template cudaError_t launch<float>(int, const Lay&, int, float*, const float*, int, double, int,
                                   int, int, cudaStream_t, bool);
template cudaError_t launch<__nv_bfloat16>(int, const Lay&, int, __nv_bfloat16*,
                                           const __nv_bfloat16*, int, double, int, int, int,
                                           cudaStream_t, bool);
template cudaError_t launch<df32>(int, const Lay&, int, df32*, const df32*, int, double, int, int,
                                  int, cudaStream_t, bool);

}  // namespace tail
}  // namespace gmg
