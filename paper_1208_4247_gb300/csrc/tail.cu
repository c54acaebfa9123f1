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

constexpr int kMaxGridLevels = 12;
constexpr int kGridThreads = 512;

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

// f.template operator()<NN>() for the level size n (a power of two, 2..128)
template <class F>
__device__ inline void dispatch_n(int n, F&& f) {
    switch (n) {
        case 2: f.template operator()<2>(); break;
        case 4: f.template operator()<4>(); break;
        case 8: f.template operator()<8>(); break;
        case 16: f.template operator()<16>(); break;
        case 32: f.template operator()<32>(); break;
        case 64: f.template operator()<64>(); break;
        default: f.template operator()<128>(); break;
    }
}

// Interior nodes of one colour ((i + j + k) & 1 == color), NN/2 slots per
// interior row: slot idx -> (node index, i, j, k); false for the one slot per
// row that lies past the row's end.
template <int DIM, int NN>
__device__ constexpr int color_slots() {
    return DIM == 3 ? (NN - 1) * (NN - 1) * (NN / 2) : (NN - 1) * (NN / 2);
}
template <int DIM, int NN>
__device__ inline bool cnode(int idx, int color, int64_t& p, int& i, int& j, int& k) {
    constexpr int h = NN / 2, m = NN - 1;
    const int t = idx % h;
    const int row = idx / h;
    j = row % m + 1;
    k = DIM == 3 ? row / m + 1 : 0;
    i = 2 * t + (((color + j + k) & 1) ? 1 : 2);
    p = ((int64_t)k * (NN + 1) + j) * (NN + 1) + i;
    return i <= m;
}

// Who runs a step and how the steps are separated: one CTA (__syncthreads),
// or every CTA of a cooperative launch (a grid barrier).
struct CtaX {
    __device__ int tid() const { return threadIdx.x; }
    __device__ int nt() const { return blockDim.x; }
    __device__ void sync() { __syncthreads(); }
};

// Grid barrier: a monotonic arrival count (zeroed before the launch); the
// b-th barrier waits until b * gridDim.x CTAs have arrived.  Thread 0 of each
// CTA publishes the CTA's writes (fence after the CTA barrier), arrives and
// spins with a limit of kSpinCycles SM clocks; past it the barrier sets
// bar->fault and every later one returns at once, so the kernel always ends
// (the host then reports the fault).  The fence after the spin orders the
// CTA's later loads after the other CTAs' published writes.
struct GridBar {
    unsigned count;
    int fault;
};
constexpr long long kSpinCycles = 200000000LL;  // about 0.1 s
struct GridX {
    GridBar* bar;
    unsigned target = 0;
    __device__ int tid() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ int nt() const { return gridDim.x * blockDim.x; }
    __device__ void sync() {
        __syncthreads();
        target += gridDim.x;
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&bar->count, 1u);
            volatile unsigned* c = &bar->count;
            volatile int* f = &bar->fault;
            const long long t0 = clock64();
            while (*c < target && *f == 0) {
                if (clock64() - t0 > kSpinCycles) {
                    *f = 1;
                    break;
                }
            }
            __threadfence();
        }
        __syncthreads();
    }
};

// The whole grid is one thread-block cluster: the hardware cluster barrier
// (release / acquire at cluster scope, which orders the CTAs' global
// memory accesses too) between the steps.  Every thread of every CTA
// reaches each barrier (the steps call sync() outside divergent code).
struct ClusterX {
    __device__ int tid() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ int nt() const { return gridDim.x * blockDim.x; }
    __device__ void sync() {
        asm volatile(
            "barrier.cluster.arrive.release.aligned;\n\t"
            "barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
};

// ex: the unbiased FP64 3D value (lk::gs_value), as the grid kernels take
// it on level 0 of a plain FP64 hierarchy
template <int DIM, typename T, class X>
__device__ void rb_half(X& x, SLevel<T>& L, int color, bool ex = false) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = DIM == 3 ? C(1.0 / 6.0) : C(0.25);
    dispatch_n(L.n, [&]<int NN>() {
        constexpr int64_t sy = NN + 1, sz = DIM == 3 ? sy * sy : 0;
        for (int idx = x.tid(); idx < color_slots<DIM, NN>(); idx += x.nt()) {
            int i, j, k;
            int64_t p;
            if (!cnode<DIM, NN>(idx, color, p, i, j, k)) continue;
            const C s = lk::nbr_sum<DIM>(L.u, p, sy, sz);
            L.u[p] = N::st(ex ? lk::gs_value<DIM, true>(c, s, N::ld(L.q[p]))
                              : lk::gs_value<DIM, false>(c, s, N::ld(L.q[p])));
        }
    });
    x.sync();
}

template <int DIM, typename T, class X>
__device__ void wj_sweep(X& x, SLevel<T>& L, double omega_d) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = DIM == 3 ? C(1.0 / 6.0) : C(0.25);
    const C omega = C(omega_d);
    dispatch_n(L.n, [&]<int NN>() {
        constexpr int64_t sy = NN + 1, sz = DIM == 3 ? sy * sy : 0;
        for (int idx = x.tid(); idx < interior_count<DIM, NN>(); idx += x.nt()) {
            int i, j, k;
            const int64_t p = inode<DIM, NN>(idx, i, j, k);
            const C up = N::ld(L.u[p]);
            const C sig =
                lk::gs_value<DIM, false>(c, lk::nbr_sum<DIM>(L.u, p, sy, sz), N::ld(L.q[p])) - up;
            L.u2[p] = N::st(fma(omega, sig, up));
        }
    });
    x.sync();
    T* t = L.u;
    L.u = L.u2;
    L.u2 = t;
}

template <int DIM, typename T, class X>
__device__ void relax(X& x, SLevel<T>& L, int smoother, double omega, int sweeps,
                      bool exact_last = false) {
    for (int s = 0; s < sweeps; ++s) {
        if (smoother == GMG_WJACOBI) {
            wj_sweep<DIM>(x, L, omega);
        } else {
            rb_half<DIM>(x, L, 0);
            rb_half<DIM>(x, L, 1, exact_last && s == sweeps - 1);
        }
    }
}

template <int DIM, typename T, class X>
__device__ void residual(X& x, SLevel<T>& L, bool red_only, bool ex = false) {
    using N = Num<T>;
    using C = typename N::C;
    const C c = DIM == 3 ? C(1.0 / 6.0) : C(0.25);
    dispatch_n(L.n, [&]<int NN>() {
        constexpr int64_t sy = NN + 1, sz = DIM == 3 ? sy * sy : 0;
        auto node = [&](int64_t p) {
            const C s = lk::nbr_sum<DIM>(L.u, p, sy, sz);
            const C v = ex ? lk::gs_value<DIM, true>(c, s, N::ld(L.q[p]))
                           : lk::gs_value<DIM, false>(c, s, N::ld(L.q[p]));
            L.r[p] = N::st(v - N::ld(L.u[p]));
        };
        if (red_only) {
            for (int idx = x.tid(); idx < color_slots<DIM, NN>(); idx += x.nt()) {
                int i, j, k;
                int64_t p;
                if (cnode<DIM, NN>(idx, 0, p, i, j, k)) node(p);
            }
        } else {
            for (int idx = x.tid(); idx < interior_count<DIM, NN>(); idx += x.nt()) {
                int i, j, k;
                node(inode<DIM, NN>(idx, i, j, k));
            }
        }
    });
    x.sync();
}

template <int DIM, typename T, class X>
__device__ void restrict_fw(X& x, SLevel<T>& F, SLevel<T>& Cl, bool red_only) {
    using N = Num<T>;
    using C = typename N::C;
    const int nc = Cl.n;
    const int64_t sy = F.n + 1, sz = DIM == 3 ? sy * sy : 0;
    const bool exact = nc == 2;
    dispatch_n(nc, [&]<int NC>() {
    for (int idx = x.tid(); idx < interior_count<DIM, NC>(); idx += x.nt()) {
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
    x.sync();
}

template <int DIM, typename T, class X>
__device__ void prolong_add(X& x, SLevel<T>& Cl, SLevel<T>& F) {
    using N = Num<T>;
    using C = typename N::C;
    const int nc = Cl.n;
    const int64_t sy = F.n + 1, sz = DIM == 3 ? sy * sy : 0;
    const int64_t cy = nc + 1, cz = DIM == 3 ? cy * cy : 0;
    T* u = F.u;
    const T* uc = Cl.u;
    dispatch_n(nc, [&]<int NC>() {
    constexpr int cells = DIM == 3 ? NC * NC * NC : NC * NC;
    for (int cell = x.tid(); cell < cells; cell += x.nt()) {
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
    x.sync();
}

// The V-cycle on levels lv[from..levels-1] (lv[from] given: q set, u = 0 or
// a start), run by x: down (pre-smoothing, residual, restriction), the
// coarsest grid, up (prolongation with correction, post-smoothing).
// exact0: lv[from] is level 0 of a plain FP64 3D hierarchy (unbiased value).
template <int DIM, typename T, class X>
__device__ void vcycle(X& x, SLevel<T>* lv, int from, int levels, int smoother, double omega,
                       int nu1, int nu2, int coarse_sweeps, bool exact0) {
    const bool red_only = smoother != GMG_WJACOBI && nu1 > 0;
    for (int l = from; l + 1 < levels; ++l) {
        relax<DIM>(x, lv[l], smoother, omega, nu1, exact0 && l == from);
        residual<DIM>(x, lv[l], red_only, exact0 && l == from);
        restrict_fw<DIM>(x, lv[l], lv[l + 1], red_only);
    }
    SLevel<T>& B = lv[levels - 1];
    if (levels - from == 1) {
        relax<DIM>(x, B, smoother, omega, nu1);
    } else if (B.n > 2) {
        for (int s = 0; s < coarse_sweeps; ++s) {
            rb_half<DIM>(x, B, 0);
            rb_half<DIM>(x, B, 1);
        }
    }
    for (int l = levels - 2; l >= from; --l) {
        prolong_add<DIM>(x, lv[l + 1], lv[l]);
        relax<DIM>(x, lv[l], smoother, omega, nu2);
    }
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
    CtaX x;
    vcycle<DIM>(x, lv, 0, levels, smoother, omega, nu1, nu2, coarse_sweeps, exact0 != 0);
    for (int64_t p = threadIdx.x; p < nodes_of<DIM>(n_top); p += blockDim.x)
        u_top[gaddr(p)] = lv[0].u[p];
}

// The same V-cycle on the levels' own arrays in global memory (dense
// layout), run by every CTA of a cooperative launch with grid barriers
// between the steps, on the levels with n > cta_n; block 0 alone runs the
// levels with n <= cta_n (__syncthreads) while the others wait at the next
// grid barrier.  One launch replaces the grid kernels of the middle levels
// (launch latency bound there) and the single-CTA tail.
template <typename T>
struct GridArgs {
    SLevel<T> lv[kMaxGridLevels];
    int levels, smoother, nu1, nu2, coarse_sweeps, cta_n;
    double omega;
    GridBar* bar;
};

template <int DIM, typename T, class X>
__device__ void gtail_body(X& gx, GridArgs<T>& a) {
    SLevel<T>* lv = a.lv;
    const bool red_only = a.smoother != GMG_WJACOBI && a.nu1 > 0;
    int lc = 0;  // first level that block 0 takes alone
    while (lc + 1 < a.levels && lv[lc].n > a.cta_n) ++lc;
    for (int l = 0; l < lc; ++l) {
        relax<DIM>(gx, lv[l], a.smoother, a.omega, a.nu1);
        residual<DIM>(gx, lv[l], red_only);
        restrict_fw<DIM>(gx, lv[l], lv[l + 1], red_only);
    }
    if (blockIdx.x == 0) {
        CtaX cx;
        vcycle<DIM>(cx, lv, lc, a.levels, a.smoother, a.omega, a.nu1, a.nu2, a.coarse_sweeps,
                    false);
    }
    gx.sync();
    for (int l = lc - 1; l >= 0; --l) {
        prolong_add<DIM>(gx, lv[l + 1], lv[l]);
        relax<DIM>(gx, lv[l], a.smoother, a.omega, a.nu2);
    }
}

template <int DIM, typename T>
__global__ void __launch_bounds__(kGridThreads) k_gtail(GridArgs<T> a) {
    GridX gx{a.bar};
    gtail_body<DIM>(gx, a);
}

// The same as one thread-block cluster (the grid is the cluster).
template <int DIM, typename T>
__global__ void __launch_bounds__(kGridThreads) k_ctail(GridArgs<T> a) {
    ClusterX cx;
    gtail_body<DIM>(cx, a);
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

template <typename T>
int grid_blocks(int d) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
        return 0;
    const cudaError_t e =
        d == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gtail<3, T>,
                                                               kGridThreads, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gtail<2, T>,
                                                               kGridThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms * per_sm;
}

template <typename T>
cudaError_t launch_grid(int d, int levels, const int* n, T* const* u, T* const* q, T* const* r,
                        int smoother, double omega, int nu1, int nu2, int coarse_sweeps,
                        int cta_n, void* bar, int blocks, cudaStream_t s, int cluster) {
    if (levels < 1 || levels > kMaxGridLevels || smoother != GMG_RBGS ||
        (cluster <= 0 && blocks < 1) || cluster > 16)
        return cudaErrorInvalidValue;
    GridArgs<T> a{};
    for (int l = 0; l < levels; ++l) a.lv[l] = SLevel<T>{n[l], u[l], nullptr, q[l], r[l]};
    a.levels = levels;
    a.smoother = smoother;
    a.nu1 = nu1;
    a.nu2 = nu2;
    a.coarse_sweeps = coarse_sweeps;
    a.cta_n = cta_n;
    a.omega = omega;
    a.bar = static_cast<GridBar*>(bar);
    if (cluster > 0) {
        auto kern = d == 3 ? k_ctail<3, T> : k_ctail<2, T>;
        cudaError_t e = cudaSuccess;
        if (cluster > 8)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(cluster);
        cfg.blockDim = dim3(kGridThreads);
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, kern, a);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(&a.bar->count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    void* args[] = {&a};
    e = d == 3 ? cudaLaunchCooperativeKernel((const void*)k_gtail<3, T>, dim3(blocks),
                                             dim3(kGridThreads), args, 0, s)
               : cudaLaunchCooperativeKernel((const void*)k_gtail<2, T>, dim3(blocks),
                                             dim3(kGridThreads), args, 0, s);
    return e != cudaSuccess ? e : cudaGetLastError();
}

size_t grid_bar_bytes() { return sizeof(GridBar); }

int grid_fault(const void* bar) {
    int v = 0;
    if (cudaMemcpy(&v, &static_cast<const GridBar*>(bar)->fault, sizeof(int),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    return v;
}

#define GMG_GRID_INST(T)                                                                        \
    template int grid_blocks<T>(int);                                                           \
    template cudaError_t launch_grid<T>(int, int, const int*, T* const*, T* const*, T* const*,  \
                                        int, double, int, int, int, int, void*, int,            \
                                        cudaStream_t, int);
GMG_GRID_INST(double)
GMG_GRID_INST(float)
GMG_GRID_INST(__nv_bfloat16)
GMG_GRID_INST(df32)
#undef GMG_GRID_INST

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
