// FP64 kernels of the plain V-cycle: right-hand-side preparation, the
// stopping-test residual norm (Algorithm 3's res), and the double-precision
// instantiation of the level kernels (level_kernels.cuh).
#include <cstdlib>
#include <type_traits>

#include "level_kernels.cuh"

namespace gmg {

namespace lk {
bool rb_walk_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("GMG_RB_WALK");
        return !(v && v[0] == '0');
    }();
    return on;
}

template void rb_half<double>(int, const Lay&, double*, const double*, int, cudaStream_t, bool);
template void wj_sweep<double>(int, const Lay&, const double*, double*, const double*, double,
                               cudaStream_t);
template void residual<double>(int, const Lay&, const double*, const double*, double*, bool,
                               cudaStream_t, bool);
template void restrict_fw<double>(int, const Lay&, const Lay&, const double*, double*, double*,
                                  bool, bool, cudaStream_t);
template void prolong_add<double>(int, const Lay&, const Lay&, const double*, double*,
                                  cudaStream_t, bool);
template void mc_sweep<double>(int, const Lay&, double*, const double*, int, cudaStream_t);
template void restrict_paper<double>(int, const Lay&, const Lay&, const double*, double*,
                                     double*, bool, cudaStream_t);
template void prolong_paper<double>(int, const Lay&, const Lay&, const double*, double*,
                                    cudaStream_t);
}  // namespace lk

namespace fp64 {
namespace {

using lk::sy_of;
using lk::sz_of;

// q = scale * f on interior nodes (scale = h^2 / (2d)); q = u = 0 on the
// boundary.
template <int DIM>
__global__ void __launch_bounds__(256) k_prepare(const double* __restrict__ f, double* __restrict__ q,
                                                 double* __restrict__ u, int n, double scale,
                                                 int* __restrict__ u_nonzero) {
    bool nz = false;
    // rows (j, k) of (n+1) nodes, x contiguous (no per-node index division)
    const int64_t m = sy_of(n);
    const int64_t rows = DIM == 3 ? m * m : m;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; r < rows;
         r += (int64_t)gridDim.x * blockDim.y) {
        const int j = (int)(r % m);
        const int k = DIM == 3 ? (int)(r / m) : 1;
        const bool row_inner = j > 0 && j < n && k > 0 && k < (DIM == 3 ? n : 2);
        const int64_t base = r * m;
        for (int i = threadIdx.x; i <= n; i += blockDim.x) {
            const int64_t p = base + i;
            if (row_inner && i > 0 && i < n) {
                q[p] = scale * f[p];
                if (u_nonzero) nz = nz || __double_as_longlong(u[p]) != 0;
            } else {
                q[p] = 0.0;
                u[p] = 0.0;
            }
        }
    }
    if (nz) *u_nonzero = 1;  // every writer stores the same value
}

constexpr int kNormThreads = 256;

// Sum of sigma^2 over interior nodes.  Blocks stride over the interior rows
// (j, k) so that each thread accumulates many nodes before the fixed warp
// shuffle tree and the fixed cross-warp order; one partial per block.  The
// grid depends on n only, so the result is deterministic.
// With STORE, sigma is also written to sig_out (the learned smoother's input).
// With RED, only red nodes (i + j + k even) are summed: right after a black
// half sweep every black node holds fma(c, nbr_sum, q) of its unchanged red
// neighbours, which this kernel recomputes with the same expression, so each
// black sigma is exactly 0.0 and leaving it out changes the sum only through
// the order of the red terms.
template <int DIM, bool STORE, bool RED>
__global__ void __launch_bounds__(kNormThreads) k_resnorm(const double* __restrict__ u,
                                                          const double* __restrict__ q,
                                                          double* __restrict__ partial, int n,
                                                          double* __restrict__ sig_out) {
    __shared__ double warp_sums[kNormThreads / 32];
    const double c = DIM == 3 ? 1.0 / 6.0 : 0.25;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t rows = DIM == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    double acc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; r < rows;
         r += (int64_t)gridDim.x * blockDim.y) {
        const int j = (int)(r % (n - 1)) + 1;
        const int k = DIM == 3 ? (int)(r / (n - 1)) + 1 : 0;
        const int64_t row = k * sz + j * sy;
        const int step = RED ? 2 : 1;
        const int i0 = RED ? 1 + ((1 + j + k) & 1) : 1;
        for (int i = i0 + step * threadIdx.x; i < n; i += step * blockDim.x) {
            const int64_t p = row + i;
            const double sig = fma(c, lk::nbr_sum<DIM>(u, p, sy, sz), q[p]) - u[p];
            if (STORE) sig_out[p] = sig;
            acc = fma(sig, sig, acc);
        }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if ((t & 31) == 0) warp_sums[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kNormThreads / 32; ++w) s += warp_sums[w];
        partial[blockIdx.x] = s;
    }
}

// One-colour norm by the diagonal walkers (3D, 128 <= n <= 512).  Colour 0
// (red): the same sigma^2 terms as k_resnorm<3, false, true>, summed in
// walker order.  Colour 1 (black): the black half of a solve's first norm.
// A fixed grid strides over the walkers, so the result is deterministic.
__global__ void __launch_bounds__(256, 4) k_resnorm3_walk(const double* __restrict__ u,
                                                          const double* __restrict__ q,
                                                          double* __restrict__ partial, int n,
                                                          int segs, int color) {
    __shared__ double warp_sums[kNormThreads / 32];
    const double c = 1.0 / 6.0;
    const int64_t walkers = (int64_t)(n - 1) * segs;
    double acc = 0.0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; w < walkers;
         w += (int64_t)gridDim.x * blockDim.y)
        lk::walk_nodes(u, n, color, w, segs, [&](int64_t p, double sum, int, int, int) {
            const double sig = fma(c, sum, q[p]) - u[p];
            acc = fma(sig, sig, acc);
        });
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if ((t & 31) == 0) warp_sums[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kNormThreads / 32; ++w) s += warp_sums[w];
        partial[blockIdx.x] = s;
    }
}

// The stopping-test norm after a red-black cycle fused with the first red
// half sweep of the next cycle (3D FP64 walkers).  At a red node the sweep's
// new value fma(c, sum, q) minus the old value is exactly the red-only norm's
// sigma, so one pass gives both: the sigma^2 terms of k_resnorm3_walk (the
// same bits, summed in another fixed order: deterministic) and the node
// updated as k_rb_half3_walk updates it (the same bits), with the old red
// value kept in `save` so that a solve that stops on this norm can put it
// back.  NORM = false: the sweep and the save only.  Every operand of a run
// is loaded before its first store, as in k_rb_half3_walk.
// 256 threads, 3 CTAs per SM: the sixth operand row (the old red value) does
// not fit in 64 registers without spills, and this beats 4 CTAs with spills
// (257^3 and 513^3 solves).
template <int N, bool NORM>
__global__ void __launch_bounds__(256, 3) k_red_ahead3_walk(double* __restrict__ u,
                                                            const double* __restrict__ q,
                                                            double* __restrict__ save,
                                                            double* __restrict__ partial) {
    // the level size is a template argument: every operand address is one
    // base plus an immediate offset, which keeps the kernel within 64
    // registers with four rows of operands in flight
    constexpr int W = lk::kWalk, m = N - 1, segs = (m + W - 1) / W, walkers = m * segs;
    constexpr int64_t sy = N + 1, sz = (int64_t)(N + 1) * (N + 1), dp = sy + sz;
    __shared__ double warp_sums[kNormThreads / 32];
    const double c = 1.0 / 6.0;
    double acc = 0.0;
    for (int w = blockIdx.x * blockDim.y + threadIdx.y; w < walkers; w += gridDim.x * blockDim.y) {
        const int seg = w / m, line = w % m;
        int j = 1 + seg * W;
        const int jend = min(j + W, N);
        int k = 1 + (j - 1 + line) % m;
        while (j < jend) {
            const int run = min(jend - j, N - k);
            const int i = 1 + ((1 + j + k) & 1) + 2 * (int)threadIdx.x;
            if (i < N) {
                const int64_t p0 = (int64_t)k * sz + (int64_t)j * sy + i;
                const double* up = u + p0;
                double xm[W], xp[W], yp[W], zp[W], qv[W], uo[W];
                const double ym0 = up[-sy], zm0 = up[-sz];
#pragma unroll
                for (int r = 0; r < W; ++r) {
                    if (r < run) {
                        xm[r] = up[r * dp - 1];
                        xp[r] = up[r * dp + 1];
                        yp[r] = up[r * dp + sy];
                        zp[r] = up[r * dp + sz];
                        qv[r] = q[p0 + r * dp];
                        uo[r] = up[r * dp];
                    }
                }
                double lo = ym0 + zm0;
#pragma unroll
                for (int r = 0; r < W; ++r) {
                    if (r < run) {
                        const int64_t p = p0 + r * dp;
                        const double hi = yp[r] + zp[r];
                        const double un = fma(c, ((xm[r] + xp[r]) + lo) + hi, qv[r]);
                        if (NORM) {
                            const double sig = un - uo[r];
                            acc = fma(sig, sig, acc);
                        }
                        save[p] = uo[r];
                        u[p] = un;
                        lo = hi;
                    }
                }
            }
            j += run;
            k = 1;
        }
    }
    if (!NORM) return;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if ((t & 31) == 0) warp_sums[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int v = 0; v < kNormThreads / 32; ++v) s += warp_sums[v];
        partial[blockIdx.x] = s;
    }
}

// u = save on the red interior nodes of a dense 3D level n (undoes
// k_red_ahead3_walk's sweep).
__global__ void __launch_bounds__(256) k_red_restore3(double* __restrict__ u,
                                                      const double* __restrict__ save, int n) {
    const int half = n / 2;
    const int64_t m = n - 1, total = m * m * half;
    const int64_t sy = lk::sy_of(n), sz = lk::sz_of<3>(n);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / half;
        const int x = (int)(t - row * half);
        const int j = 1 + (int)(row % m), k = 1 + (int)(row / m);
        const int i = 1 + ((1 + j + k) & 1) + 2 * x;
        if (i < n) {
            const int64_t p = (int64_t)k * sz + (int64_t)j * sy + i;
            u[p] = save[p];
        }
    }
}

// out = (plus ? *plus : 0) + the sum of count partials, in k_sum_partials'
// order.
__global__ void __launch_bounds__(1024) k_sum_partials_plus(const double* __restrict__ partial,
                                                            int count,
                                                            const double* __restrict__ plus,
                                                            double* __restrict__ out) {
    __shared__ double warp_sums[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partial[i];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += warp_sums[w];
        out[0] = plus ? plus[0] + t : t;
    }
}

struct NormLaunch {
    dim3 grid, block;
};

NormLaunch norm_launch(int d, int n, bool red_only = false) {
    const int xcount = red_only ? n / 2 : n;
    int bx = 32;
    while (bx < xcount && bx < 128) bx *= 2;
    const int by = kNormThreads / bx;
    const int64_t rows = d == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    const int64_t blocks = std::min<int64_t>((rows + by - 1) / by, 152 * 8);
    NormLaunch L;
    L.block = dim3(bx, by, 1);
    L.grid = dim3((unsigned)blocks, 1, 1);
    return L;
}

}  // namespace

__global__ void __launch_bounds__(1024) k_sum_partials(const double* __restrict__ partial,
                                                       int count, double* __restrict__ out) {
    __shared__ double warp_sums[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partial[i];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += warp_sums[w];
        out[0] = s;
    }
}

void prepare(int d, int n, const double* f, double* q, double* u, cudaStream_t s,
             int* u_nonzero) {
    const double h = 1.0 / n;
    const double scale = h * h / (2.0 * d);
    int bx = 32;
    while (bx < n + 1 && bx < 256) bx *= 2;
    const dim3 block(bx, 256 / bx, 1);
    const int64_t rows = d == 3 ? (int64_t)(n + 1) * (n + 1) : (int64_t)(n + 1);
    const int blocks = (int)std::min<int64_t>((rows + block.y - 1) / block.y, 152 * 16);
    if (d == 3)
        k_prepare<3><<<blocks, block, 0, s>>>(f, q, u, n, scale, u_nonzero);
    else
        k_prepare<2><<<blocks, block, 0, s>>>(f, q, u, n, scale, u_nonzero);
}

namespace {
// dst = src on all (n+1)^d nodes, each array with its own row / plane pitch
template <int DIM>
__global__ void __launch_bounds__(256) k_copy_strided(const double* __restrict__ src, int64_t ssy,
                                                      int64_t ssz, double* __restrict__ dst,
                                                      int64_t dsy, int64_t dsz, int n) {
    const int64_t m = n + 1;
    const int64_t rows = DIM == 3 ? m * m : m;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; r < rows;
         r += (int64_t)gridDim.x * blockDim.y) {
        const int64_t j = r % m, k = DIM == 3 ? r / m : 0;
        for (int i = threadIdx.x; i <= n; i += blockDim.x)
            dst[k * dsz + j * dsy + i] = src[k * ssz + j * ssy + i];
    }
}
}  // namespace

void copy_strided(int d, int n, const double* src, int64_t ssy, int64_t ssz, double* dst,
                  int64_t dsy, int64_t dsz, cudaStream_t s) {
    int bx = 32;
    while (bx < n + 1 && bx < 128) bx *= 2;
    dim3 block(bx, 256 / bx, 1);
    const int64_t rows = d == 3 ? (int64_t)(n + 1) * (n + 1) : (n + 1);
    const unsigned blocks = (unsigned)std::min<int64_t>((rows + block.y - 1) / block.y, 152 * 16);
    if (d == 3)
        k_copy_strided<3><<<blocks, block, 0, s>>>(src, ssy, ssz, dst, dsy, dsz, n);
    else
        k_copy_strided<2><<<blocks, block, 0, s>>>(src, ssy, ssz, dst, dsy, dsz, n);
}

int resnorm_partials(int d, int n) { return (int)norm_launch(d, n).grid.x; }

bool red_ahead_applies(int d, int n) {
    static const bool on = [] {
        const char* v = std::getenv("GMG_NORM_AHEAD");
        return !(v && v[0] == '0');
    }();
    return on && lk::walk_applies(d, n, sizeof(double));
}

void red_ahead(int n, double* u, const double* q, double* save, double* partial, double* out,
               bool norm, cudaStream_t s, const double* plus) {
    // two waves of 3 resident CTAs per SM stride over the walkers; the
    // partial sums (one per CTA) fit the resnorm buffer (resnorm_partials)
    const lk::WalkLaunch W = lk::walk_launch(n);
    const unsigned blocks = std::min<unsigned>(W.blocks, 152u * 3 * 2);
    auto launch = [&](auto kn) {
        constexpr int N = decltype(kn)::value;
        if (norm)
            k_red_ahead3_walk<N, true><<<blocks, W.block, 0, s>>>(u, q, save, partial);
        else
            k_red_ahead3_walk<N, false><<<blocks, W.block, 0, s>>>(u, q, save, nullptr);
    };
    if (n == 128)
        launch(std::integral_constant<int, 128>{});
    else if (n == 256)
        launch(std::integral_constant<int, 256>{});
    else
        launch(std::integral_constant<int, 512>{});
    if (norm) k_sum_partials_plus<<<1, 1024, 0, s>>>(partial, (int)blocks, plus, out);
}

void resnorm_black(int n, const double* u, const double* q, double* partial, double* out,
                   cudaStream_t s) {
    const lk::WalkLaunch W = lk::walk_launch(n);
    const unsigned blocks = std::min<unsigned>(W.blocks, (unsigned)resnorm_partials(3, n));
    k_resnorm3_walk<<<blocks, W.block, 0, s>>>(u, q, partial, n, W.segs, 1);
    k_sum_partials<<<1, 1024, 0, s>>>(partial, (int)blocks, out);
}

void red_restore(int n, double* u, const double* save, cudaStream_t s) {
    const int64_t total = (int64_t)(n - 1) * (n - 1) * (n / 2);
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 8);
    k_red_restore3<<<blocks, 256, 0, s>>>(u, save, n);
}

void resnorm(int d, int n, const double* u, const double* q, double* partial, double* out,
             cudaStream_t s, double* sigma_out, bool red_only) {
    if (red_only && !sigma_out && lk::walk_applies(d, n, sizeof(double))) {
        const lk::WalkLaunch W = lk::walk_launch(n);
        const unsigned blocks = std::min<unsigned>(W.blocks, (unsigned)resnorm_partials(d, n));
        k_resnorm3_walk<<<blocks, W.block, 0, s>>>(u, q, partial, n, W.segs, 0);
        k_sum_partials<<<1, 1024, 0, s>>>(partial, (int)blocks, out);
        return;
    }
    NormLaunch L = norm_launch(d, n, red_only && !sigma_out);
    if (sigma_out) {
        if (d == 3)
            k_resnorm<3, true, false><<<L.grid, L.block, 0, s>>>(u, q, partial, n, sigma_out);
        else
            k_resnorm<2, true, false><<<L.grid, L.block, 0, s>>>(u, q, partial, n, sigma_out);
    } else if (red_only) {
        if (d == 3)
            k_resnorm<3, false, true><<<L.grid, L.block, 0, s>>>(u, q, partial, n, nullptr);
        else
            k_resnorm<2, false, true><<<L.grid, L.block, 0, s>>>(u, q, partial, n, nullptr);
    } else {
        if (d == 3)
            k_resnorm<3, false, false><<<L.grid, L.block, 0, s>>>(u, q, partial, n, nullptr);
        else
            k_resnorm<2, false, false><<<L.grid, L.block, 0, s>>>(u, q, partial, n, nullptr);
    }
    k_sum_partials<<<1, 1024, 0, s>>>(partial, (int)L.grid.x, out);
}

}  // namespace fp64
}  // namespace gmg
