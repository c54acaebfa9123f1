// Mixed-precision form: V-cycles in FP32, in BF16 storage with FP32
// arithmetic, or in double-float arithmetic (df.cuh), inside FP64 iterative
// refinement.  FP64 stays on the GPU for
// the outer residual (and its norm, the stopping test) and the solution
// update; the inner cycles solve A'e = b - A'u approximately from e = 0.
//
// In the scaled variables the inner right-hand side is the outer scaled
// residual itself: A'e = b - A'u  <=>  e = sigma + c * (sum of e's
// neighbours) at the fixed point, so q_inner = sigma rounded to the storage
// type.
#include "level_kernels.cuh"

namespace gmg {

namespace lk {
#define GMG_INSTANTIATE(T)                                                                      \
    template void rb_half<T>(int, const Lay&, T*, const T*, int, cudaStream_t, bool);           \
    template void wj_sweep<T>(int, const Lay&, const T*, T*, const T*, double, cudaStream_t);   \
    template void residual<T>(int, const Lay&, const T*, const T*, T*, bool, cudaStream_t,      \
                              bool);                                                            \
    template void restrict_fw<T>(int, const Lay&, const Lay&, const T*, T*, T*, bool, bool,     \
                                 cudaStream_t);                                                 \
    template void prolong_add<T>(int, const Lay&, const Lay&, const T*, T*, cudaStream_t, bool);
GMG_INSTANTIATE(float)
GMG_INSTANTIATE(__nv_bfloat16)
GMG_INSTANTIATE(df32)
#undef GMG_INSTANTIATE
}  // namespace lk

namespace mixed {
namespace {

using lk::sy_of;
using lk::sz_of;

constexpr int kThreads = 256;

// sigma = q + c * sum - u in FP64 on every interior node (in 3D with 1/6
// as a double-double: the outer residual of the full iterate must not carry
// the bias of fl(1/6), lk::gs_value), stored to the inner right-hand side in
// T (layout `in`); partial sums of sigma^2 as in the FP64 norm.
// e_init (may be NULL): also the inner iterate after the first red half
// sweep from e = 0 -- sigma on the red nodes (q_in + c * 0), 0 on the black
// ones -- so that the first inner cycle starts with its black half sweep.
// resid (double-float inner storage only; may be NULL): on the black nodes
// the part of sigma the double-float value of q_in leaves out (about 2^-49
// of sigma; see k_black_exact_update).
template <typename T>
__device__ inline void store_inner(T* __restrict__ q_in, T* __restrict__ e_init, int64_t idx,
                                   double sig, bool red, float* __restrict__ resid) {
    using N = lk::Num<T>;
    using C = typename N::C;
    const T s = N::st(C(sig));
    q_in[idx] = s;
    if (e_init) e_init[idx] = red ? s : N::st(C(0));
    if constexpr (std::is_same<T, df32>::value) {
        if (resid && !red) resid[idx] = (float)((sig - cvt::widen(s.hi)) - cvt::widen(s.lo));
    }
}

// The block's sum of acc (a fixed order: warp shuffles, then the warps in
// turn) into *slot; every thread of the block calls it.
__device__ inline void block_partial(double acc, double* warp_sums, double* slot) {
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if ((t & 31) == 0) warp_sums[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += warp_sums[w];
        *slot = s;
    }
    __syncthreads();
}

// sigma of the iterate u = +0.0 everywhere: q + 0.0, the stencil's value bit
// for bit (every product with a +0 sum is +0, and q + (+0) turns a -0 q into
// +0 as the stencil's adds do).  Rows of the interior over the CTAs' thread
// rows; the stores and sums are those of the stencil path.
template <int DIM, bool SPLIT, typename T>
__device__ inline void zero_iterate_sigma(const double* __restrict__ q, T* __restrict__ q_in,
                                          T* __restrict__ e_init, const Lay& in,
                                          float* __restrict__ resid, bool qsum, double& acc,
                                          float& accq) {
    const int n = in.n;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t rows = DIM == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.y + ty; r < rows;
         r += (int64_t)gridDim.x * blockDim.y) {
        const int j = (int)(r % (n - 1)) + 1;
        const int k = DIM == 3 ? (int)(r / (n - 1)) + 1 : 0;
        const int64_t row = k * sz + j * sy;
        const int64_t row_in = k * in.sz + j * in.sy;
        for (int i = 1 + tx; i < n; i += blockDim.x) {
            const double sig = q[row + i] + 0.0;
            store_inner(q_in, e_init, row_in + lk::xo<SPLIT>(in, i), sig, ((i + j + k) & 1) == 0,
                        resid);
            acc = fma(sig, sig, acc);
            if (qsum) {
                const float qf = (float)q[row + i];
                accq = fmaf(qf, qf, accq);
            }
        }
    }
}

template <int DIM, bool SPLIT, typename T>
__global__ void __launch_bounds__(kThreads) k_outer_residual(const double* __restrict__ u,
                                                             const double* __restrict__ q,
                                                             T* __restrict__ q_in,
                                                             T* __restrict__ e_init,
                                                             double* __restrict__ partial,
                                                             Lay in, float* __restrict__ resid,
                                                             int* __restrict__ resid_flag,
                                                             double* __restrict__ qpart,
                                                             const int* __restrict__ unz) {
    __shared__ double warp_sums[kThreads / 32];
    const double c = DIM == 3 ? 1.0 / 6.0 : 0.25;
    if (resid_flag && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) *resid_flag = 1;
    const int n = in.n;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t rows = DIM == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    double acc = 0.0;
    float accq = 0.f;
    if (unz && *unz == 0)
        zero_iterate_sigma<DIM, SPLIT>(q, q_in, e_init, in, resid, qpart != nullptr, acc, accq);
    else
    for (int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; r < rows;
         r += (int64_t)gridDim.x * blockDim.y) {
        const int j = (int)(r % (n - 1)) + 1;
        const int k = DIM == 3 ? (int)(r / (n - 1)) + 1 : 0;
        const int64_t row = k * sz + j * sy;
        const int64_t row_in = k * in.sz + j * in.sy;
        for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
            const int64_t p = row + i;
            const double sig = lk::gs_value<DIM, true>(c, lk::nbr_sum<DIM>(u, p, sy, sz), q[p]) - u[p];
            store_inner(q_in, e_init, row_in + lk::xo<SPLIT>(in, i), sig, ((i + j + k) & 1) == 0,
                        resid);
            acc = fma(sig, sig, acc);
            if (qpart) {  // FP32: a threshold test, kept off the FP64 pipe
                const float qf = (float)q[p];
                accq = fmaf(qf, qf, accq);
            }
        }
    }
    block_partial(acc, warp_sums, partial + blockIdx.x);
    if (qpart) block_partial((double)accq, warp_sums, qpart + blockIdx.x);
}

// The same by the diagonal walkers of the FP64 3D sweeps (both colours per
// walker): 6.25 instead of 7 FP64 instructions per node for sigma, the same
// sigma values; a fixed grid strides over the walkers (deterministic sum).
template <bool SPLIT, typename T>
__global__ void __launch_bounds__(256, 4) k_outer_residual3_walk(const double* __restrict__ u,
                                                                 const double* __restrict__ q,
                                                                 T* __restrict__ q_in,
                                                                 T* __restrict__ e_init,
                                                                 double* __restrict__ partial,
                                                                 Lay in, int segs,
                                                                 float* __restrict__ resid,
                                                                 int* __restrict__ resid_flag,
                                                                 double* __restrict__ qpart,
                                                                 const int* __restrict__ unz) {
    __shared__ double warp_sums[kThreads / 32];
    const double c = 1.0 / 6.0;
    const int n = in.n;
    const int64_t walkers = (int64_t)(n - 1) * segs;
    if (resid_flag && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) *resid_flag = 1;
    double acc = 0.0;
    float accq = 0.f;
    if (unz && *unz == 0)
        zero_iterate_sigma<3, SPLIT>(q, q_in, e_init, in, resid, qpart != nullptr, acc, accq);
    else
    for (int64_t w = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; w < walkers;
         w += (int64_t)gridDim.x * blockDim.y)
        for (int color = 0; color < 2; ++color)
            lk::walk_nodes(u, n, color, w, segs, [&](int64_t p, double sum, int i, int j, int k) {
                const double sig = lk::gs_value<3, true>(c, sum, q[p]) - u[p];
                store_inner(q_in, e_init, k * in.sz + j * in.sy + lk::xo<SPLIT>(in, i), sig,
                            color == 0, resid);
                acc = fma(sig, sig, acc);
                if (qpart) {  // FP32: a threshold test, kept off the FP64 pipe
                const float qf = (float)q[p];
                accq = fmaf(qf, qf, accq);
            }
            });
    block_partial(acc, warp_sums, partial + blockIdx.x);
    if (qpart) block_partial((double)accq, warp_sums, qpart + blockIdx.x);
}

// u += e on the interior nodes (e, layout `in`, is zero on the boundary;
// so is u).
template <int DIM, bool SPLIT, typename T>
__global__ void __launch_bounds__(256) k_update(double* __restrict__ u, const T* __restrict__ e,
                                                Lay in) {
    const int n = in.n;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t rows = DIM == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    for (int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; r < rows;
         r += (int64_t)gridDim.x * blockDim.y) {
        const int j = (int)(r % (n - 1)) + 1;
        const int k = DIM == 3 ? (int)(r / (n - 1)) + 1 : 0;
        const int64_t row = k * sz + j * sy;
        const int64_t row_in = k * in.sz + j * in.sy;
        for (int i = 1 + threadIdx.x; i < n; i += blockDim.x)
            u[row + i] += (double)lk::Num<T>::ld(e[row_in + lk::xo<SPLIT>(in, i)]);
    }
}

// Double-float refinement after the inner cycles (red-black): the black
// nodes' last Gauss-Seidel values are formed here, from the red corrections,
// in triple-float (df.cuh, sum_tf / fma_tf) and added to u in FP64, so that
// the black residual of the new u is zero up to FP64 rounding, and the next
// outer residual runs on the red nodes only (k_outer_red).  (Stored as
// double-float, the black correction's own rounding, 2^-47 of it, would stay
// in the black residual for good: the red-only residual never sees it.)
// e = q_in = 0 on the black nodes: the next step's inner iterate after its
// first red half sweep, and its black right-hand side.  Replaces the inner
// cycle's last level-0 black half sweep (it is a function of the red values
// only, so recomputing it after a tail that ran it changes nothing).
// After a full outer residual (the start of a solve) the black right-hand
// side is sigma rounded to a double-float; its remainder (resid, valid while
// *resid_flag is set) is added here, once: left out, it would stay in the
// black residual for the rest of the solve, about 2^-49 of the starting
// residual, which is far larger than the solution when the solve starts from
// a rough iterate.
template <int DIM, bool SPLIT>
__global__ void __launch_bounds__(256) k_black_exact_update(double* __restrict__ u,
                                                            df32* __restrict__ e,
                                                            df32* __restrict__ q_in, Lay in,
                                                            const float* __restrict__ resid,
                                                            const int* __restrict__ resid_flag,
                                                            const int* __restrict__ skip) {
    if (skip && *skip) return;
    const bool add_resid = resid && *resid_flag;
    const int n = in.n;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t rows = DIM == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    for (int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; r < rows;
         r += (int64_t)gridDim.x * blockDim.y) {
        const int j = (int)(r % (n - 1)) + 1;
        const int k = DIM == 3 ? (int)(r / (n - 1)) + 1 : 0;
        const int64_t row = k * sz + j * sy;
        const int64_t row_in = k * in.sz + j * in.sy;
        for (int i = 1 + ((j + k) & 1) + 2 * threadIdx.x; i < n; i += 2 * blockDim.x) {
            const int64_t idx = row_in + lk::xo<SPLIT>(in, i);
            int64_t xm, xp;
            lk::xnb<SPLIT>(in, i, xm, xp);
            tf32 v;
            if constexpr (DIM == 3) {
                const df32 x[6] = {e[idx + xm],    e[idx + xp],    e[idx - in.sy],
                                   e[idx - in.sz], e[idx + in.sy], e[idx + in.sz]};
                v = fma_tf(sum_tf(x), kSixth0, kSixth1, kSixth2, q_in[idx]);
            } else {
                const df32 x[4] = {e[idx + xm], e[idx + xp], e[idx - in.sy], e[idx + in.sy]};
                v = fma_tf(sum_tf(x), 0.25f, 0.f, 0.f, q_in[idx]);
            }
            if (add_resid) v.t2 = rn::add(v.t2, resid[idx]);
            u[row + i] += tf_to_double(v);
            e[idx] = df32(0.f, 0.f);
            q_in[idx] = df32(0.f, 0.f);
        }
    }
}

// The red nodes: u += e, sigma (unbiased 1/(2d)) from the updated neighbours,
// q_in = e = sigma (the next step's first inner red half sweep), partial sums
// of sigma^2 (the stopping-test norm: the black terms are zero to rounding).
template <int DIM, bool SPLIT, typename T>
__global__ void __launch_bounds__(kThreads) k_outer_red(double* __restrict__ u,
                                                        const double* __restrict__ q,
                                                        T* __restrict__ q_in, T* __restrict__ e,
                                                        double* __restrict__ partial, Lay in,
                                                        int* __restrict__ resid_flag,
                                                        const int* __restrict__ skip) {
    using N = lk::Num<T>;
    __shared__ double warp_sums[kThreads / 32];
    if (skip && *skip) return;  // uniform over the grid: before any barrier
    if (resid_flag && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) *resid_flag = 0;
    const double c = DIM == 3 ? 1.0 / 6.0 : 0.25;
    const int n = in.n;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t rows = DIM == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    double acc = 0.0;
    df32 acc2(0.f, 0.f);  // sigma^2 summed in double-float (2^-47 relative)
    for (int64_t r = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; r < rows;
         r += (int64_t)gridDim.x * blockDim.y) {
        const int j = (int)(r % (n - 1)) + 1;
        const int k = DIM == 3 ? (int)(r / (n - 1)) + 1 : 0;
        const int64_t row = k * sz + j * sy;
        const int64_t row_in = k * in.sz + j * in.sy;
        for (int i = 1 + ((1 + j + k) & 1) + 2 * threadIdx.x; i < n; i += 2 * blockDim.x) {
            const int64_t p = row + i;
            const int64_t idx = row_in + lk::xo<SPLIT>(in, i);
            const double un = u[p] + (double)N::ld(e[idx]);
            u[p] = un;
            const double sig = lk::gs_value<DIM, true>(c, lk::nbr_sum<DIM>(u, p, sy, sz), q[p]) - un;
            const T st = N::st(typename N::C(sig));
            q_in[idx] = st;
            e[idx] = st;
            acc2 = acc2 + st * st;  // on the FP32 pipe: the FP64 pipe bounds this kernel
        }
    }
    acc = (double)acc2;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if ((t & 31) == 0) warp_sums[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double sum = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) sum += warp_sums[w];
        partial[blockIdx.x] = sum;
    }
}

// The same by the diagonal walkers (red nodes; the black neighbours are read
// through uc, never written here; each red node is read and written through
// u by its own thread only).
template <bool SPLIT, typename T>
__global__ void __launch_bounds__(256, 4) k_outer_red3_walk(double* __restrict__ u,
                                                            const double* __restrict__ uc,
                                                            const double* __restrict__ q,
                                                            T* __restrict__ q_in,
                                                            T* __restrict__ e,
                                                            double* __restrict__ partial, Lay in,
                                                            int segs, int* __restrict__ resid_flag,
                                                            const int* __restrict__ skip) {
    using N = lk::Num<T>;
    __shared__ double warp_sums[kThreads / 32];
    if (skip && *skip) return;  // uniform over the grid: before any barrier
    if (resid_flag && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) *resid_flag = 0;
    const double c = 1.0 / 6.0;
    const int n = in.n;
    const int64_t walkers = (int64_t)(n - 1) * segs;
    double acc = 0.0;
    df32 acc2(0.f, 0.f);  // sigma^2 summed in double-float (2^-47 relative)
    for (int64_t w = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; w < walkers;
         w += (int64_t)gridDim.x * blockDim.y)
        lk::walk_nodes(uc, n, 0, w, segs, [&](int64_t p, double sum, int i, int j, int k) {
            const int64_t idx = k * in.sz + j * in.sy + lk::xo<SPLIT>(in, i);
            const double un = u[p] + (double)N::ld(e[idx]);
            u[p] = un;
            const double sig = lk::gs_value<3, true>(c, sum, q[p]) - un;
            const T st = N::st(typename N::C(sig));
            q_in[idx] = st;
            e[idx] = st;
            acc2 = acc2 + st * st;  // on the FP32 pipe: the FP64 pipe bounds this kernel
        });
    acc = (double)acc2;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if ((t & 31) == 0) warp_sums[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double sum = 0.0;
        for (int ww = 0; ww < kThreads / 32; ++ww) sum += warp_sums[ww];
        partial[blockIdx.x] = sum;
    }
}

// fp64::k_sum_partials (the same order) while *skip is zero.
__global__ void __launch_bounds__(1024) k_sum_partials_skip(const double* __restrict__ partial,
                                                            int count, double* __restrict__ out,
                                                            const int* __restrict__ skip) {
    __shared__ double warp_sums[32];
    if (skip && *skip) return;
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partial[i];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += warp_sums[w];
        out[0] = t;
    }
}

}  // namespace

template <typename T>
void outer_red_update(int d, const Lay& in, double* u, const double* q, T* q_in, T* e,
                      double* partial, double* out, cudaStream_t s, const float* resid,
                      int* resid_flag, const int* skip) {
    static_assert(std::is_same<T, df32>::value, "the red-only outer residual is double-float");
    const int n = in.n;
    int bx = 32;
    while (bx < n / 2 && bx < 128) bx *= 2;
    const dim3 block(bx, kThreads / bx, 1);
    const int64_t rows = d == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    const int ublocks = (int)std::min<int64_t>((rows + block.y - 1) / block.y, 152 * 16);
    if (d == 3) {
        if (in.he)
            k_black_exact_update<3, true><<<ublocks, block, 0, s>>>(u, e, q_in, in, resid,
                                                                   resid_flag, skip);
        else
            k_black_exact_update<3, false><<<ublocks, block, 0, s>>>(u, e, q_in, in, resid,
                                                                   resid_flag, skip);
    } else {
        if (in.he)
            k_black_exact_update<2, true><<<ublocks, block, 0, s>>>(u, e, q_in, in, resid,
                                                                   resid_flag, skip);
        else
            k_black_exact_update<2, false><<<ublocks, block, 0, s>>>(u, e, q_in, in, resid,
                                                                   resid_flag, skip);
    }
    if (lk::walk_applies(d, n, sizeof(double))) {
        const lk::WalkLaunch W = lk::walk_launch(n);
        const int blocks = (int)std::min<int64_t>(W.blocks, outer_partials(d, n));
        if (in.he)
            k_outer_red3_walk<true, T><<<blocks, W.block, 0, s>>>(u, u, q, q_in, e, partial, in,
                                                                  W.segs, resid_flag, skip);
        else
            k_outer_red3_walk<false, T><<<blocks, W.block, 0, s>>>(u, u, q, q_in, e, partial, in,
                                                                   W.segs, resid_flag, skip);
        k_sum_partials_skip<<<1, 1024, 0, s>>>(partial, blocks, out, skip);
        return;
    }
    const int blocks = outer_partials(d, n);
    if (d == 3) {
        if (in.he)
            k_outer_red<3, true, T><<<blocks, block, 0, s>>>(u, q, q_in, e, partial, in,
                                                          resid_flag, skip);
        else
            k_outer_red<3, false, T><<<blocks, block, 0, s>>>(u, q, q_in, e, partial, in,
                                                          resid_flag, skip);
    } else {
        if (in.he)
            k_outer_red<2, true, T><<<blocks, block, 0, s>>>(u, q, q_in, e, partial, in,
                                                          resid_flag, skip);
        else
            k_outer_red<2, false, T><<<blocks, block, 0, s>>>(u, q, q_in, e, partial, in,
                                                          resid_flag, skip);
    }
    k_sum_partials_skip<<<1, 1024, 0, s>>>(partial, blocks, out, skip);
}

int outer_partials(int d, int n) {
    int bx = 32;
    while (bx < n && bx < 128) bx *= 2;
    const int by = kThreads / bx;
    const int64_t rows = d == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    return (int)std::min<int64_t>((rows + by - 1) / by, 152 * 8);
}

template <typename T>
void outer_residual(int d, const Lay& in, const double* u, const double* q, T* q_in,
                    double* partial, double* out, cudaStream_t s, T* e_init, float* resid,
                    int* resid_flag, double* qnorm_out, const int* unz) {
    const int n = in.n;
    const int np = outer_partials(d, n);  // the q partials follow the sigma partials
    double* qpart = qnorm_out ? partial + np : nullptr;
    if (lk::walk_applies(d, n, sizeof(double))) {
        const lk::WalkLaunch W = lk::walk_launch(n);
        const int blocks = (int)std::min<int64_t>(W.blocks, outer_partials(d, n));
        if (in.he)
            k_outer_residual3_walk<true, T><<<blocks, W.block, 0, s>>>(u, q, q_in, e_init, partial, in,
                                                                     W.segs, resid, resid_flag, qpart, unz);
        else
            k_outer_residual3_walk<false, T><<<blocks, W.block, 0, s>>>(u, q, q_in, e_init, partial, in,
                                                                      W.segs, resid, resid_flag, qpart, unz);
        fp64::k_sum_partials<<<1, 1024, 0, s>>>(partial, blocks, out);
        if (qpart) fp64::k_sum_partials<<<1, 1024, 0, s>>>(qpart, blocks, qnorm_out);
        return;
    }
    int bx = 32;
    while (bx < n && bx < 128) bx *= 2;
    dim3 block(bx, kThreads / bx, 1);
    const int blocks = outer_partials(d, n);
    if (d == 3) {
        if (in.he)
            k_outer_residual<3, true, T><<<blocks, block, 0, s>>>(u, q, q_in, e_init, partial, in,
                                                                   resid, resid_flag, qpart, unz);
        else
            k_outer_residual<3, false, T><<<blocks, block, 0, s>>>(u, q, q_in, e_init, partial, in,
                                                                   resid, resid_flag, qpart, unz);
    } else {
        if (in.he)
            k_outer_residual<2, true, T><<<blocks, block, 0, s>>>(u, q, q_in, e_init, partial, in,
                                                                   resid, resid_flag, qpart, unz);
        else
            k_outer_residual<2, false, T><<<blocks, block, 0, s>>>(u, q, q_in, e_init, partial, in,
                                                                   resid, resid_flag, qpart, unz);
    }
    fp64::k_sum_partials<<<1, 1024, 0, s>>>(partial, blocks, out);
    if (qpart) fp64::k_sum_partials<<<1, 1024, 0, s>>>(qpart, blocks, qnorm_out);
}

template <typename T>
void update(int d, const Lay& in, double* u, const T* e, cudaStream_t s) {
    const int n = in.n;
    int bx = 32;
    while (bx < n && bx < 128) bx *= 2;
    dim3 block(bx, 256 / bx, 1);
    const int64_t rows = d == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    const int blocks = (int)std::min<int64_t>((rows + block.y - 1) / block.y, 152 * 16);
    if (d == 3) {
        if (in.he)
            k_update<3, true, T><<<blocks, block, 0, s>>>(u, e, in);
        else
            k_update<3, false, T><<<blocks, block, 0, s>>>(u, e, in);
    } else {
        if (in.he)
            k_update<2, true, T><<<blocks, block, 0, s>>>(u, e, in);
        else
            k_update<2, false, T><<<blocks, block, 0, s>>>(u, e, in);
    }
}

template void outer_residual<float>(int, const Lay&, const double*, const double*, float*,
                                    double*, double*, cudaStream_t, float*, float*, int*,
                                    double*, const int*);
template void outer_residual<__nv_bfloat16>(int, const Lay&, const double*, const double*,
                                            __nv_bfloat16*, double*, double*, cudaStream_t,
                                            __nv_bfloat16*, float*, int*, double*, const int*);
template void outer_residual<df32>(int, const Lay&, const double*, const double*, df32*, double*,
                                   double*, cudaStream_t, df32*, float*, int*, double*,
                                   const int*);
template void outer_red_update<df32>(int, const Lay&, double*, const double*, df32*, df32*,
                                     double*, double*, cudaStream_t, const float*, int*,
                                     const int*);

// Work items of the colour-split double-float kernels on level `in`: groups
// of lk::kDfVec nodes of one colour in a row, rows (j, k).
struct DfItems {
    lk::FastDiv fG, fm;
    uint32_t items;
};
DfItems df_items(int d, const Lay& in) {
    const int n = in.n;
    constexpr int V = lk::kDfVec;
    const int G = (n / 2 + 1 + V - 1) / V;
    const int64_t items = (int64_t)G * (d == 3 ? (int64_t)(n - 1) * (n - 1) : n - 1);
    return {lk::fastdiv_make((uint32_t)G), lk::fastdiv_make((uint32_t)(n - 1)), (uint32_t)items};
}

void df_black_half(int d, const Lay& in, df32* e, const df32* q_in, const int* skip,
                   cudaStream_t s) {
    constexpr int V = lk::kDfVec;
    const DfItems I = df_items(d, in);
    const unsigned blocks = (I.items + 255) / 256;
    if (d == 3)
        lk::k_rb_half_vec_df<3, V><<<blocks, 256, 0, s>>>(e, q_in, in, 1, I.fG, I.fm, I.items,
                                                          nullptr, skip);
    else
        lk::k_rb_half_vec_df<2, V><<<blocks, 256, 0, s>>>(e, q_in, in, 1, I.fG, I.fm, I.items,
                                                          nullptr, skip);
}

int df_red_ahead(int d, const Lay& in, df32* e, const df32* q_in, df32* r, double* partial,
                 const int* skip, cudaStream_t s) {
    constexpr int V = lk::kDfVec;
    const DfItems I = df_items(d, in);
    const int blocks = (int)std::min<int64_t>(((int64_t)I.items + 255) / 256,
                                              std::min(152 * lk::kAheadCtasPerSm,
                                                       outer_partials(d, in.n)));
    if (d == 3)
        lk::k_red_ahead_df<3, V><<<blocks, 256, 0, s>>>(e, q_in, r, in, I.fG, I.fm, I.items,
                                                        partial, skip);
    else
        lk::k_red_ahead_df<2, V><<<blocks, 256, 0, s>>>(e, q_in, r, in, I.fG, I.fm, I.items,
                                                        partial, skip);
    return blocks;
}

void df_red_restore(int d, const Lay& in, df32* e, const df32* r, const int* flag,
                    cudaStream_t s) {
    constexpr int V = lk::kDfVec;
    const DfItems I = df_items(d, in);
    const unsigned blocks = std::min<unsigned>((I.items + 255) / 256, 152 * 8);
    if (d == 3)
        lk::k_red_restore_df<3, V><<<blocks, 256, 0, s>>>(e, r, in, I.fG, I.fm, I.items, flag);
    else
        lk::k_red_restore_df<2, V><<<blocks, 256, 0, s>>>(e, r, in, I.fG, I.fm, I.items, flag);
}
template void update<float>(int, const Lay&, double*, const float*, cudaStream_t);
template void update<df32>(int, const Lay&, double*, const df32*, cudaStream_t);
template void update<__nv_bfloat16>(int, const Lay&, double*, const __nv_bfloat16*, cudaStream_t);

}  // namespace mixed
}  // namespace gmg
