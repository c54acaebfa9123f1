// Learned smoother: a per-level convolutional smoother u <- u + N(sigma),
// sigma = (b - A'u)/(2d), N = conv2(ReLU(conv1(sigma))) with conv1: 1 -> 8
// channels and conv2: 8 -> 1 channel, 3^d taps, zero padding at the
// Dirichlet boundary, no biases, BF16 weights with FP32 accumulation.
//
// Training minimises the measured two-grid error contraction
//     L = ||S(CG(S(e0)))||^2 / ||e0||^2,  S e = e - N(A'e/(2d)),
//     CG e = e - P A_c'^{-1} 4 FW(A'e),
// over error samples e0 drawn from plain red-black V(1,1) cycles applied to
// seeded white noise, with this file's forward and backward kernels and an
// Adam step, all on the GPU.  The coarse system inside the loss is solved by
// red-black V(2,2) cycles run to round-off.
//
// Weight layout (host and device): 2 x 8 x T floats, W1[c][t] then W2[c][t],
// tap t = (c3+1)*9 + (b+1)*3 + (a+1) for the offset (a, b, c3) (x fastest);
// T = 27 in 3D, 9 in 2D.
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gmg_internal.cuh"
#include "level_kernels.cuh"

namespace gmg {
namespace learned {
namespace {

constexpr int H = 8;  // hidden channels

using lk::sy_of;
using lk::sz_of;

template <int DIM>
constexpr int taps() {
    return DIM == 3 ? 27 : 9;
}

template <int DIM>
__device__ inline int64_t tap_offset(int t, int64_t sy, int64_t sz) {
    const int a = t % 3 - 1, b = (t / 3) % 3 - 1, c = DIM == 3 ? t / 9 - 1 : 0;
    return a + b * sy + c * sz;
}

template <int DIM>
__device__ inline void load_weights(const float* W, float* ws) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y;
    for (int i = tid; i < 2 * H * taps<DIM>(); i += nt) ws[i] = W[i];
    __syncthreads();
}

// z_c(p) = sum_t W1[c][t] x(p + o_t) on interior nodes (x is zero on the
// boundary; z's boundary entries are never written and stay zero)
template <int DIM, typename TI>
__global__ void __launch_bounds__(256) k_conv1(const TI* __restrict__ x, float* __restrict__ z,
                                               int n, int64_t zs, const float* __restrict__ W) {
    constexpr int T = taps<DIM>();
    __shared__ float ws[2 * H * T];
    load_weights<DIM>(W, ws);
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    if (j >= n) return;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t row = k * sz + j * sy;
    for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
        const int64_t p = row + i;
        float xv[T];
#pragma unroll
        for (int t = 0; t < T; ++t) xv[t] = (float)x[p + tap_offset<DIM>(t, sy, sz)];
#pragma unroll
        for (int c = 0; c < H; ++c) {
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t < T; ++t) acc = fmaf(ws[c * T + t], xv[t], acc);
            z[c * zs + p] = acc;
        }
    }
}

// y(p) = sum_c sum_t W2[c][t] relu(z_c(p + o_t)); mode 0: out = y,
// 1: out += y, 2: out -= y (out in FP64)
template <int DIM, int MODE>
__global__ void __launch_bounds__(256) k_conv2(const float* __restrict__ z, double* __restrict__ out,
                                               int n, int64_t zs, const float* __restrict__ W) {
    constexpr int T = taps<DIM>();
    __shared__ float ws[2 * H * T];
    load_weights<DIM>(W, ws);
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    if (j >= n) return;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t row = k * sz + j * sy;
    const float* w2 = ws + H * T;
    for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
        const int64_t p = row + i;
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < H; ++c)
#pragma unroll
            for (int t = 0; t < T; ++t)
                acc = fmaf(w2[c * T + t], fmaxf(z[c * zs + p + tap_offset<DIM>(t, sy, sz)], 0.f), acc);
        if (MODE == 0)
            out[p] = (double)acc;
        else if (MODE == 1)
            out[p] += (double)acc;
        else
            out[p] -= (double)acc;
    }
}

// gz_c(p) = [z_c(p) > 0] * sum_t W2[c][t] gy(p - o_t)
template <int DIM>
__global__ void __launch_bounds__(256) k_conv2_bwd(const double* __restrict__ gy,
                                                   const float* __restrict__ z,
                                                   float* __restrict__ gz, int n, int64_t zs,
                                                   const float* __restrict__ W) {
    constexpr int T = taps<DIM>();
    __shared__ float ws[2 * H * T];
    load_weights<DIM>(W, ws);
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    if (j >= n) return;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t row = k * sz + j * sy;
    const float* w2 = ws + H * T;
    for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
        const int64_t p = row + i;
        float gv[T];
#pragma unroll
        for (int t = 0; t < T; ++t) gv[t] = (float)gy[p - tap_offset<DIM>(t, sy, sz)];
#pragma unroll
        for (int c = 0; c < H; ++c) {
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t < T; ++t) acc = fmaf(w2[c * T + t], gv[t], acc);
            gz[c * zs + p] = z[c * zs + p] > 0.f ? acc : 0.f;
        }
    }
}

// gx(p) = sum_c sum_t W1[c][t] gz_c(p - o_t)
template <int DIM>
__global__ void __launch_bounds__(256) k_conv1_bwd(const float* __restrict__ gz,
                                                   double* __restrict__ gx, int n, int64_t zs,
                                                   const float* __restrict__ W) {
    constexpr int T = taps<DIM>();
    __shared__ float ws[2 * H * T];
    load_weights<DIM>(W, ws);
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    if (j >= n) return;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t row = k * sz + j * sy;
    for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
        const int64_t p = row + i;
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < H; ++c)
#pragma unroll
            for (int t = 0; t < T; ++t)
                acc = fmaf(ws[c * T + t], gz[c * zs + p - tap_offset<DIM>(t, sy, sz)], acc);
        gx[p] = (double)acc;
    }
}

__device__ inline int64_t interior_node(int d, int n, int64_t idx) {
    const int m = n - 1;
    const int i = (int)(idx % m) + 1;
    const int64_t t = idx / m;
    const int j = (int)(t % m) + 1;
    const int k = d == 3 ? (int)(t / m) + 1 : 0;
    return ((int64_t)k * (n + 1) + j) * (n + 1) + i;
}

// Weight-gradient partials over `rpb` consecutive interior rows, one thread
// per (channel, tap):  KIND 1: sum_p gz_c(p) x(p + o_t);  KIND 2: sum_p gy(p)
// relu(z_c(p + o_t)).  FP32 within the block, one double per (block, c, t).
template <int DIM, int KIND>
__global__ void __launch_bounds__(256) k_wgrad(const double* __restrict__ dense,
                                               const float* __restrict__ chan, int n, int64_t zs,
                                               int rpb, double* __restrict__ partial) {
    constexpr int T = taps<DIM>();
    const int ct = threadIdx.x;
    if (ct >= H * T) return;
    const int c = ct / T, t = ct % T;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t off = tap_offset<DIM>(t, sy, sz);
    const int64_t rows = DIM == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < rows ? r0 + rpb : rows;
    const float* ch = chan + c * zs;
    float acc = 0.f;
    for (int64_t r = r0; r < r1; ++r) {
        const int j = (int)(r % (n - 1)) + 1;
        const int k = DIM == 3 ? (int)(r / (n - 1)) + 1 : 0;
        const int64_t row = k * sz + j * sy;
        for (int i = 1; i < n; ++i) {
            const int64_t p = row + i;
            if (KIND == 1)
                acc = fmaf(ch[p], (float)dense[p + off], acc);
            else
                acc = fmaf((float)dense[p], fmaxf(ch[p + off], 0.f), acc);
        }
    }
    partial[(int64_t)blockIdx.x * (2 * H * T) + (KIND == 1 ? 0 : H * T) + ct] = (double)acc;
}

// grad[i] += scale * sum_b partial[b][i] (fixed order) for the KIND's half
__global__ void k_wgrad_reduce(const double* __restrict__ partial, int blocks, int half, int base,
                               const double* __restrict__ scale_dev, double sign,
                               double* __restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= half) return;
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s += partial[(int64_t)b * 2 * half + base + i];
    grad[base + i] += sign * scale_dev[0] * s;
}

// s = A'e/(2d) = e - c * (sum of neighbours) on interior nodes
template <int DIM>
__global__ void __launch_bounds__(256) k_scaled_apply(const double* __restrict__ e,
                                                      double* __restrict__ s, int n) {
    const double c = DIM == 3 ? 1.0 / 6.0 : 0.25;
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    if (j >= n) return;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t row = k * sz + j * sy;
    for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
        const int64_t p = row + i;
        s[p] = e[p] - c * lk::nbr_sum<DIM>(e, p, sy, sz);
    }
}

// y = a * x + y over all nodes (a from a device scalar times a constant)
__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, int64_t nodes,
                       double a, const double* __restrict__ a_dev) {
    const double f = a_dev ? a * a_dev[0] : a;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nodes;
         p += (int64_t)gridDim.x * blockDim.x)
        y[p] = fma(f, x[p], y[p]);
}

// out[0] = sum x^2 (deterministic: fixed grid, fixed trees)
__global__ void __launch_bounds__(256) k_sumsq_partial(const double* __restrict__ x, int64_t nodes,
                                                       double* __restrict__ partial) {
    __shared__ double ws[8];
    double acc = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nodes;
         p += (int64_t)gridDim.x * blockDim.x)
        acc = fma(x[p], x[p], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += ws[w];
        partial[blockIdx.x] = s;
    }
}

// scalars: out[0] = op(partials) ; op 0: sum ; 1: 2 / sum (gradient scale) ;
// 2: acc[0] += sum * inv_den[0] / batch (loss)
__global__ void k_scalar(const double* __restrict__ partial, int count, int op, double batch,
                         const double* __restrict__ inv_den, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < count; ++i) s += partial[i];
    if (op == 0) out[0] = s;
    if (op == 1) out[0] = 2.0 / s;
    if (op == 2) out[0] += s * inv_den[0] * 0.5 / batch;
}

// seeded white noise U[-1,1) on interior nodes (splitmix64 of seed and index)
__global__ void k_white_noise(double* __restrict__ e, int d, int n, uint64_t seed) {
    const int64_t m = n - 1;
    const int64_t total = d == 3 ? m * m * m : m * m;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(idx + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        e[interior_node(d, n, idx)] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
}

// Adam on the master weights; the working copy is their BF16 rounding.
__global__ void k_adam(float* __restrict__ master, float* __restrict__ work,
                       const double* __restrict__ grad, double* __restrict__ m1,
                       double* __restrict__ m2, int count, int step, double lr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double b1 = 0.9, b2 = 0.999, eps = 1e-12;
    const double g = grad[i];
    m1[i] = b1 * m1[i] + (1 - b1) * g;
    m2[i] = b2 * m2[i] + (1 - b2) * g * g;
    const double mh = m1[i] / (1 - pow(b1, step));
    const double vh = m2[i] / (1 - pow(b2, step));
    master[i] = (float)((double)master[i] - lr * mh / (sqrt(vh) + eps));
    work[i] = __bfloat162float(__float2bfloat16_rn(master[i]));
}

__global__ void k_round_bf16(const float* __restrict__ in, float* __restrict__ out, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = __bfloat162float(__float2bfloat16_rn(in[i]));
}

lk::RowLaunch rows(int d, int n) { return lk::row_launch(d, n, n); }

int64_t nodes_of(int d, int n) {
    const int64_t m = n + 1;
    return d == 3 ? m * m * m : m * m;
}
int64_t interior_of(int d, int n) {
    const int64_t m = n - 1;
    return d == 3 ? m * m * m : m * m;
}
int flat_blocks(int64_t nodes) { return (int)std::min<int64_t>((nodes + 255) / 256, 152 * 8); }

}  // namespace

// --------------------------------------------------------------- launchers

void conv1(int d, int n, const double* x, float* z, const float* W, cudaStream_t s) {
    auto L = rows(d, n);
    const int64_t zs = nodes_of(d, n);
    if (d == 3)
        k_conv1<3, double><<<L.grid, L.block, 0, s>>>(x, z, n, zs, W);
    else
        k_conv1<2, double><<<L.grid, L.block, 0, s>>>(x, z, n, zs, W);
}

void conv2(int d, int n, const float* z, double* out, int mode, const float* W, cudaStream_t s) {
    auto L = rows(d, n);
    const int64_t zs = nodes_of(d, n);
    if (d == 3) {
        if (mode == 0) k_conv2<3, 0><<<L.grid, L.block, 0, s>>>(z, out, n, zs, W);
        if (mode == 1) k_conv2<3, 1><<<L.grid, L.block, 0, s>>>(z, out, n, zs, W);
        if (mode == 2) k_conv2<3, 2><<<L.grid, L.block, 0, s>>>(z, out, n, zs, W);
    } else {
        if (mode == 0) k_conv2<2, 0><<<L.grid, L.block, 0, s>>>(z, out, n, zs, W);
        if (mode == 1) k_conv2<2, 1><<<L.grid, L.block, 0, s>>>(z, out, n, zs, W);
        if (mode == 2) k_conv2<2, 2><<<L.grid, L.block, 0, s>>>(z, out, n, zs, W);
    }
}

void upload_weights(int d, const float* host, float* dev, float* scratch, cudaStream_t s) {
    const int W = 2 * H * (d == 3 ? 27 : 9);
    cudaMemcpyAsync(scratch, host, sizeof(float) * W, cudaMemcpyHostToDevice, s);
    k_round_bf16<<<(W + 255) / 256, 256, 0, s>>>(scratch, dev, W);
}

namespace {

void conv2_bwd(int d, int n, const double* gy, const float* z, float* gz, const float* W,
               cudaStream_t s) {
    auto L = rows(d, n);
    const int64_t zs = nodes_of(d, n);
    if (d == 3)
        k_conv2_bwd<3><<<L.grid, L.block, 0, s>>>(gy, z, gz, n, zs, W);
    else
        k_conv2_bwd<2><<<L.grid, L.block, 0, s>>>(gy, z, gz, n, zs, W);
}

void conv1_bwd(int d, int n, const float* gz, double* gx, const float* W, cudaStream_t s) {
    auto L = rows(d, n);
    const int64_t zs = nodes_of(d, n);
    if (d == 3)
        k_conv1_bwd<3><<<L.grid, L.block, 0, s>>>(gz, gx, n, zs, W);
    else
        k_conv1_bwd<2><<<L.grid, L.block, 0, s>>>(gz, gx, n, zs, W);
}

int wgrad_rpb(int n) { return std::max(1, 2048 / (n - 1)); }
int wgrad_blocks(int d, int n) {
    const int64_t rows = d == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    return (int)((rows + wgrad_rpb(n) - 1) / wgrad_rpb(n));
}

// grad += sign * scale * (dW1 from (x, gz), dW2 from (gy, z))
void wgrad(int d, int n, const double* x, const float* gz, const double* gy, const float* z,
           double* partial, const double* scale_dev, double sign, double* grad, cudaStream_t s) {
    const int T = d == 3 ? 27 : 9;
    const int blocks = wgrad_blocks(d, n), rpb = wgrad_rpb(n);
    const int64_t zs = nodes_of(d, n);
    if (d == 3) {
        k_wgrad<3, 1><<<blocks, 256, 0, s>>>(x, gz, n, zs, rpb, partial);
        k_wgrad<3, 2><<<blocks, 256, 0, s>>>(gy, z, n, zs, rpb, partial);
    } else {
        k_wgrad<2, 1><<<blocks, 256, 0, s>>>(x, gz, n, zs, rpb, partial);
        k_wgrad<2, 2><<<blocks, 256, 0, s>>>(gy, z, n, zs, rpb, partial);
    }
    const int half = H * T;
    k_wgrad_reduce<<<1, 256, 0, s>>>(partial, blocks, half, 0, scale_dev, sign, grad);
    k_wgrad_reduce<<<1, 256, 0, s>>>(partial, blocks, half, half, scale_dev, sign, grad);
}

void scaled_apply(int d, int n, const double* e, double* out, cudaStream_t s) {
    auto L = rows(d, n);
    if (d == 3)
        k_scaled_apply<3><<<L.grid, L.block, 0, s>>>(e, out, n);
    else
        k_scaled_apply<2><<<L.grid, L.block, 0, s>>>(e, out, n);
}

// Work buffers of a training / loss evaluation on one grid.
struct Trainer {
    int d = 3, n = 0, T = 27, coarse_cycles = 30, pair_cycles = 1;
    cudaStream_t s = nullptr;
    int64_t nodes = 0;
    double *e0 = nullptr, *e1 = nullptr, *e2 = nullptr, *e3 = nullptr;  // error states
    double *s1 = nullptr, *s2 = nullptr, *s3 = nullptr;                 // A'e/(2d)
    double *g = nullptr, *gx = nullptr, *w = nullptr;
    float *z1 = nullptr, *z3 = nullptr, *gz = nullptr;
    double *partial = nullptr, *wpart = nullptr, *scal = nullptr;  // scal: [0] 1/||e0||^2*2, [1] loss
    double* grad = nullptr;
    std::vector<Level<double>> coarse;  // hierarchy of the n/2 grid (coarse solve)
    std::vector<Level<double>> pair;    // hierarchy of the n grid (sample generation)
    std::vector<void*> allocs;

    cudaError_t alloc(void** p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) return e;
        allocs.push_back(*p);
        return cudaMemsetAsync(*p, 0, bytes, s);
    }
    void release() {
        for (void* p : allocs) cudaFree(p);
        allocs.clear();
    }
    cudaError_t hierarchy(std::vector<Level<double>>& lv, int nn) {
        int L = 0;
        while ((2 << L) <= nn) ++L;
        lv.resize(L);
        for (int l = 0; l < L; ++l) {
            lv[l].n = nn >> l;
            lv[l].nodes = nodes_of(d, lv[l].n);
            const size_t b = sizeof(double) * lv[l].nodes;
            cudaError_t e;
            if ((e = alloc((void**)&lv[l].u[0], b)) != cudaSuccess) return e;
            if ((e = alloc((void**)&lv[l].q, b)) != cudaSuccess) return e;
            if (l + 1 < L && (e = alloc((void**)&lv[l].r, b)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    cudaError_t init(int d_, int n_, int cc, int pc, cudaStream_t st) {
        d = d_;
        n = n_;
        T = d == 3 ? 27 : 9;
        coarse_cycles = cc;
        pair_cycles = pc;
        s = st;
        nodes = nodes_of(d, n);
        const size_t b = sizeof(double) * nodes, bz = sizeof(float) * nodes * H;
        cudaError_t e = cudaSuccess;
        for (double** p : {&e0, &e1, &e2, &e3, &s1, &s2, &s3, &g, &gx, &w})
            if (e == cudaSuccess) e = alloc((void**)p, b);
        for (float** p : {&z1, &z3, &gz})
            if (e == cudaSuccess) e = alloc((void**)p, bz);
        if (e == cudaSuccess) e = alloc((void**)&partial, sizeof(double) * 152 * 8);
        if (e == cudaSuccess)
            e = alloc((void**)&wpart, sizeof(double) * wgrad_blocks(d, n) * 2 * H * T);
        if (e == cudaSuccess) e = alloc((void**)&scal, sizeof(double) * 4);
        if (e == cudaSuccess) e = alloc((void**)&grad, sizeof(double) * 2 * H * T);
        if (e == cudaSuccess) e = hierarchy(coarse, n / 2);
        if (e == cudaSuccess) e = hierarchy(pair, n);
        return e;
    }

    // RB-GS V(nu,nu) cycle on hierarchy lv (level-0 iterate lv[0].u[0], rhs lv[0].q)
    void vcycle(std::vector<Level<double>>& lv, int nu) {
        const int L = (int)lv.size();
        for (int l = 0; l + 1 < L; ++l) {
            for (int k = 0; k < nu; ++k)
                for (int c = 0; c < 2; ++c) lk::rb_half<double>(d, lv[l].n, lv[l].u[0], lv[l].q, c, s);
            lk::residual<double>(d, lv[l].n, lv[l].u[0], lv[l].q, lv[l].r, nu > 0, s);
            lk::restrict_fw<double>(d, lv[l].n, lv[l].r, lv[l + 1].q, lv[l + 1].u[0], nu > 0,
                                    lv[l + 1].n == 2, s);
        }
        if (L == 1)
            for (int k = 0; k < nu; ++k)
                for (int c = 0; c < 2; ++c) lk::rb_half<double>(d, lv[0].n, lv[0].u[0], lv[0].q, c, s);
        for (int l = L - 2; l >= 0; --l) {
            lk::prolong_add<double>(d, lv[l + 1].n, lv[l + 1].u[0], lv[l].u[0], s);
            for (int k = 0; k < nu; ++k)
                for (int c = 0; c < 2; ++c) lk::rb_half<double>(d, lv[l].n, lv[l].u[0], lv[l].q, c, s);
        }
    }

    // u_c = (2d) A_c'^{-1} q_c with q_c = 4 FW(src) restricted from src (fine)
    void coarse_solve_of(double* src) {
        Level<double>& C = coarse[0];
        // restrict_fw writes q_c and zeroes u_c (or u_c = q_c on a one-unknown grid)
        lk::restrict_fw<double>(d, n, src, C.q, C.u[0], false, C.n == 2, s);
        if (C.n > 2)
            for (int k = 0; k < coarse_cycles; ++k) vcycle(coarse, 2);
    }

    // e_out = e_in - P u_c (error-form coarse-grid correction), s2 = A'e_in/(2d)
    void cgc(const double* e_in, double* e_out) {
        scaled_apply(d, n, e_in, s2, s);
        coarse_solve_of(s2);
        cudaMemcpyAsync(e_out, e_in, sizeof(double) * nodes, cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(w, 0, sizeof(double) * nodes, s);
        lk::prolong_add<double>(d, coarse[0].n, coarse[0].u[0], w, s);
        k_axpy<<<flat_blocks(nodes), 256, 0, s>>>(e_out, w, nodes, -1.0, nullptr);
    }

    // g <- g - (A'/(2d)) P u_c' with u_c' = (2d) A_c'^{-1} 4FW(g)
    void cgc_adjoint(double* gg) {
        coarse_solve_of(gg);
        cudaMemsetAsync(w, 0, sizeof(double) * nodes, s);
        lk::prolong_add<double>(d, coarse[0].n, coarse[0].u[0], w, s);
        scaled_apply(d, n, w, gx, s);
        k_axpy<<<flat_blocks(nodes), 256, 0, s>>>(gg, gx, nodes, -1.0, nullptr);
    }

    // e_out = e_in - N(s_in), s_in = A'e_in/(2d), keeping z
    void smooth(const double* e_in, double* s_in, float* z, double* e_out, const float* W) {
        scaled_apply(d, n, e_in, s_in, s);
        conv1(d, n, s_in, z, W, s);
        cudaMemcpyAsync(e_out, e_in, sizeof(double) * nodes, cudaMemcpyDeviceToDevice, s);
        conv2(d, n, z, e_out, 2, W, s);
    }

    void sumsq(const double* x, int op, double batch) {
        const int blocks = flat_blocks(nodes);
        k_sumsq_partial<<<blocks, 256, 0, s>>>(x, nodes, partial);
        k_scalar<<<1, 32, 0, s>>>(partial, blocks, op, batch, scal, op == 2 ? scal + 1 : scal);
    }

    // loss (accumulated into scal[1] / batch) and, if want_grad, its
    // gradient (accumulated into grad / batch) for the sample in e0
    void loss_grad(const float* W, double batch, bool want_grad) {
        smooth(e0, s1, z1, e1, W);
        cgc(e1, e2);
        smooth(e2, s3, z3, e3, W);
        sumsq(e0, 1, batch);         // scal[0] = 2 / ||e0||^2
        sumsq(e3, 2, batch);         // scal[1] += ||e3||^2 / ||e0||^2 / batch
        if (!want_grad) return;
        // g3 = 2 e3 / ||e0||^2 (scaled by 1/batch in the weight reduction)
        cudaMemsetAsync(g, 0, sizeof(double) * nodes, s);
        k_axpy<<<flat_blocks(nodes), 256, 0, s>>>(g, e3, nodes, 1.0, scal);
        // post-smoother: dtheta -= J^T g ; g2 = g - (A'/(2d)) J_x^T g
        conv2_bwd(d, n, g, z3, gz, W, s);
        wgrad(d, n, s3, gz, g, z3, wpart, scal + 2, -1.0, grad, s);
        conv1_bwd(d, n, gz, gx, W, s);
        scaled_apply(d, n, gx, w, s);
        k_axpy<<<flat_blocks(nodes), 256, 0, s>>>(g, w, nodes, -1.0, nullptr);
        // coarse-grid correction adjoint
        cgc_adjoint(g);
        // pre-smoother weight gradient
        conv2_bwd(d, n, g, z1, gz, W, s);
        wgrad(d, n, s1, gz, g, z1, wpart, scal + 2, -1.0, grad, s);
    }

    // e0 = error after pair_cycles plain RB-GS V(1,1) cycles from white noise
    void sample(uint64_t seed) {
        Level<double>& F = pair[0];
        k_white_noise<<<flat_blocks(interior_of(d, n)), 256, 0, s>>>(F.u[0], d, n, seed);
        for (int k = 0; k < pair_cycles; ++k) vcycle(pair, 1);
        cudaMemcpyAsync(e0, F.u[0], sizeof(double) * nodes, cudaMemcpyDeviceToDevice, s);
    }
};

gmg_status check_dn(int d, int n) {
    if (d != 2 && d != 3) {
        set_error("d must be 2 or 3");
        return GMG_ERR_ARG;
    }
    const int nmax = d == 3 ? 512 : 4096;
    if (n < 4 || n > nmax || (n & (n - 1))) {
        set_error("n must be a power of two in [4, " + std::to_string(nmax) + "]");
        return GMG_ERR_ARG;
    }
    return GMG_OK;
}

}  // namespace
}  // namespace learned
}  // namespace gmg

using namespace gmg;
using namespace gmg::learned;

#define GMG_TRY_CUDA_RELEASE(expr, tr)                                             \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));        \
            (tr).release();                                                        \
            return e_ == cudaErrorMemoryAllocation ? GMG_ERR_ALLOC : GMG_ERR_CUDA; \
        }                                                                          \
    } while (0)

extern "C" {

gmg_status gmg_learned_conv(int d, int n, const float* weights, const double* x, double* y,
                            int tensor_cores, void* cuda_stream) {
    gmg_status st = check_dn(d, n);
    if (st != GMG_OK) return st;
    if (!weights || !x || !y) {
        set_error("weights, x, y must be non-NULL");
        return GMG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int T = d == 3 ? 27 : 9;
    float *wd = nullptr, *wr = nullptr, *z = nullptr;
    const int64_t nodes = nodes_of(d, n);
    GMG_CUDA_TRY(cudaMalloc(&wd, sizeof(float) * 2 * H * T * 2));
    wr = wd + 2 * H * T;
    cudaError_t e = cudaMalloc(&z, sizeof(float) * H * nodes);
    if (e == cudaSuccess) e = cudaMemsetAsync(z, 0, sizeof(float) * H * nodes, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(wd, weights, sizeof(float) * 2 * H * T, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_round_bf16<<<(2 * H * T + 255) / 256, 256, 0, s>>>(wd, wr, 2 * H * T);
        if (tensor_cores) {
            conv_tc(d, n, x, y, 0, wr, s);
        } else {
            conv1(d, n, x, z, wr, s);
            conv2(d, n, z, y, 0, wr, s);
        }
        e = cudaStreamSynchronize(s);
    }
    cudaFree(wd);
    cudaFree(z);
    if (e != cudaSuccess) {
        set_error(std::string("gmg_learned_conv: ") + cudaGetErrorString(e));
        return GMG_ERR_CUDA;
    }
    return GMG_OK;
}

gmg_status gmg_learned_loss_grad(int d, int n, const float* weights, const double* e0,
                                 int coarse_cycles, double* loss_out, double* grad_out,
                                 void* cuda_stream) {
    gmg_status st = check_dn(d, n);
    if (st != GMG_OK) return st;
    if (!weights || !e0 || !loss_out || coarse_cycles < 1) {
        set_error("weights, e0, loss_out must be non-NULL and coarse_cycles >= 1");
        return GMG_ERR_ARG;
    }
    Trainer tr;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    GMG_TRY_CUDA_RELEASE(tr.init(d, n, coarse_cycles, 0, s), tr);
    const int W = 2 * H * tr.T;
    float* wd = nullptr;
    GMG_TRY_CUDA_RELEASE(tr.alloc((void**)&wd, sizeof(float) * 2 * W), tr);
    GMG_TRY_CUDA_RELEASE(cudaMemcpyAsync(wd, weights, sizeof(float) * W, cudaMemcpyHostToDevice, s),
                         tr);
    k_round_bf16<<<(W + 255) / 256, 256, 0, s>>>(wd, wd + W, W);
    GMG_TRY_CUDA_RELEASE(cudaMemcpyAsync(tr.e0, e0, sizeof(double) * tr.nodes,
                                         cudaMemcpyDeviceToDevice, s),
                         tr);
    // scal[2] = 1 (the batch scale of the weight-gradient reduction)
    const double one = 1.0;
    GMG_TRY_CUDA_RELEASE(cudaMemcpyAsync(tr.scal + 2, &one, sizeof(double), cudaMemcpyHostToDevice, s),
                         tr);
    tr.loss_grad(wd + W, 1.0, grad_out != nullptr);
    double sc[2];
    GMG_TRY_CUDA_RELEASE(cudaMemcpyAsync(sc, tr.scal, sizeof(double) * 2, cudaMemcpyDeviceToHost, s),
                         tr);
    if (grad_out)
        GMG_TRY_CUDA_RELEASE(cudaMemcpyAsync(grad_out, tr.grad, sizeof(double) * W,
                                             cudaMemcpyDeviceToHost, s),
                             tr);
    GMG_TRY_CUDA_RELEASE(cudaStreamSynchronize(s), tr);
    *loss_out = sc[1];
    tr.release();
    return GMG_OK;
}

gmg_status gmg_learned_train(int d, int n, int steps, int batch, int pair_cycles, int coarse_cycles,
                             double lr, uint64_t seed, const float* w_init, float* w_out,
                             double* loss_history, void* cuda_stream) {
    gmg_status st = check_dn(d, n);
    if (st != GMG_OK) return st;
    if (steps < 1 || steps > 1000000 || batch < 1 || batch > 4096 || pair_cycles < 0 ||
        pair_cycles > 16 || coarse_cycles < 1 || coarse_cycles > 200 || !(lr > 0.0) || !w_init ||
        !w_out) {
        set_error("gmg_learned_train: bad arguments");
        return GMG_ERR_ARG;
    }
    Trainer tr;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    GMG_TRY_CUDA_RELEASE(tr.init(d, n, coarse_cycles, pair_cycles, s), tr);
    const int W = 2 * H * tr.T;
    float *master = nullptr, *work = nullptr;
    double *m1 = nullptr, *m2 = nullptr;
    GMG_TRY_CUDA_RELEASE(tr.alloc((void**)&master, sizeof(float) * W), tr);
    GMG_TRY_CUDA_RELEASE(tr.alloc((void**)&work, sizeof(float) * W), tr);
    GMG_TRY_CUDA_RELEASE(tr.alloc((void**)&m1, sizeof(double) * W), tr);
    GMG_TRY_CUDA_RELEASE(tr.alloc((void**)&m2, sizeof(double) * W), tr);
    GMG_TRY_CUDA_RELEASE(cudaMemcpyAsync(master, w_init, sizeof(float) * W, cudaMemcpyHostToDevice, s),
                         tr);
    k_round_bf16<<<(W + 255) / 256, 256, 0, s>>>(master, work, W);
    const double inv_batch = 1.0 / batch;
    GMG_TRY_CUDA_RELEASE(cudaMemcpyAsync(tr.scal + 2, &inv_batch, sizeof(double),
                                         cudaMemcpyHostToDevice, s),
                         tr);
    std::vector<double> hloss(1);
    for (int it = 0; it < steps; ++it) {
        cudaMemsetAsync(tr.grad, 0, sizeof(double) * W, s);
        cudaMemsetAsync(tr.scal + 1, 0, sizeof(double), s);
        for (int b = 0; b < batch; ++b) {
            tr.sample(seed * 1000003ull + (uint64_t)it * 4096ull + (uint64_t)b);
            tr.loss_grad(work, (double)batch, true);
        }
        k_adam<<<(W + 255) / 256, 256, 0, s>>>(master, work, tr.grad, m1, m2, W, it + 1, lr);
        if (loss_history) {
            GMG_TRY_CUDA_RELEASE(cudaMemcpyAsync(&loss_history[it], tr.scal + 1, sizeof(double),
                                                 cudaMemcpyDeviceToHost, s),
                                 tr);
        }
    }
    GMG_TRY_CUDA_RELEASE(cudaMemcpyAsync(w_out, master, sizeof(float) * W, cudaMemcpyDeviceToHost, s),
                         tr);
    GMG_TRY_CUDA_RELEASE(cudaStreamSynchronize(s), tr);
    tr.release();
    return GMG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Fused tensor-core network for the V-cycle: u += N(sigma) in one kernel.
//
// One CTA (8 warps) owns a TX x TY x TZ tile of output nodes.  sigma is
// staged in shared memory as BF16 on the tile plus a 2-node halo; conv1 runs
// on the tile plus a 1-node halo as a [16 nodes x 32 taps] x [32 taps x 8
// channels] product per 16 nodes (two mma.sync m16n8k16 BF16, FP32
// accumulate, taps 27..31 zero), its ReLU'd result stored channel-last in
// BF16 (16 bytes per node, zero outside the interior); conv2 runs per 16
// consecutive output nodes as sum over tap pairs of [16 nodes x (2 taps x 8
// channels)] x [16 x 8] with ldmatrix gathering each node's 8 channels at
// the tapped position and only column 0 of the B operand non-zero.  Hidden
// activations and sigma therefore enter the tensor cores in BF16; weights
// are BF16; every sum accumulates in FP32.
namespace gmg {
namespace learned {
namespace {

template <int DIM>
struct TcTile {
    // TX = 14: a halo-1 x-row is exactly 16 nodes, one conv1 mma group
    static constexpr int TX = 14, TY = DIM == 3 ? 8 : 16, TZ = DIM == 3 ? 8 : 1;
    static constexpr int HZ = DIM == 3 ? 1 : 0;                   // halo in z
    static constexpr int X1 = TX + 2, Y1 = TY + 2, Z1 = TZ + 2 * HZ;  // halo-1 region
    static constexpr int X2 = TX + 4, Y2 = TY + 4, Z2 = TZ + 4 * HZ;  // halo-2 region
    static constexpr int N1 = X1 * Y1 * Z1;
    static constexpr int N2 = X2 * Y2 * Z2;
    static constexpr int T = DIM == 3 ? 27 : 9;
    static constexpr int K1 = (T + 15) / 16;  // conv1 k-steps of 16 taps
    static constexpr int P2 = (T + 1) / 2;    // conv2 tap pairs
};

__device__ inline uint32_t pack_bf16(float lo, float hi) {
    const uint32_t l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return l | (h << 16);
}

__device__ inline void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ inline void ldmatrix_x4(uint32_t* r, const void* smem_row) {
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(smem_row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

template <int DIM>
__device__ inline int tap_dx(int t) { return t % 3 - 1; }
template <int DIM>
__device__ inline int tap_dy(int t) { return (t / 3) % 3 - 1; }
template <int DIM>
__device__ inline int tap_dz(int t) { return DIM == 3 ? t / 9 - 1 : 0; }

// MODE 1: u += N(sigma);  MODE 0: u = N(sigma) (interior nodes)
template <int DIM, int MODE>
__global__ void __launch_bounds__(256) k_conv_tc(const double* __restrict__ sigma,
                                                 double* __restrict__ u, int n,
                                                 const float* __restrict__ W) {
    using G = TcTile<DIM>;
    __shared__ __nv_bfloat16 xs[G::N2];
    __shared__ __align__(16) uint4 zs[G::N1];  // 8 BF16 channels per node
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int i0 = 1 + G::TX * blockIdx.x, j0 = 1 + G::TY * blockIdx.y,
              k0 = DIM == 3 ? 1 + G::TZ * blockIdx.z : 0;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    auto inside = [&](int i, int j, int k) {
        return i >= 1 && i < n && j >= 1 && j < n && (DIM == 2 || (k >= 1 && k < n));
    };
    // 1. sigma on the halo-2 region, BF16, zero outside the interior
    for (int m = threadIdx.x; m < G::N2; m += blockDim.x) {
        const int hx = m % G::X2, hy = (m / G::X2) % G::Y2, hz = m / (G::X2 * G::Y2);
        const int i = i0 - 2 + hx, j = j0 - 2 + hy, k = DIM == 3 ? k0 - 2 + hz : 0;
        const float v = inside(i, j, k) ? (float)sigma[k * sz + j * sy + i] : 0.f;
        xs[m] = __float2bfloat16_rn(v);
    }
    // B operands (weights) in registers
    uint32_t b1w[G::K1][2];
#pragma unroll
    for (int kh = 0; kh < G::K1; ++kh) {
        const int t0 = 16 * kh + 2 * tig;
        auto w1 = [&](int t) { return t < G::T ? W[gid * G::T + t] : 0.f; };
        b1w[kh][0] = pack_bf16(w1(t0), w1(t0 + 1));
        b1w[kh][1] = pack_bf16(w1(t0 + 8), w1(t0 + 9));
    }
    uint32_t b2w[G::P2][2];
#pragma unroll
    for (int pp = 0; pp < G::P2; ++pp) {
        const float* W2 = W + 8 * G::T;
        const int ta = 2 * pp, tb = 2 * pp + 1;
        auto w2 = [&](int c, int t) { return (gid == 0 && t < G::T) ? W2[c * G::T + t] : 0.f; };
        b2w[pp][0] = pack_bf16(w2(2 * tig, ta), w2(2 * tig + 1, ta));
        b2w[pp][1] = pack_bf16(w2(2 * tig, tb), w2(2 * tig + 1, tb));
    }
    __syncthreads();
    // 2. conv1 on the halo-1 region: groups of 16 nodes, one group per warp
    // turn.  This lane's taps (fixed per lane) as offsets in the halo-2 tile.
    constexpr int NT1 = 4 * G::K1;
    int toff[NT1];
    bool tok[NT1];
#pragma unroll
    for (int q = 0; q < NT1; ++q) {
        const int kh = q / 4, sub = q % 4;
        const int t = 16 * kh + 2 * tig + (sub & 1) + (sub >> 1) * 8;
        tok[q] = t < G::T;
        const int tt = tok[q] ? t : 0;
        toff[q] = (tap_dz<DIM>(tt) * G::Y2 + tap_dy<DIM>(tt)) * G::X2 + tap_dx<DIM>(tt);
    }
    static_assert(G::X1 == 16, "a halo-1 row must be one 16-node mma group");
    // this lane's two nodes of a row: x = gid and gid + 8 of the halo-1 row
    const bool xin0 = i0 - 1 + gid >= 1 && i0 - 1 + gid < n;
    const bool xin1 = i0 - 1 + gid + 8 >= 1 && i0 - 1 + gid + 8 < n;
    const unsigned short* xr = reinterpret_cast<const unsigned short*>(xs);
    const int rows1 = G::Y1 * G::Z1;
    for (int g = warp; g < rows1; g += 8) {
        const int hy = g % G::Y1, hz = g / G::Y1;
        const int j = j0 - 1 + hy, k = DIM == 3 ? k0 - 1 + hz : 0;
        const bool yzin = j >= 1 && j < n && (DIM == 2 || (k >= 1 && k < n));
        // centre of node (gid, hy, hz) in the halo-2 tile
        const int m0 = ((hz + G::HZ) * G::Y2 + (hy + 1)) * G::X2 + (gid + 1);
        const int m1 = m0 + 8;
        auto xb = [&](int m, int q) -> uint32_t {
            return tok[q] ? (uint32_t)xr[m + toff[q]] : 0u;
        };
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kh = 0; kh < G::K1; ++kh) {
            const int q = 4 * kh;
            uint32_t a[4];
            a[0] = xb(m0, q) | (xb(m0, q + 1) << 16);
            a[1] = xb(m1, q) | (xb(m1, q + 1) << 16);
            a[2] = xb(m0, q + 2) | (xb(m0, q + 3) << 16);
            a[3] = xb(m1, q + 2) | (xb(m1, q + 3) << 16);
            mma_bf16(c, a, b1w[kh][0], b1w[kh][1]);
        }
        // relu, BF16, channel-last; zero outside the interior
        uint32_t* z0 = reinterpret_cast<uint32_t*>(&zs[16 * g + gid]);
        uint32_t* z1 = reinterpret_cast<uint32_t*>(&zs[16 * g + gid + 8]);
        z0[tig] = (yzin && xin0) ? pack_bf16(fmaxf(c[0], 0.f), fmaxf(c[1], 0.f)) : 0u;
        z1[tig] = (yzin && xin1) ? pack_bf16(fmaxf(c[2], 0.f), fmaxf(c[3], 0.f)) : 0u;
    }
    __syncthreads();
    // 3. conv2 on 16-node x-rows of the output tile
    const int rows2 = G::TY * G::TZ;
    for (int row = warp; row < rows2; row += 8) {
        const int oy = row % G::TY, oz = row / G::TY;
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        const int mtx = lane >> 3, rr = lane & 7;  // ldmatrix: this lane's matrix and row
        // rows past the tile's last x (TX..15) are computed but discarded: read
        // the last column's neighbourhood there so every address stays in its row
        const int ox = min((mtx & 1) * 8 + rr, G::TX - 1);
        const int mc = ((oz + G::HZ) * G::Y1 + (oy + 1)) * G::X1 + (ox + 1);
        const int hi = mtx >> 1;
#pragma unroll
        for (int pp = 0; pp < G::P2; ++pp) {
            // tap 2pp (matrices 0, 1) or 2pp + 1 (matrices 2, 3); a padding tap
            // reads the centre row (its weight is zero)
            const int ta = 2 * pp, tb = 2 * pp + 1 < G::T ? 2 * pp + 1 : G::T / 2;
            const int oa = (tap_dz<DIM>(ta) * G::Y1 + tap_dy<DIM>(ta)) * G::X1 + tap_dx<DIM>(ta);
            const int ob = (tap_dz<DIM>(tb) * G::Y1 + tap_dy<DIM>(tb)) * G::X1 + tap_dx<DIM>(tb);
            uint32_t a[4];
            ldmatrix_x4(a, &zs[mc + (hi ? ob : oa)]);
            mma_bf16(c, a, b2w[pp][0], b2w[pp][1]);
        }
        if (tig == 0) {
            const int j = j0 + oy, k = DIM == 3 ? k0 + oz : 0;
            for (int h = 0; h < 2; ++h) {
                const int ox_ = gid + 8 * h;
                const int i = i0 + ox_;
                if (ox_ >= G::TX || !inside(i, j, k)) continue;
                const int64_t p = k * sz + j * sy + i;
                const double y = (double)c[2 * h];
                if (MODE == 1)
                    u[p] += y;
                else
                    u[p] = y;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// z-streaming 3D network: u += N(sigma) with conv2 as a GEMM over taps.
//
// A CTA owns a 14 x 14 column of output nodes and a chunk of planes and walks
// the planes.  Per plane kk (with a one-plane halo on either side of the
// chunk):
//  1. conv1 on the 16 x 16 halo-1 nodes of plane kk: per 16-node row a
//     [16 nodes x 48] x [48 x 8 channels] product, K = 9 (dz, dy) groups x 4
//     dx slots (dx = -1, 0, +1, one zero-weight slot); sigma (planes kk-1 ..
//     kk+1) sits in a ring of four BF16 planes stored twice (element e, and
//     shifted by one), so each A register is one aligned 32-bit load (three
//     mma.sync m16n8k16 BF16 per row);
//  2. the ReLU'd accumulators, rounded to BF16, are directly the A operand
//     of z = h W2 ([16 x 8(16)] x [16 x 32 taps], four mma): z[t][node], the
//     contribution of the node's hidden vector to tap t, FP32, one plane in
//     shared memory (zero outside the interior: h is zero there);
//  3. each thread owns one output column (x, y) and adds plane kk's
//     contributions to its three open outputs, planes kk+1, kk, kk-1 (taps
//     dz = -1, 0, +1), in registers; plane kk-1 is then complete: u += y.
// Sigma of plane kk+2 is fetched into registers while plane kk is computed.
// The hidden activations and sigma enter the tensor cores in BF16, weights
// are BF16, every sum is FP32 -- the numerics of k_conv_tc, with the taps of
// conv2 summed in a different order.
constexpr int ZS_T = 14;              // output tile (x and y)
constexpr int ZS_H1 = ZS_T + 2;       // halo-1 width: 16 nodes = one mma row group
constexpr int ZS_H2 = ZS_T + 4;       // halo-2 rows
constexpr int ZS_SW = 20;             // smem row stride of a sigma plane (18 + pad)
constexpr int ZS_SP = ZS_H2 * ZS_SW + 4;  // elements per sigma plane (+4: planes
                                          // 182 words apart, not a multiple of 32 banks)
constexpr int ZS_TS = 260;            // floats per tap of the z plane (256 nodes + pad)
constexpr int ZS_ZP = 27 * ZS_TS;     // floats of the z plane
constexpr int ZS_PLANES = 16;         // output planes per CTA
constexpr int ZS_PF = (ZS_SP + 255) / 256;  // sigma elements fetched per thread

constexpr size_t zs_smem_bytes() {
    return sizeof(float) * ZS_ZP + sizeof(__nv_bfloat16) * 2 * 4 * ZS_SP;
}

// sigma value of the halo-2 element m of plane k (0 outside the interior)
__device__ inline float zs_sigma(const double* sigma, int64_t sy, int64_t sz, int n, int i0,
                                 int j0, int k, int m) {
    const int x2 = m % ZS_SW, y2 = m / ZS_SW;
    const int i = i0 - 2 + x2, j = j0 - 2 + y2;
    if (m >= ZS_SP || x2 >= ZS_H2 || y2 >= ZS_H2 || i < 1 || i >= n || j < 1 || j >= n || k < 1 || k >= n)
        return 0.f;
    return (float)sigma[(int64_t)k * sz + (int64_t)j * sy + i];
}

template <int MODE>
__global__ void __launch_bounds__(256, 4) k_conv_zs(const double* __restrict__ sigma,
                                                    double* __restrict__ u, int n,
                                                    const float* __restrict__ W) {
    extern __shared__ __align__(16) unsigned char zs_smem[];
    float* zp = reinterpret_cast<float*>(zs_smem);                         // [27][260]
    __nv_bfloat16* sa = reinterpret_cast<__nv_bfloat16*>(zp + ZS_ZP);      // [4][SP]
    __nv_bfloat16* sb = sa + 4 * ZS_SP;                                    // shifted copy
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int i0 = 1 + ZS_T * blockIdx.x, j0 = 1 + ZS_T * blockIdx.y;
    const int k0 = 1 + ZS_PLANES * blockIdx.z;
    const int kend = min(k0 + ZS_PLANES, n);  // output planes k0 .. kend-1
    const int64_t sy = (int64_t)n + 1, sz = sy * sy;

    // conv1 B operand: k = 16 kh + (0..15) -> group g = k / 4 (dz, dy), slot
    // k % 4 (dx = slot - 1; slot 3 and groups >= 9 have weight 0)
    uint32_t b1w[3][2];
#pragma unroll
    for (int kh = 0; kh < 3; ++kh) {
        auto w1 = [&](int g, int slot) {
            return (g < 9 && slot < 3) ? W[gid * 27 + 3 * g + slot] : 0.f;
        };
        const int g = 4 * kh + (tig >> 1), sl = 2 * (tig & 1);
        b1w[kh][0] = pack_bf16(w1(g, sl), w1(g, sl + 1));
        b1w[kh][1] = pack_bf16(w1(g + 2, sl), w1(g + 2, sl + 1));
    }
    // z-GEMM B operand: k = channel (8..15 zero), n = tap 8 jn + gid
    uint32_t b2w[4];
#pragma unroll
    for (int jn = 0; jn < 4; ++jn) {
        const int t = 8 * jn + gid;
        auto w2 = [&](int c) { return t < 27 ? W[8 * 27 + c * 27 + t] : 0.f; };
        b2w[jn] = pack_bf16(w2(2 * tig), w2(2 * tig + 1));
    }

    float pf[ZS_PF];
    auto fetch = [&](int k) {
#pragma unroll
        for (int r = 0; r < ZS_PF; ++r)
            pf[r] = zs_sigma(sigma, sy, sz, n, i0, j0, k, threadIdx.x + 256 * r);
    };
    auto store = [&](int k) {  // the fetched plane k -> ring slot k & 3, both copies
        __nv_bfloat16* a = sa + (k & 3) * ZS_SP;
        __nv_bfloat16* b = sb + (k & 3) * ZS_SP;
#pragma unroll
        for (int r = 0; r < ZS_PF; ++r) {
            const int m = threadIdx.x + 256 * r;
            if (m < ZS_SP) {
                const __nv_bfloat16 v = __float2bfloat16_rn(pf[r]);
                a[m] = v;
                if (m > 0) b[m - 1] = v;
            }
        }
    };
    for (int k = k0 - 2; k <= k0; ++k) {
        fetch(k);
        store(k);
    }
    fetch(k0 + 1);

    // this thread's conv1 rows are x = gid, gid + 8 of each 16-node row: the
    // 32-bit pair of x-adjacent sigma values it reads starts at halo-2
    // column x (dx = -1, 0) or x + 2 (dx = +1, pad); its parity is gid's
    const int xoff = (tig & 1) ? 2 : 0;
    const __nv_bfloat16* src = (gid & 1) ? sb : sa;
    const int sh = (gid & 1) ? -1 : 0;  // element index in the chosen copy
    // the output column of this thread and its open sums (planes kk-1, kk, kk+1)
    const bool owner = threadIdx.x < ZS_T * ZS_T;
    const int ox = threadIdx.x % ZS_T, oy = threadIdx.x / ZS_T;
    const bool col_in = owner && i0 + ox < n && j0 + oy < n;
    float y_prev = 0.f, y_cur = 0.f, y_next = 0.f;
    for (int kk = k0 - 1; kk <= kend; ++kk) {
        // u of the output finished this plane, read early (used after conv1)
        const int64_t po = (int64_t)(kk - 1) * sz + (int64_t)(j0 + oy) * sy + i0 + ox;
        const bool out = col_in && kk - 1 >= k0;
        const double u_old = (MODE == 1 && out) ? u[po] : 0.0;
        __syncthreads();  // sigma planes kk-1 .. kk+1 stored; z plane free
        for (int ry = warp; ry < ZS_H1; ry += 8) {
            const int j = j0 - 1 + ry;
            const bool yk = j >= 1 && j < n && kk >= 1 && kk < n;
            const int ia = i0 - 1 + gid, ib = ia + 8;
            const bool ina = yk && ia >= 1 && ia < n, inb = yk && ib >= 1 && ib < n;
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kh = 0; kh < 3; ++kh) {
                uint32_t a[4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    int g = 4 * kh + (tig >> 1) + 2 * h;
                    if (g >= 9) g = 4;  // zero-weight group: any in-tile pair
                    const int dz = g / 3 - 1, dy = g % 3 - 1;
                    const int e = ((kk + dz) & 3) * ZS_SP + (ry + 1 + dy) * ZS_SW + xoff + sh;
                    a[2 * h] = *reinterpret_cast<const uint32_t*>(src + e + gid);
                    a[2 * h + 1] = *reinterpret_cast<const uint32_t*>(src + e + gid + 8);
                }
                mma_bf16(c, a, b1w[kh][0], b1w[kh][1]);
            }
            uint32_t ah[4];
            ah[0] = ina ? pack_bf16(fmaxf(c[0], 0.f), fmaxf(c[1], 0.f)) : 0u;
            ah[1] = inb ? pack_bf16(fmaxf(c[2], 0.f), fmaxf(c[3], 0.f)) : 0u;
            ah[2] = 0u;
            ah[3] = 0u;
#pragma unroll
            for (int jn = 0; jn < 4; ++jn) {
                float z[4] = {0.f, 0.f, 0.f, 0.f};
                mma_bf16(z, ah, b2w[jn], 0u);
                const int t = 8 * jn + 2 * tig;
                float* zt = zp + t * ZS_TS + ry * ZS_H1;
                if (t < 27) {
                    zt[gid] = z[0];
                    zt[gid + 8] = z[2];
                }
                if (t + 1 < 27) {
                    zt[ZS_TS + gid] = z[1];
                    zt[ZS_TS + gid + 8] = z[3];
                }
            }
        }
        store(kk + 2);  // slot (kk+2) & 3 is not read by this plane's conv1
        fetch(kk + 3);
        __syncthreads();  // z plane kk complete
        if (col_in) {
            // plane kk's taps: dz = +1 -> output kk-1, 0 -> kk, -1 -> kk+1
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
                const float v = zp[t * ZS_TS + (oy + 1 + dy) * ZS_H1 + ox + 1 + dx];
                if (dz == 1)
                    y_prev += v;
                else if (dz == 0)
                    y_cur += v;
                else
                    y_next += v;
            }
            if (out) u[po] = u_old + (double)y_prev;
        }
        y_prev = y_cur;
        y_cur = y_next;
        y_next = 0.f;
    }
}

}  // namespace

// 3D uses the z-streaming kernel unless GMG_CONV_ZS=0 (then the tile kernel;
// the two agree to FP32 rounding of the conv2 sums).
bool conv_zs_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("GMG_CONV_ZS");
        return !(v && v[0] == '0');
    }();
    return on;
}

void conv_tc(int d, int n, const double* sigma, double* u, int mode, const float* W,
             cudaStream_t s) {
    if (d == 3 && conv_zs_enabled()) {
        const size_t bytes = zs_smem_bytes();
        auto kern = mode == 1 ? k_conv_zs<1> : k_conv_zs<0>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        dim3 grid((n - 1 + ZS_T - 1) / ZS_T, (n - 1 + ZS_T - 1) / ZS_T,
                  (n - 1 + ZS_PLANES - 1) / ZS_PLANES);
        kern<<<grid, 256, bytes, s>>>(sigma, u, n, W);
        return;
    }
    if (d == 3) {
        using G = TcTile<3>;
        dim3 grid((n - 1 + G::TX - 1) / G::TX, (n - 1 + G::TY - 1) / G::TY,
                  (n - 1 + G::TZ - 1) / G::TZ);
        if (mode == 1)
            k_conv_tc<3, 1><<<grid, 256, 0, s>>>(sigma, u, n, W);
        else
            k_conv_tc<3, 0><<<grid, 256, 0, s>>>(sigma, u, n, W);
    } else {
        using G = TcTile<2>;
        dim3 grid((n - 1 + G::TX - 1) / G::TX, (n - 1 + G::TY - 1) / G::TY, 1);
        if (mode == 1)
            k_conv_tc<2, 1><<<grid, 256, 0, s>>>(sigma, u, n, W);
        else
            k_conv_tc<2, 0><<<grid, 256, 0, s>>>(sigma, u, n, W);
    }
}

}  // namespace learned
}  // namespace gmg
