// FP64 level kernels of the plain V-cycle (Algorithm 1 on every level).
//
// Scaled variables: with the unscaled 5/7-point operator A' (section 2.2)
// and b = h^2 f, each level stores q = b / (2d); the Gauss-Seidel value of a
// node is q + c * (sum of its 2d neighbours), c = 1/(2d), and the scaled
// residual is sigma = q + c * sum - u = (b - A'u) / (2d).  Full weighting of
// b_{l+1} = 4 FW(b - A'u) then reads q_{l+1} = 4 FW(sigma): every transfer
// weight is a power of two.
//
// On GB300 FP64 arithmetic (2 DFMA/clk/SM) rather than HBM bounds these
// kernels, so each is written to issue as few double-precision instructions
// per node as the operation allows:
//   red-black half sweep   5 DADD + 1 DFMA per updated node
//   residual (+norm)       5 DADD + 1 DFMA + 1 DADD (+1 DFMA)
//   restriction            red nodes only after a black half sweep (the black
//                          residual is zero in exact arithmetic): 13 ops per
//                          coarse node in 3D
//   prolongation+correct   per coarse cell, pair/quad/octet sums shared by
//                          its 2^d fine nodes: 2.5 ops per fine node in 3D
#include "gmg_internal.cuh"

namespace gmg {
namespace fp64 {
namespace {

__host__ __device__ inline int64_t sy_of(int n) { return (int64_t)n + 1; }
template <int DIM>
__host__ __device__ inline int64_t sz_of(int n) { return DIM == 3 ? ((int64_t)n + 1) * (n + 1) : 0; }

// Launch shape for kernels that walk interior rows: x threads along a row,
// y over rows j, z over planes k (3D).
struct RowLaunch {
    dim3 grid, block;
};

RowLaunch row_launch(int d, int n, int xcount) {
    int bx = 32;
    while (bx < xcount && bx < 128) bx *= 2;
    int by = 256 / bx;
    RowLaunch L;
    L.block = dim3(bx, by, 1);
    L.grid = dim3((unsigned)((n - 1 + by - 1) / by), d == 3 ? (unsigned)(n - 1) : 1u, 1);
    return L;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_prepare(const double* __restrict__ f, double* __restrict__ q,
                                                 double* __restrict__ u, int n, double scale) {
    const int64_t nodes = DIM == 3 ? sy_of(n) * sy_of(n) * sy_of(n) : sy_of(n) * sy_of(n);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nodes;
         p += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(p % sy_of(n));
        int64_t t = p / sy_of(n);
        int j = (int)(t % sy_of(n));
        int k = DIM == 3 ? (int)(t / sy_of(n)) : 1;
        bool inner = i > 0 && i < n && j > 0 && j < n && k > 0 && k < (DIM == 3 ? n : 2);
        if (inner) {
            q[p] = scale * f[p];
        } else {
            q[p] = 0.0;
            u[p] = 0.0;
        }
    }
}

template <int DIM>
__device__ inline double nbr_sum(const double* u, int64_t p, int64_t sy, int64_t sz) {
    double s = u[p - 1] + u[p + 1];
    s += u[p - sy];
    s += u[p + sy];
    if (DIM == 3) {
        s += u[p - sz];
        s += u[p + sz];
    }
    return s;
}

// One colour of red-black Gauss-Seidel: nodes with (i+j+k) % 2 == color.
template <int DIM>
__global__ void __launch_bounds__(256) k_rb_half(double* __restrict__ u, const double* __restrict__ q,
                                                 int n, int color, double c) {
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    if (j >= n) return;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t row = k * sz + j * sy;
    const int i0 = 1 + ((1 + j + k + color) & 1);
    for (int i = i0 + 2 * threadIdx.x; i < n; i += 2 * blockDim.x) {
        const int64_t p = row + i;
        u[p] = fma(c, nbr_sum<DIM>(u, p, sy, sz), q[p]);
    }
}

// Weighted Jacobi: u_out = u + omega * sigma, all nodes from u_in.
template <int DIM>
__global__ void __launch_bounds__(256) k_wj(const double* __restrict__ u, double* __restrict__ uo,
                                            const double* __restrict__ q, int n, double c,
                                            double omega) {
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    if (j >= n) return;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t row = k * sz + j * sy;
    for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
        const int64_t p = row + i;
        const double up = u[p];
        const double sig = fma(c, nbr_sum<DIM>(u, p, sy, sz), q[p]) - up;
        uo[p] = fma(omega, sig, up);
    }
}

// sigma on all interior nodes, or on red nodes only (black entries of r are
// never written and never read in that mode).
template <int DIM, bool RED_ONLY>
__global__ void __launch_bounds__(256) k_residual(const double* __restrict__ u, const double* __restrict__ q,
                                                  double* __restrict__ r, int n, double c) {
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    if (j >= n) return;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t row = k * sz + j * sy;
    const int step = RED_ONLY ? 2 : 1;
    const int i0 = RED_ONLY ? 1 + ((1 + j + k) & 1) : 1;
    for (int i = i0 + step * threadIdx.x; i < n; i += step * blockDim.x) {
        const int64_t p = row + i;
        r[p] = fma(c, nbr_sum<DIM>(u, p, sy, sz), q[p]) - u[p];
    }
}

// q_c = 4 FW(sigma) at every coarse interior node; u_c = 0 (a fresh coarse
// iterate) or u_c = q_c when the coarse grid has its single unknown (exact
// solve u = b/(2d)).  With RED_ONLY the black-node terms (faces and corners
// in 3D, faces in 2D) are zero and skipped.
template <int DIM, bool RED_ONLY>
__global__ void __launch_bounds__(256) k_restrict(const double* __restrict__ r, double* __restrict__ qc,
                                                  double* __restrict__ uc, int nc, int exact) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int J = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int K = DIM == 3 ? blockIdx.z + 1 : 0;
    if (I >= nc || J >= nc) return;
    const int n = 2 * nc;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t p = (2 * K) * sz + (2 * J) * sy + 2 * I;
    double v;
    if (DIM == 3) {
        double e = r[p - 1 - sy] + r[p + 1 - sy];
        e += r[p - 1 + sy];
        e += r[p + 1 + sy];
        e += r[p - 1 - sz];
        e += r[p + 1 - sz];
        e += r[p - sy - sz];
        e += r[p + sy - sz];
        e += r[p - 1 + sz];
        e += r[p + 1 + sz];
        e += r[p - sy + sz];
        e += r[p + sy + sz];
        if (RED_ONLY) {
            v = fma(0.125, e, 0.5 * r[p]);
        } else {
            double fc = r[p - 1] + r[p + 1];
            fc += r[p - sy];
            fc += r[p + sy];
            fc += r[p - sz];
            fc += r[p + sz];
            double co = r[p - 1 - sy - sz] + r[p + 1 - sy - sz];
            co += r[p - 1 + sy - sz];
            co += r[p + 1 + sy - sz];
            co += r[p - 1 - sy + sz];
            co += r[p + 1 - sy + sz];
            co += r[p - 1 + sy + sz];
            co += r[p + 1 + sy + sz];
            v = fma(0.0625, co, fma(0.125, e, fma(0.25, fc, 0.5 * r[p])));
        }
    } else {
        double co = r[p - 1 - sy] + r[p + 1 - sy];
        co += r[p - 1 + sy];
        co += r[p + 1 + sy];
        if (RED_ONLY) {
            v = fma(0.25, co, r[p]);
        } else {
            double fc = r[p - 1] + r[p + 1];
            fc += r[p - sy];
            fc += r[p + sy];
            v = fma(0.25, co, fma(0.5, fc, r[p]));
        }
    }
    const int64_t sc = sy_of(nc);
    const int64_t P = ((int64_t)K * sc + J) * sc + I;
    qc[P] = v;
    uc[P] = exact ? v : 0.0;
}

// u += P u_c, one thread per coarse cell (I,J,K) in [0, nc-1]^d updating
// the fine nodes (2I+a, 2J+b, 2K+c), a,b,c in {0,1}, that are interior.
template <int DIM>
__global__ void __launch_bounds__(256) k_prolong_add(const double* __restrict__ uc, double* __restrict__ u,
                                                     int nc) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = DIM == 3 ? blockIdx.z : 0;
    if (I >= nc || J >= nc) return;
    const int n = 2 * nc;
    const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
    const int64_t cy = sy_of(nc), cz = sz_of<DIM>(nc);
    const int64_t P = K * cz + J * cy + I;
    const int64_t p = (2 * K) * sz + (2 * J) * sy + 2 * I;
    const double c000 = uc[P], c100 = uc[P + 1], c010 = uc[P + cy], c110 = uc[P + 1 + cy];
    const double x00 = c000 + c100;
    const double x10 = c010 + c110;
    const double y00 = c000 + c010;
    const double qxy = x00 + x10;
    if (DIM == 2) {
        if (I > 0 && J > 0) u[p] += c000;
        if (J > 0) u[p + 1] = fma(0.5, x00, u[p + 1]);
        if (I > 0) u[p + sy] = fma(0.5, y00, u[p + sy]);
        u[p + 1 + sy] = fma(0.25, qxy, u[p + 1 + sy]);
    } else {
        const double c001 = uc[P + cz], c101 = uc[P + 1 + cz], c011 = uc[P + cy + cz],
                     c111 = uc[P + 1 + cy + cz];
        const double x01 = c001 + c101;
        const double x11 = c011 + c111;
        const double y01 = c001 + c011;
        const double z00 = c000 + c001;
        const double qxz = x00 + x01;
        const double qyz = y00 + y01;
        const double oct = qxy + (x01 + x11);
        if (K > 0) {
            if (I > 0 && J > 0) u[p] += c000;
            if (J > 0) u[p + 1] = fma(0.5, x00, u[p + 1]);
            if (I > 0) u[p + sy] = fma(0.5, y00, u[p + sy]);
            u[p + 1 + sy] = fma(0.25, qxy, u[p + 1 + sy]);
        }
        const int64_t pz = p + sz;
        if (I > 0 && J > 0) u[pz] = fma(0.5, z00, u[pz]);
        if (J > 0) u[pz + 1] = fma(0.25, qxz, u[pz + 1]);
        if (I > 0) u[pz + sy] = fma(0.25, qyz, u[pz + sy]);
        u[pz + 1 + sy] = fma(0.125, oct, u[pz + 1 + sy]);
    }
}

constexpr int kNormThreads = 256;

// Sum of sigma^2 over interior nodes: fixed per-thread order, fixed warp
// shuffle tree, fixed cross-warp order, one partial per block.
template <int DIM>
__global__ void __launch_bounds__(kNormThreads) k_resnorm(const double* __restrict__ u,
                                                          const double* __restrict__ q,
                                                          double* __restrict__ partial, int n,
                                                          double c) {
    __shared__ double warp_sums[kNormThreads / 32];
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    double acc = 0.0;
    if (j < n) {
        const int64_t sy = sy_of(n), sz = sz_of<DIM>(n);
        const int64_t row = k * sz + j * sy;
        for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
            const int64_t p = row + i;
            const double sig = fma(c, nbr_sum<DIM>(u, p, sy, sz), q[p]) - u[p];
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
        partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(1024) k_sum_partials(const double* __restrict__ partial, int count,
                                                       double* __restrict__ out) {
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

}  // namespace

void prepare(int d, int n, const double* f, double* q, double* u, cudaStream_t s) {
    const double h = 1.0 / n;
    const double scale = h * h / (2.0 * d);
    const int64_t nodes = d == 3 ? (int64_t)(n + 1) * (n + 1) * (n + 1) : (int64_t)(n + 1) * (n + 1);
    const int blocks = (int)std::min<int64_t>((nodes + 255) / 256, 152 * 16);
    if (d == 3)
        k_prepare<3><<<blocks, 256, 0, s>>>(f, q, u, n, scale);
    else
        k_prepare<2><<<blocks, 256, 0, s>>>(f, q, u, n, scale);
}

void rb_half(int d, int n, double* u, const double* q, int color, cudaStream_t s) {
    RowLaunch L = row_launch(d, n, n / 2);
    if (d == 3)
        k_rb_half<3><<<L.grid, L.block, 0, s>>>(u, q, n, color, 1.0 / 6.0);
    else
        k_rb_half<2><<<L.grid, L.block, 0, s>>>(u, q, n, color, 0.25);
}

void wj_sweep(int d, int n, const double* u_in, double* u_out, const double* q, double omega,
              cudaStream_t s) {
    RowLaunch L = row_launch(d, n, n);
    if (d == 3)
        k_wj<3><<<L.grid, L.block, 0, s>>>(u_in, u_out, q, n, 1.0 / 6.0, omega);
    else
        k_wj<2><<<L.grid, L.block, 0, s>>>(u_in, u_out, q, n, 0.25, omega);
}

void residual(int d, int n, const double* u, const double* q, double* r, bool red_only,
              cudaStream_t s) {
    RowLaunch L = row_launch(d, n, red_only ? n / 2 : n);
    const double c = d == 3 ? 1.0 / 6.0 : 0.25;
    if (d == 3) {
        if (red_only)
            k_residual<3, true><<<L.grid, L.block, 0, s>>>(u, q, r, n, c);
        else
            k_residual<3, false><<<L.grid, L.block, 0, s>>>(u, q, r, n, c);
    } else {
        if (red_only)
            k_residual<2, true><<<L.grid, L.block, 0, s>>>(u, q, r, n, c);
        else
            k_residual<2, false><<<L.grid, L.block, 0, s>>>(u, q, r, n, c);
    }
}

void restrict_fw(int d, int n, const double* r, double* qc, double* uc, bool red_only,
                 bool exact_coarsest, cudaStream_t s) {
    const int nc = n / 2;
    int bx = 32;
    while (bx < nc - 1 && bx < 128) bx *= 2;
    const int by = 256 / bx;
    dim3 block(bx, by, 1);
    dim3 grid((nc - 1 + bx - 1) / bx, (nc - 1 + by - 1) / by, d == 3 ? nc - 1 : 1);
    const int ex = exact_coarsest ? 1 : 0;
    if (d == 3) {
        if (red_only)
            k_restrict<3, true><<<grid, block, 0, s>>>(r, qc, uc, nc, ex);
        else
            k_restrict<3, false><<<grid, block, 0, s>>>(r, qc, uc, nc, ex);
    } else {
        if (red_only)
            k_restrict<2, true><<<grid, block, 0, s>>>(r, qc, uc, nc, ex);
        else
            k_restrict<2, false><<<grid, block, 0, s>>>(r, qc, uc, nc, ex);
    }
}

void prolong_add(int d, int nc, const double* uc, double* u, cudaStream_t s) {
    int bx = 32;
    while (bx < nc && bx < 128) bx *= 2;
    const int by = 256 / bx;
    dim3 block(bx, by, 1);
    dim3 grid((nc + bx - 1) / bx, (nc + by - 1) / by, d == 3 ? nc : 1);
    if (d == 3)
        k_prolong_add<3><<<grid, block, 0, s>>>(uc, u, nc);
    else
        k_prolong_add<2><<<grid, block, 0, s>>>(uc, u, nc);
}

int resnorm_partials(int d, int n) {
    RowLaunch L = row_launch(d, n, n);
    return (int)(L.grid.x * L.grid.y);
}

void resnorm(int d, int n, const double* u, const double* q, double* partial, double* out,
             cudaStream_t s) {
    RowLaunch L = row_launch(d, n, n);
    const double c = d == 3 ? 1.0 / 6.0 : 0.25;
    if (d == 3)
        k_resnorm<3><<<L.grid, L.block, 0, s>>>(u, q, partial, n, c);
    else
        k_resnorm<2><<<L.grid, L.block, 0, s>>>(u, q, partial, n, c);
    k_sum_partials<<<1, 1024, 0, s>>>(partial, (int)(L.grid.x * L.grid.y), out);
}

}  // namespace fp64
}  // namespace gmg
