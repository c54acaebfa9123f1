// Allocation-free FP64 residual norm (gmg_residual_norm_noalloc).
//
// Who needs it: code that must not allocate device memory at the moment it
// wants a residual -- a callback running inside a custom device allocator or
// memory-pool hook (re-entering cudaMalloc there deadlocks or recurses), a
// real-time loop that forbids cudaMalloc/cudaFree because they can
// synchronise the whole device, or an embedding host that hands the library
// a fixed memory budget up front.  Such a caller cannot create a gmg_handle
// (it allocates the level hierarchy and a partial-sum buffer), so this entry
// point takes only the caller's f, u and output and keeps its scratch in a
// fixed static array instead.
//
// Scratch: g_partials, a file-scope __device__ array of kMaxPartials doubles
// (512 KiB) that every GPU which loads this library holds until the process
// exits.  Host code cannot use the symbol g_partials as a device address
// (on the host it names a host-side shadow), so the first call on each
// device looks up the real address with cudaGetSymbolAddress, with that
// device current, and caches it.  Make that first call before any stream
// capture.  Every call shares the one array and keeps the last call's
// contents: each call writes every partial sum it later reads, so nothing
// has to start at zero, but calls whose kernels overlap on the GPU (other
// streams, other host threads) race on the array and must be serialised by
// the caller.
#include <cmath>
#include <mutex>
#include <string>

#include "gmg_internal.cuh"

namespace {

constexpr int kMaxPartials = 65536;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_partials[kMaxPartials];

std::mutex g_mu;
double* g_partials_addr[kMaxDevices] = {};

// Device address of g_partials on the current device (looked up once).
cudaError_t partials_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_addr[dev];
    return cudaSuccess;
}

struct Shape {
    dim3 grid, block;
};

// The launch shape of the handle path's residual-norm kernel: 256 threads,
// x along a row (32..128 threads), one block per 256/x rows of a plane.
Shape shape(int d, int n) {
    int bx = 32;
    while (bx < n && bx < 128) bx *= 2;
    const int by = 256 / bx;
    Shape s;
    s.block = dim3(bx, by, 1);
    s.grid = dim3((unsigned)((n - 1 + by - 1) / by), d == 3 ? (unsigned)(n - 1) : 1u, 1);
    return s;
}

// Partial sums of sigma^2, sigma = q + c * (sum of neighbours) - u with
// q = h^2 f / (2d) formed on the fly; boundary neighbours read as 0 whatever
// u holds there.  One partial per block, same order as the handle path.
template <int DIM>
__global__ void __launch_bounds__(256) k_resnorm_static(const double* __restrict__ f,
                                                        const double* __restrict__ u,
                                                        double* __restrict__ partial, int n,
                                                        double scale, double c) {
    __shared__ double warp_sums[8];
    const int j = blockIdx.x * blockDim.y + threadIdx.y + 1;
    const int k = DIM == 3 ? blockIdx.y + 1 : 0;
    double acc = 0.0;
    if (j < n) {
        const int64_t sy = (int64_t)n + 1;
        const int64_t sz = DIM == 3 ? sy * sy : 0;
        const int64_t row = k * sz + j * sy;
        for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
            const int64_t p = row + i;
            double s = i > 1 ? u[p - 1] : 0.0;
            s = s + (i < n - 1 ? u[p + 1] : 0.0);
            s += j > 1 ? u[p - sy] : 0.0;
            s += j < n - 1 ? u[p + sy] : 0.0;
            if (DIM == 3) {
                s += k > 1 ? u[p - sz] : 0.0;
                s += k < n - 1 ? u[p + sz] : 0.0;
            }
            const double q = scale * f[p];
            const double sig = fma(c, s, q) - u[p];
            acc = fma(sig, sig, acc);
        }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if ((t & 31) == 0) warp_sums[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += warp_sums[w];
        partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// out = 2d * sqrt(sum of partials): the unscaled residual norm.
__global__ void __launch_bounds__(1024) k_finish_static(const double* __restrict__ partial,
                                                        int count, double two_d,
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
        out[0] = two_d * sqrt(s);
    }
}

bool device_pointer(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" gmg_status gmg_residual_norm_noalloc(int d, int n, const double* f, const double* u,
                                                double* norm_dev, void* cuda_stream) {
    using gmg::set_error;
    if (d != 2 && d != 3) {
        set_error("d must be 2 or 3");
        return GMG_ERR_ARG;
    }
    const int nmax = d == 2 ? 16384 : 1024;
    if (n < 2 || n > nmax || (n & (n - 1)) != 0) {
        set_error("n must be a power of two in [2, " + std::to_string(nmax) + "]");
        return GMG_ERR_ARG;
    }
    const Shape s = shape(d, n);
    const int64_t partials = (int64_t)s.grid.x * s.grid.y;
    if (partials > kMaxPartials) {
        set_error("gmg_residual_norm_noalloc: this grid needs " + std::to_string(partials) +
                  " partial sums but the static scratch holds " + std::to_string(kMaxPartials) +
                  " (largest grids: 3D n = 256, 2D n = 16384); use gmg_residual_norm");
        return GMG_ERR_ARG;
    }
    if (!f || !u || !norm_dev) {
        set_error("f, u and norm_dev must be non-NULL device pointers");
        return GMG_ERR_LAYOUT;
    }
    if (!device_pointer(f) || !device_pointer(u) || !device_pointer(norm_dev)) {
        set_error("f, u and norm_dev must be device pointers");
        return GMG_ERR_LAYOUT;
    }
    double* partial = nullptr;
    cudaError_t e = partials_address(&partial);
    if (e != cudaSuccess) {
        set_error(std::string("cudaGetSymbolAddress(g_partials): ") + cudaGetErrorString(e));
        return GMG_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const double h = 1.0 / n;
    const double scale = h * h / (2.0 * d);
    const double c = d == 3 ? 1.0 / 6.0 : 0.25;
    if (d == 3)
        k_resnorm_static<3><<<s.grid, s.block, 0, st>>>(f, u, partial, n, scale, c);
    else
        k_resnorm_static<2><<<s.grid, s.block, 0, st>>>(f, u, partial, n, scale, c);
    k_finish_static<<<1, 1024, 0, st>>>(partial, (int)partials, 2.0 * d, norm_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("gmg_residual_norm_noalloc launch: ") + cudaGetErrorString(e));
        return GMG_ERR_CUDA;
    }
    return GMG_OK;
}
