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
// (on the host it names a host-side shadow), so every call looks up the real
// address on the current device with cudaGetSymbolAddress (a lookup that
// allocates nothing).  Looking it up on every call rather than caching it
// keeps the address right after the caller resets the device
// (cudaDeviceReset reloads the module).  The first call on a device may load
// the library's device code there: make that first call before any stream
// capture.  Every call shares the one array and keeps the last call's
// contents: each call writes every partial sum it later reads, so nothing
// has to start at zero, but calls whose kernels overlap on the GPU (other
// streams, other host threads) race on the array and must be serialised by
// the caller.
//
// The kernels are this file's own: one block per 256/x rows, no grid-stride
// loop, neighbours summed left to right.  The result agrees with the handle
// path's gmg_residual_norm to rounding (a different summation order), not
// bit for bit.
#include <cmath>
#include <string>
#include <utility>

#include "gmg_internal.cuh"

namespace {

constexpr int kMaxPartials = 65536;
__device__ __align__(256) double g_partials[kMaxPartials];

// Device address of g_partials on the current device.
cudaError_t partials_address(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

struct Shape {
    dim3 grid, block;
};

// Launch shape: 256 threads, x along a row (32..128 threads), one block per
// 256/x rows of a plane, so one partial sum per block.
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
// u holds there.  One partial per block.
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

// GMG_OK if p is 8-byte aligned device (or managed) memory usable on the
// current device; GMG_ERR_LAYOUT with a message otherwise.  Nothing is
// launched before every pointer has passed.
gmg_status check_pointer(const void* p, const char* name) {
    if (!p) {
        gmg::set_error(std::string(name) + " is NULL");
        return GMG_ERR_LAYOUT;
    }
    if (reinterpret_cast<uintptr_t>(p) % alignof(double) != 0) {
        gmg::set_error(std::string(name) + " is not 8-byte aligned");
        return GMG_ERR_LAYOUT;
    }
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        gmg::set_error(std::string(name) + " is not a device pointer");
        return GMG_ERR_LAYOUT;
    }
    if (a.type == cudaMemoryTypeManaged) return GMG_OK;
    if (a.type != cudaMemoryTypeDevice) {
        gmg::set_error(std::string(name) + " is not a device pointer");
        return GMG_ERR_LAYOUT;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || a.device != dev) {
        cudaGetLastError();
        gmg::set_error(std::string(name) + " lives on device " + std::to_string(a.device) +
                       ", not on the current device " + std::to_string(dev));
        return GMG_ERR_LAYOUT;
    }
    return GMG_OK;
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
    for (const auto& [p, name] : {std::pair<const void*, const char*>{f, "f"},
                                  {u, "u"},
                                  {norm_dev, "norm_dev"}}) {
        const gmg_status st = check_pointer(p, name);
        if (st != GMG_OK) return st;
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
