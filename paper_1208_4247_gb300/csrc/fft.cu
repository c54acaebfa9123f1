// Direct FFT Poisson solve (the paper's comparison method, section 2.3):
// the FD system A'u = h^2 f is diagonal in the sine basis, so
//     u = S^-1 diag(1 / lambda) S (h^2 f),   S = DST-I along every axis,
//     lambda_k = sum_m 4 sin^2(pi k_m / (2n)),  S^-1 = (2/n)^d S.
// (The paper divides by the continuous symbol k_x^2 + k_y^2; the discrete
// eigenvalues make the result the exact solution of the same FD system the
// multigrid solves.)  Each DST-I of length n-1 is a length-2n real-to-complex
// cuFFT of the odd extension [0, x, 0, -reverse(x)]: its k-th coefficient is
// -2i y_k.  Lines along x use a line-major extension; lines along y and z an
// element-major one (cuFFT strided layout), so every gather and scatter
// kernel reads and writes contiguous x.
#include <cufft.h>

#include <cmath>
#include <string>

#include "gmg_internal.cuh"

namespace gmg {
namespace fft {
namespace {

// axis 0 (x): ext[line][j], line = (k-1)(n-1) + (j'-1);
// axes 1, 2: ext[j][line], line = (other-1)(n-1) + (i-1)
__device__ inline int64_t node(int d, int n, int axis, int64_t line, int j) {
    const int64_t m = n + 1;
    const int a = (int)(line % (n - 1)) + 1;
    const int b = d == 3 ? (int)(line / (n - 1)) + 1 : 0;
    if (axis == 0) return ((int64_t)b * m + a) * m + j;    // a = y, b = z
    if (axis == 1) return ((int64_t)b * m + j) * m + a;    // a = x, b = z
    return ((int64_t)j * m + b) * m + a;                    // axis 2: a = x, b = y
}

__global__ void k_extend(const double* __restrict__ x, double* __restrict__ ext, int d, int n,
                         int axis, int64_t lines) {
    const int L = 2 * n;
    const int64_t total = lines * L;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t line;
        int j;
        if (axis == 0) {
            line = t / L;
            j = (int)(t % L);
        } else {
            j = (int)(t / lines);
            line = t % lines;
        }
        double v = 0.0;
        if (j > 0 && j < n)
            v = x[node(d, n, axis, line, j)];
        else if (j > n)
            v = -x[node(d, n, axis, line, L - j)];
        ext[t] = v;
    }
}

// y_k = -Im(X_k) / 2 for k = 1..n-1, times scale (and, with eig, divided by
// lambda at the node: the diagonal solve fused into the last forward pass)
__global__ void k_extract(const cufftDoubleComplex* __restrict__ X, double* __restrict__ y, int d,
                          int n, int axis, int64_t lines, double scale, int eig) {
    const int C = n + 1;
    const int64_t total = lines * (n - 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t line;
        int k;
        int64_t src;
        if (axis == 0) {
            line = t / (n - 1);
            k = (int)(t % (n - 1)) + 1;
            src = line * C + k;
        } else {
            k = (int)(t / lines) + 1;
            line = t % lines;
            src = (int64_t)k * lines + line;
        }
        const int64_t p = node(d, n, axis, line, k);
        double v = -0.5 * X[src].y * scale;
        if (eig) {
            const int64_t m = n + 1;
            const int i = (int)(p % m), jj = (int)((p / m) % m), kk = (int)(p / (m * m));
            double lam = 0.0;
            const double w = M_PI / (2.0 * n);
            double s = sin(w * i);
            lam += 4.0 * s * s;
            s = sin(w * jj);
            lam += 4.0 * s * s;
            if (d == 3) {
                s = sin(w * kk);
                lam += 4.0 * s * s;
            }
            v /= lam;
        }
        y[p] = v;
    }
}

__global__ void k_scale_rhs(const double* __restrict__ f, double* __restrict__ b, int d, int n) {
    const int64_t m = n + 1;
    const int64_t total = d == 3 ? m * m * m : m * m;
    const double h2 = 1.0 / ((double)n * n);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % m), j = (int)((p / m) % m), k = d == 3 ? (int)(p / (m * m)) : 1;
        const bool in = i > 0 && i < n && j > 0 && j < n && k > 0 && k < (d == 3 ? n : 2);
        b[p] = in ? h2 * f[p] : 0.0;
    }
}

int flat_blocks(int64_t total) { return (int)std::min<int64_t>((total + 255) / 256, 152 * 16); }

}  // namespace
}  // namespace fft
}  // namespace gmg

using namespace gmg;
using namespace gmg::fft;

struct gmg_fft_s {
    int d = 3, n = 0, device = 0;
    int64_t lines = 0;
    cudaStream_t user_stream = nullptr, stream = nullptr;
    cudaEvent_t ev = nullptr;
    cufftHandle plan_x = 0, plan_yz = 0;
    bool have_x = false, have_yz = false;
    double* ext = nullptr;
    cufftDoubleComplex* spec = nullptr;
    double* work = nullptr;
};

extern "C" {

gmg_status gmg_fft_destroy(gmg_fft h) {
    if (!h) return GMG_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->have_x) cufftDestroy(h->plan_x);
    if (h->have_yz) cufftDestroy(h->plan_yz);
    cudaFree(h->ext);
    cudaFree(h->spec);
    cudaFree(h->work);
    if (h->ev) cudaEventDestroy(h->ev);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return GMG_OK;
}

gmg_status gmg_fft_create(int d, int n, void* cuda_stream, gmg_fft* out) {
    if (!out) {
        set_error("out is NULL");
        return GMG_ERR_ARG;
    }
    *out = nullptr;
    const int nmax = d == 2 ? 8192 : 1024;
    if ((d != 2 && d != 3) || n < 2 || n > nmax || (n & (n - 1))) {
        set_error("gmg_fft_create: d must be 2 or 3 and n a power of two within limits");
        return GMG_ERR_ARG;
    }
    gmg_fft h = new gmg_fft_s();
    h->d = d;
    h->n = n;
    h->user_stream = (cudaStream_t)cuda_stream;
    h->lines = d == 3 ? (int64_t)(n - 1) * (n - 1) : (n - 1);
    auto fail = [&](gmg_status s, const std::string& m) {
        set_error("gmg_fft_create: " + m);
        gmg_fft_destroy(h);
        return s;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(GMG_ERR_CUDA, "no device");
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming) != cudaSuccess)
        return fail(GMG_ERR_CUDA, "stream/event creation failed");
    const int64_t m = n + 1;
    const int64_t nodes = d == 3 ? m * m * m : m * m;
    if (cudaMalloc(&h->ext, sizeof(double) * h->lines * 2 * n) != cudaSuccess ||
        cudaMalloc(&h->spec, sizeof(cufftDoubleComplex) * h->lines * (n + 1)) != cudaSuccess ||
        cudaMalloc(&h->work, sizeof(double) * nodes) != cudaSuccess)
        return fail(GMG_ERR_ALLOC, "cudaMalloc failed");
    int len = 2 * n;
    int batch = (int)h->lines;
    // lines along x: contiguous extensions
    if (cufftPlanMany(&h->plan_x, 1, &len, nullptr, 1, len, nullptr, 1, n + 1, CUFFT_D2Z, batch) !=
        CUFFT_SUCCESS)
        return fail(GMG_ERR_CUDA, "cufftPlanMany (x) failed");
    h->have_x = true;
    // lines along y / z: element-major extensions (stride = lines)
    int inembed = len, onembed = n + 1;
    if (cufftPlanMany(&h->plan_yz, 1, &len, &inembed, batch, 1, &onembed, batch, 1, CUFFT_D2Z,
                      batch) != CUFFT_SUCCESS)
        return fail(GMG_ERR_CUDA, "cufftPlanMany (y/z) failed");
    h->have_yz = true;
    cufftSetStream(h->plan_x, h->stream);
    cufftSetStream(h->plan_yz, h->stream);
    *out = h;
    return GMG_OK;
}

gmg_status gmg_fft_solve(gmg_fft h, const double* f, double* u) {
    if (!h || !f || !u) {
        set_error("gmg_fft_solve: NULL argument");
        return GMG_ERR_ARG;
    }
    const int d = h->d, n = h->n;
    cudaStream_t s = h->stream;
    GMG_CUDA_TRY(cudaEventRecord(h->ev, h->user_stream));
    GMG_CUDA_TRY(cudaStreamWaitEvent(s, h->ev, 0));
    const int64_t m = n + 1;
    const int64_t nodes = d == 3 ? m * m * m : m * m;
    // b = h^2 f (interior), u = 0 on the boundary; work holds the transforms
    k_scale_rhs<<<flat_blocks(nodes), 256, 0, s>>>(f, h->work, d, n);
    GMG_CUDA_TRY(cudaMemsetAsync(u, 0, sizeof(double) * nodes, s));
    const int64_t ext_total = h->lines * 2 * n, out_total = h->lines * (n - 1);
    auto pass = [&](const double* src, double* dst, int axis, double scale, int eig) -> gmg_status {
        k_extend<<<flat_blocks(ext_total), 256, 0, s>>>(src, h->ext, d, n, axis, h->lines);
        if (cufftExecD2Z(axis == 0 ? h->plan_x : h->plan_yz, h->ext, h->spec) != CUFFT_SUCCESS) {
            set_error("cufftExecD2Z failed");
            return GMG_ERR_CUDA;
        }
        k_extract<<<flat_blocks(out_total), 256, 0, s>>>(h->spec, dst, d, n, axis, h->lines,
                                                        scale, eig);
        return GMG_OK;
    };
    gmg_status st;
    // forward DST on every axis, the last pass divided by lambda
    for (int a = 0; a < d; ++a)
        if ((st = pass(h->work, h->work, a, 1.0, a == d - 1)) != GMG_OK) return st;
    // inverse: the same transforms scaled by (2/n)^d, the last pass into u
    for (int a = 0; a < d; ++a) {
        const double sc = a == 0 ? std::pow(2.0 / n, d) : 1.0;
        if ((st = pass(h->work, a == d - 1 ? u : h->work, a, sc, 0)) != GMG_OK) return st;
    }
    GMG_CUDA_TRY(cudaGetLastError());
    GMG_CUDA_TRY(cudaStreamSynchronize(s));
    return GMG_OK;
}

}  // extern "C"
