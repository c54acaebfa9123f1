// Measured FP64 pipe rate (gmg_measure_fp64_rate): the roofline peak of the
// FP64-bound level kernels, taken on the running GPU instead of a nominal
// figure.  Every thread runs eight independent dependency chains of one
// instruction kind (DFMA or DADD), so the pipe, not the latency of one
// chain, limits the rate; the grid fills every SM several times over.
#include <string>

#include "gmg_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_fp64_chains(double* __restrict__ sink, int iters,
                                                          double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = KIND == 0 ? fma(x[c], a, b) : x[c] + b;
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5678) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains
}

}  // namespace

extern "C" gmg_status gmg_measure_fp64_rate(int kind, double* inst_per_s, void* cuda_stream) {
    using gmg::set_error;
    if ((kind != 0 && kind != 1) || !inst_per_s) {
        set_error("kind must be 0 (DFMA) or 1 (DADD) and inst_per_s non-NULL");
        return GMG_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    GMG_CUDA_TRY(cudaGetDevice(&dev));
    GMG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    const int iters = 2048;
    // the DFMA chains approach b / (1 - a) = 0.1, the DADD chains grow by
    // iters * b: both stay finite and normal
    const double a = 0.999999, b = kind == 0 ? 1e-7 : 1e-9;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GMG_CUDA_TRY(cudaEventCreate(&e0));
    GMG_CUDA_TRY(cudaEventCreate(&e1));
    auto launch = [&]() {
        if (kind == 0)
            k_fp64_chains<0><<<blocks, kThreads, 0, st>>>(nullptr, iters, a, b);
        else
            k_fp64_chains<1><<<blocks, kThreads, 0, st>>>(nullptr, iters, a, b);
    };
    launch();  // warm-up (clocks, instruction cache)
    cudaEventRecord(e0, st);
    constexpr int reps = 5;
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_error(std::string("gmg_measure_fp64_rate: ") + cudaGetErrorString(e));
        return GMG_ERR_CUDA;
    }
    const double inst = (double)reps * blocks * kThreads * (double)iters * kChains;
    *inst_per_s = inst / (ms * 1e-3);
    return GMG_OK;
}
