// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "gmg.h"

namespace gmg {

// Thread-local message of the last failure (gmg_last_error).
void set_error(const std::string& msg);
const std::string& last_error();

struct Status {
    gmg_status code = GMG_OK;
    bool ok() const { return code == GMG_OK; }
};

#define GMG_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::gmg::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));       \
            return GMG_ERR_CUDA;                                                        \
        }                                                                               \
    } while (0)

// One grid of the hierarchy.  Arrays hold all (n+1)^d nodes, x fastest,
// boundary entries kept at zero.
struct Level {
    int n = 0;            // intervals per dimension
    int64_t nodes = 0;    // (n+1)^d
    double* u[2] = {nullptr, nullptr};  // iterate; u[1] = weighted-Jacobi ping-pong partner
    double* q = nullptr;  // scaled right-hand side q = h^2 f / (2d)
    double* r = nullptr;  // scaled residual sigma = q + A'-neighbour sum / (2d) - u
};

// FP64 level kernels (fp64_kernels.cu).  All take interior extents n and
// work in the scaled variables: q = b / (2d), sigma = (b - A'u) / (2d).
namespace fp64 {
void prepare(int d, int n, const double* f, double* q, double* u, cudaStream_t s);
void rb_half(int d, int n, double* u, const double* q, int color, cudaStream_t s);
void wj_sweep(int d, int n, const double* u_in, double* u_out, const double* q, double omega,
              cudaStream_t s);
void residual(int d, int n, const double* u, const double* q, double* r, bool red_only,
              cudaStream_t s);
void restrict_fw(int d, int n, const double* r, double* qc, double* uc, bool red_only,
                 bool exact_coarsest, cudaStream_t s);
void prolong_add(int d, int nc, const double* uc, double* u, cudaStream_t s);
int resnorm_partials(int d, int n);  // number of partial sums resnorm writes
void resnorm(int d, int n, const double* u, const double* q, double* partial, double* out,
             cudaStream_t s);
}  // namespace fp64

}  // namespace gmg
