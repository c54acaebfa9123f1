// Host entry points of the fused leg kernels (legs.cu; the algorithm is in
// legs.cuh).  Levels in the colour-split layout; u_in and u_out are
// different arrays of the fine level (the CTAs read u_in around their own
// columns while others write u_out).
#pragma once

#include <cuda_runtime.h>

#include "gmg_internal.cuh"

namespace gmg {
namespace legs {
// whether a 3D level of n intervals takes the leg kernels for storage T
// (float or df32): n a multiple of the column width and at least two columns
template <typename T>
bool applies(int d, int n);
// down leg on fine level F (coarse C): S half sweeps of u_in (colours
// alternating, the last black) into u_out, then q_c = 4 FW(sigma) of the red
// residual and u_c = 0 on the coarse interior; 2 <= S <= 4
template <typename T>
cudaError_t down(const Lay& F, const Lay& C, const T* u_in, T* u_out, const T* q, T* qc, T* uc,
                 int S, cudaStream_t s);
// up leg: u_out = S half sweeps (red first) of u_in + P e_c on the black
// nodes; 2 <= S <= 4
template <typename T>
cudaError_t up(const Lay& C, const Lay& F, const T* ec, const T* u_in, T* u_out, const T* q,
               int S, cudaStream_t s);
// nonzero once a leg kernel gave up waiting for its plane loads (sticky)
int fault();
}  // namespace legs
}  // namespace gmg
