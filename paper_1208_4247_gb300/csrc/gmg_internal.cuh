// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "df.cuh"
#include "gmg.h"

namespace gmg {

// Thread-local message of the last failure (gmg_last_error).
void set_error(const std::string& msg);
const std::string& last_error();

#define GMG_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::gmg::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));       \
            return GMG_ERR_CUDA;                                                        \
        }                                                                               \
    } while (0)

// Node addressing of a level array.  Dense (he == 0): node (i, j, k) at
// k*sz + j*sy + i with sy = n+1, x fastest -- the caller's layout, used by
// every FP64 array.  Colour-split (he > 0; the FP32/BF16 inner hierarchies):
// each row stores its even-x nodes first (x/2 at 0..n/2) and its odd-x
// nodes from offset he ((x-1)/2 at he..he+n/2-1), so the nodes of one colour
// in a row are contiguous and a half sweep reads and writes only the bytes
// of the colours it uses; sy is then the padded row stride.
struct Lay {
    int n = 0;
    int he = 0;
    int64_t sy = 0, sz = 0;
};
inline Lay dense_lay(int d, int n) {
    Lay L;
    L.n = n;
    L.sy = n + 1;
    L.sz = d == 3 ? L.sy * (n + 1) : 0;
    return L;
}
// halves padded to multiples of 8 elements (16 bytes in BF16, 32 in FP32)
inline Lay split_lay(int d, int n) {
    Lay L;
    L.n = n;
    L.he = (n / 2 + 1 + 7) / 8 * 8;
    L.sy = L.he + (n / 2 + 7) / 8 * 8;
    L.sz = d == 3 ? L.sy * (n + 1) : 0;
    return L;
}
// elements of a level array with layout L
inline int64_t lay_elems(int d, const Lay& L) { return d == 3 ? L.sz * (L.n + 1) : L.sy * (L.n + 1); }

// One grid of a hierarchy in storage type T.  Arrays hold all (n+1)^d
// nodes, x fastest, boundary entries kept at zero.
template <typename T>
struct Level {
    int n = 0;            // intervals per dimension
    int64_t nodes = 0;    // (n+1)^d
    T* u[2] = {nullptr, nullptr};  // iterate; u[1] = weighted-Jacobi ping-pong partner
    T* q = nullptr;       // scaled right-hand side q = h^2 f / (2d)
    T* r = nullptr;       // scaled residual sigma = q + A'-neighbour sum / (2d) - u
    Lay lay;              // addressing of u, q, r
};

// Level kernels, explicitly instantiated for double (fp64_kernels.cu) and
// float / __nv_bfloat16 (mixed_kernels.cu); definitions in level_kernels.cuh.
namespace lk {
// rows per diagonal walker of the FP64 3D half sweep; GMG_RB_WALK=0 turns
// the walkers off (fp64_kernels.cu reads it once)
constexpr int kWalk = 4;
bool rb_walk_enabled();
// Launchers on a level with layout L (restriction: fine F -> coarse C;
// prolongation: coarse C -> fine F).
// exact (FP64 3D only): 1/(2d) = 1/6 carried as a double-double, an
// unbiased Gauss-Seidel value and residual (level_kernels.cuh, gs_value)
template <typename T>
void rb_half(int d, const Lay& L, T* u, const T* q, int color, cudaStream_t s, bool exact = false);
template <typename T>
void wj_sweep(int d, const Lay& L, const T* u_in, T* u_out, const T* q, double omega,
              cudaStream_t s);
template <typename T>
void residual(int d, const Lay& L, const T* u, const T* q, T* r, bool red_only, cudaStream_t s,
              bool exact = false);
template <typename T>
void restrict_fw(int d, const Lay& F, const Lay& C, const T* r, T* qc, T* uc, bool red_only,
                 bool exact_coarsest, cudaStream_t s);
// black_only: correct the black fine nodes only (valid when a red half sweep
// follows, which overwrites every red node without reading it)
template <typename T>
void prolong_add(int d, const Lay& C, const Lay& F, const T* uc, T* u, cudaStream_t s,
                 bool black_only = false);

// The paper's own variant on dense FP64 levels: one colour of the 4/8-colour
// Gauss-Seidel, the 7/15-point restriction, the diagonal prolongation.
template <typename T>
void mc_sweep(int d, const Lay& L, T* u, const T* q, int color, cudaStream_t s);
template <typename T>
void restrict_paper(int d, const Lay& F, const Lay& C, const T* r, T* qc, T* uc,
                    bool exact_coarsest, cudaStream_t s);
template <typename T>
void prolong_paper(int d, const Lay& C, const Lay& F, const T* uc, T* u, cudaStream_t s);

// The same on dense levels given by n.
template <typename T>
inline void rb_half(int d, int n, T* u, const T* q, int color, cudaStream_t s,
                    bool exact = false) {
    rb_half<T>(d, dense_lay(d, n), u, q, color, s, exact);
}
template <typename T>
inline void residual(int d, int n, const T* u, const T* q, T* r, bool red_only, cudaStream_t s,
                     bool exact = false) {
    residual<T>(d, dense_lay(d, n), u, q, r, red_only, s, exact);
}
template <typename T>
inline void restrict_fw(int d, int n, const T* r, T* qc, T* uc, bool red_only,
                        bool exact_coarsest, cudaStream_t s) {
    restrict_fw<T>(d, dense_lay(d, n), dense_lay(d, n / 2), r, qc, uc, red_only, exact_coarsest,
                   s);
}
template <typename T>
inline void prolong_add(int d, int nc, const T* uc, T* u, cudaStream_t s,
                        bool black_only = false) {
    prolong_add<T>(d, dense_lay(d, nc), dense_lay(d, 2 * nc), uc, u, s, black_only);
}
}  // namespace lk

// FP64 preparation and stopping-test norm (fp64_kernels.cu).
namespace fp64 {
// u_nonzero (may be NULL; zeroed by the caller): set to 1 when an interior
// entry of u has a bit pattern other than +0.0.
void prepare(int d, int n, const double* f, double* q, double* u, cudaStream_t s,
             int* u_nonzero = nullptr);
int resnorm_partials(int d, int n);
// dst = src on every node of a (n+1)^d grid; src / dst row and plane pitches
// in elements (x contiguous)
void copy_strided(int d, int n, const double* src, int64_t ssy, int64_t ssz, double* dst,
                  int64_t dsy, int64_t dsz, cudaStream_t s);
// sum of sigma^2 into *out; sigma_out (may be NULL) also receives sigma;
// red_only (ignored with sigma_out) sums red nodes only, valid right after a
// black half sweep of level 0 (black sigma is then exactly zero)
void resnorm(int d, int n, const double* u, const double* q, double* partial, double* out,
             cudaStream_t s, double* sigma_out = nullptr, bool red_only = false);
__global__ void k_sum_partials(const double* partial, int count, double* out);
// The stopping-test norm of a red-black cycle fused with the next cycle's
// first red half sweep (3D FP64 levels the diagonal walkers take, unless
// GMG_NORM_AHEAD=0): the red-only norm of u into *out (norm = true; plus
// (may be NULL): *out = *plus + that norm) and one red half sweep of u, the
// old red values kept in save.  red_restore puts them back (u = save on the
// red interior nodes).  resnorm_black: the black nodes' sigma^2 sum (the
// other half of a first norm whose red half red_ahead sums).
bool red_ahead_applies(int d, int n);
void red_ahead(int n, double* u, const double* q, double* save, double* partial, double* out,
               bool norm, cudaStream_t s, const double* plus = nullptr);
void resnorm_black(int n, const double* u, const double* q, double* partial, double* out,
                   cudaStream_t s);
void red_restore(int n, double* u, const double* save, cudaStream_t s);
}  // namespace fp64

// Outer FP64 kernels of iterative refinement (mixed_kernels.cu).
namespace mixed {
int outer_partials(int d, int n);
// q_in, e: the inner level-0 arrays, layout `in` (dense u, q: FP64, n = in.n).
// e_init (may be NULL) receives the inner iterate after the first red half
// sweep from e = 0: sigma on the red nodes, 0 on the black ones.
// resid (double-float only; may be NULL): the black nodes' sigma minus its
// double-float value, for the first outer_red_update after this residual
// (*resid_flag set here, cleared there).  qnorm_out (may be NULL): the sum
// of q^2, the squared norm of the residual of u = 0 (partial must then hold
// 2 outer_partials entries).
// u_nonzero (may be NULL): fp64::prepare's flag; where it is 0 (u = +0.0
// everywhere) sigma = q + 0.0 exactly (the stencil's value for a zero
// iterate, bit for bit), formed without the FP64 stencil.
template <typename T>
void outer_residual(int d, const Lay& in, const double* u, const double* q, T* q_in,
                    double* partial, double* out, cudaStream_t s, T* e_init = nullptr,
                    float* resid = nullptr, int* resid_flag = nullptr,
                    double* qnorm_out = nullptr, const int* u_nonzero = nullptr);
template <typename T>
void update(int d, const Lay& in, double* u, const T* e, cudaStream_t s);
// After red-black double-float inner cycles: the last black Gauss-Seidel
// values formed in triple-float and added to u in FP64 (they replace the
// inner cycle's last level-0 black half sweep), u += e on the red nodes, and
// the next outer residual on the red nodes only (the black one is zero to
// FP64 rounding): q_in = e = sigma on red nodes, 0 on black ones; sigma^2
// sum into *out.  Two kernels and the sum.
// skip (may be NULL): the kernels do nothing while *skip is nonzero.
template <typename T>
void outer_red_update(int d, const Lay& in, double* u, const double* q, T* q_in, T* e,
                      double* partial, double* out, cudaStream_t s, const float* resid = nullptr,
                      int* resid_flag = nullptr, const int* skip = nullptr);

// Steps of several double-float cycles (mixed_kernels.cu), on the inner
// level 0 (colour-split layout `in`, red = i+j+k even).  skip / flag: device
// flags read by every thread; a launch does nothing while *skip is nonzero
// (while *flag is zero for the restore).
// The level's black half sweep.
void df_black_half(int d, const Lay& in, df32* e, const df32* q_in, const int* skip,
                   cudaStream_t s);
// The next cycle's first red half sweep with the stopping-test norm folded
// in: e = the red Gauss-Seidel values, r = their change (the red residual),
// per block the sum of its squares into partial; returns the partial count
// (at most outer_partials(d, n)).
int df_red_ahead(int d, const Lay& in, df32* e, const df32* q_in, df32* r, double* partial,
                 const int* skip, cudaStream_t s);
// e -= r on the red nodes: undoes df_red_ahead.
void df_red_restore(int d, const Lay& in, df32* e, const df32* r, const int* flag,
                    cudaStream_t s);
}  // namespace mixed

// Fused red-black sweep (fused.cu, 3D FP32): u_out = one full sweep of u_in
// (red then black), one pass over memory.
namespace fused {
void rb_sweep3_f32(int n, const float* uin, float* uout, const float* q, cudaStream_t s);
}  // namespace fused

// Persistent single-CTA tail (tail.cu): the V-cycle on levels n_top, n_top/2,
// ... (levels of them) in shared memory; u_top in/out, q_top in.
namespace tail {
size_t smem_bytes(int d, int n_top, int levels, int smoother, size_t elem);
// top: layout of u_top / q_top in global memory (n_top = top.n)
// exact_top: the top level is level 0 of a plain FP64 3D hierarchy, whose
// last pre-smoothing half sweep and residual use the unbiased value
// (level_kernels.cuh, gs_value), as the grid kernels there do
template <typename T>
cudaError_t launch(int d, const Lay& top, int levels, T* u_top, const T* q_top, int smoother,
                   double omega, int nu1, int nu2, int coarse_sweeps, cudaStream_t s,
                   bool exact_top = false);
// The same on the levels' own dense arrays (n[l], u[l], q[l], r[l] for the
// `levels` levels from the first one down), one cooperative launch of
// `blocks` CTAs (grid_blocks: one wave; 0 when the device cannot) with grid
// barriers between the steps on levels with n > cta_n and one CTA below;
// cluster > 0 (at most 16): instead one thread-block cluster of that many
// CTAs with the hardware cluster barrier (bar unused).
// bar: grid_bar_bytes() of device memory, zeroed once; its fault flag
// (grid_fault) is set if a barrier wait ran past its limit (the results of
// that launch are then invalid).  Red-black smoothing only.
template <typename T>
int grid_blocks(int d);
template <typename T>
cudaError_t launch_grid(int d, int levels, const int* n, T* const* u, T* const* q, T* const* r,
                        int smoother, double omega, int nu1, int nu2, int coarse_sweeps,
                        int cta_n, void* bar, int blocks, cudaStream_t s, int cluster = 0);
size_t grid_bar_bytes();
int grid_fault(const void* bar);
}  // namespace tail

// Learned-smoother network kernels (learned.cu): z = conv1(x) (8 channel
// planes of (n+1)^d floats), out = / += / -= conv2(relu(z)) for mode 0/1/2.
// W: 2 x 8 x 3^d BF16-rounded floats on the device.
namespace learned {
void conv1(int d, int n, const double* x, float* z, const float* W, cudaStream_t s);
void conv2(int d, int n, const float* z, double* out, int mode, const float* W, cudaStream_t s);
// u += N(sigma) (mode 1) or u = N(sigma) (mode 0) with the fused tensor-core
// kernel (BF16 operands: sigma, weights and hidden activations; FP32 sums)
void conv_tc(int d, int n, const double* sigma, double* u, int mode, const float* W,
             cudaStream_t s);
// dev = BF16 rounding of the host weights (scratch: 2 x 8 x 3^d device floats)
void upload_weights(int d, const float* host, float* dev, float* scratch, cudaStream_t s);
}  // namespace learned

}  // namespace gmg
