// C ABI of the solver (include/gmg.h): handle lifetime, the V-cycle schedule
// of Algorithm 1 captured once into a CUDA graph, and the stopping loop of
// Algorithm 3 with every level on the device.  Two forms share the
// schedule: plain FP64 cycles, and FP32 / BF16 cycles inside FP64 iterative
// refinement.
#include <algorithm>
#include <cmath>
#include <limits>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <type_traits>
#include <utility>
#include <vector>

#include "gmg_internal.cuh"
#include "legs_api.h"
#include "timing.cuh"

namespace gmg {

namespace {
thread_local std::string g_err;
}
void set_error(const std::string& msg) { g_err = msg; }
const std::string& last_error() { return g_err; }

}  // namespace gmg

using namespace gmg;
using bf16 = __nv_bfloat16;

namespace gmg {
// Device side of the stopping loop (Algorithm 3's test after each cycle):
// parameters written by the host before the loop graph runs, the cycle
// count and the relative residual history written by the device.
struct LoopState {
    double res0, rtol, res;  // initial and latest ||h^2 f - A'u|| (scaled), rtol
    int cap, stop, it, pad;  // cycle cap; stop on rtol; cycles run so far
    double hist[1];          // [cap]: relative residual after each cycle
};
constexpr size_t kLoopHeader = offsetof(LoopState, hist);

// Double-float refinement in steps of several cycles (chain_on): the device's
// plan for the cycle that runs now, and the step it belongs to.
struct ChainState {
    int step_it;   // cycles of the current step before this one
    int kmax;      // cycles per step after a solve's first step (which has one)
    int skip_mid;  // the cycle continues the step: black half sweep, red half sweep + norm
    int skip_end;  // the cycle ends the step: the FP64 red update, residual and norm
    int restore;   // the step ends after the norm said stop: undo that red half sweep
    int counted;   // the norm inside the step counted this cycle
};
}  // namespace gmg

struct gmg_handle_s {
    gmg_config cfg{};
    int device = 0;
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;  // owned, non-blocking; ordered after user_stream per call
    cudaEvent_t ev = nullptr;
    // plain form: the whole FP64 hierarchy; refinement forms: level 0 only
    // (u = the caller's iterate, q = FP64 scaled right-hand side)
    std::vector<Level<double>> lv;
    std::vector<Level<float>> lvf;  // FP32 inner hierarchy (GMG_FP32_IR)
    std::vector<Level<bf16>> lvb;   // BF16 inner hierarchy (GMG_BF16_IR)
    std::vector<Level<df32>> lvd;   // double-float inner hierarchy (GMG_DF_IR)
    double* partial = nullptr;
    // double-float red-only refinement: the black remainder of the starting
    // outer residual and its flag (mixed::outer_residual / outer_red_update)
    float* resid_b = nullptr;
    int* resid_flag = nullptr;
    // the steps of this solve use the full outer residual (step_full): a
    // double-float solve whose starting residual exceeds twice that of u = 0
    // (section 4.11); the captured graphs' mode (graph_step_full)
    bool step_full = false;
    bool graph_step_full = false;
    double* d_res2 = nullptr;
    double* h_res2 = nullptr;  // pinned
    cudaGraphExec_t graph = nullptr;
    const double* graph_u = nullptr;  // level-0 iterate baked into the graph
    cudaGraphExec_t fmg_graph = nullptr;  // GMG_FMG: the first cycle of a solve
    // while-node graph around one step: the stopping test runs on the device
    // (k_loop_test), one launch and one sync per solve (timing off only)
    cudaGraphExec_t loop_graph = nullptr;
    cudaGraphConditionalHandle loop_cond = 0;
    int loop_kernels = 0;         // kernel launches per loop iteration
    int loop_cap = 0;             // history capacity of d_loop
    LoopState* d_loop = nullptr;
    LoopState* h_loop = nullptr;  // pinned
    bool device_loop = true;      // GMG_DEVICE_LOOP=0 at create: host loop
    // double-float refinement: cycles per step after the first (chain_on;
    // GMG_DF_STEP_CYCLES at create, 1 = one cycle per step), device plan
    int chain_k = 8;
    ChainState* d_chain = nullptr;
    ChainState* h_chain = nullptr;  // pinned
    // refinement forms: set by the start's prepare when the starting iterate
    // has a nonzero interior entry (else the first outer residual is q)
    int* d_unz = nullptr;
    bool graph_chain = false;       // the captured graphs are chain bodies
    int fmg_kernels = 0;
    std::vector<KernelTimer::Pending> fmg_pending;
    std::vector<double> hist;
    double* f_stage = nullptr;  // device copies for gmg_solve_host
    double* u_stage = nullptr;
    std::vector<void*> allocs;
    KernelTimer timer;  // launch accounting and optional per-kernel event timing
    bool fused_rb = false;  // GMG_FUSED_RB=1 at create: fused FP32 3D red-black sweeps
    bool inner_ahead = true;  // GMG_INNER_AHEAD=0 at create: memset e + first red half sweep
    bool outer_red = true;    // GMG_OUTER_RED=0 at create: full outer residual (double-float)
    // plain red-black form: the stopping-test norm runs fused with the next
    // cycle's first level-0 red half sweep (norm_ahead_ok)
    bool ahead = false;
    int tail_max = 0;       // GMG_TAIL_N at create: largest tail level n (0 = default)
    // fused leg kernels (legs.cu) on large 3D levels of the red-black inner
    // hierarchies.  legs_mode 1 (default): FP32 levels with n >= 512, where
    // they beat the unfused kernels; 2 (GMG_FUSED_LEGS=1 at create): FP32
    // and double-float levels with n >= 128; 0 (GMG_FUSED_LEGS=0): off.
    // GMG_LEG_NMIN overrides the smallest level n.
    int legs_mode = 1;
    int leg_nmin = 0;
    int leg_nmax = 0;  // GMG_LEG_NMAX: the largest level n (0 = no bound)
    // grid tail (tail::launch_grid): the levels with n <= gtail_nmax (and the
    // small ones, n <= gtail_cta_n in one CTA) in one cooperative launch of
    // gtail_blocks CTAs; GMG_GRID_TAIL_N at create (default 0 = off: slower
    // than the per-level kernels and the single-CTA tail on GB300),
    // GMG_GRID_TAIL_CTA_N
    int gtail_nmax = 0;
    int gtail_cta_n = 8;
    int gtail_blocks = 0;
    int gtail_cluster = 0;  // GMG_GRID_TAIL_CLUSTER=c: one cluster of c CTAs instead
    void* gtail_bar = nullptr;
    bool gtail_used = false;
    bool legs_used = false;
    // learned smoother (GMG_LEARNED): per level BF16-rounded weights on the
    // device (NULL: red-black GS on that level) and the hidden-layer buffer
    std::vector<float*> lw, lz;
    float* lw_scratch = nullptr;
};

namespace {

bool is_pow2(int v) { return v >= 2 && (v & (v - 1)) == 0; }
int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}
int64_t nodes_of(int d, int n) {
    int64_t m = n + 1;
    return d == 3 ? m * m * m : m * m;
}

gmg_status check_cfg(const gmg_config* c) {
    if (!c) {
        set_error("config is NULL");
        return GMG_ERR_ARG;
    }
    if (c->d != 2 && c->d != 3) {
        set_error("d must be 2 or 3");
        return GMG_ERR_ARG;
    }
    const int nmax = c->d == 2 ? 16384 : 1024;
    if (!is_pow2(c->n) || c->n > nmax) {
        set_error("n must be a power of two in [2, " + std::to_string(nmax) + "]");
        return GMG_ERR_ARG;
    }
    const int lmax = ilog2(c->n);
    if (c->levels < 0 || c->levels > lmax) {
        set_error("levels must be 0 (all) or 1.." + std::to_string(lmax));
        return GMG_ERR_ARG;
    }
    if (c->smoother != GMG_WJACOBI && c->smoother != GMG_RBGS && c->smoother != GMG_LEARNED &&
        c->smoother != GMG_MCGS) {
        set_error("unknown smoother");
        return GMG_ERR_ARG;
    }
    if (c->transfer != GMG_TRANSFER_FW && c->transfer != GMG_TRANSFER_PAPER) {
        set_error("unknown transfer");
        return GMG_ERR_ARG;
    }
    if ((c->smoother == GMG_MCGS || c->transfer == GMG_TRANSFER_PAPER) &&
        (c->precision != GMG_FP64 || c->smoother == GMG_LEARNED)) {
        set_error("the paper's smoother and transfers run in the plain FP64 form");
        return GMG_ERR_UNSUPPORTED;
    }
    if (c->smoother == GMG_LEARNED && c->precision != GMG_FP64) {
        set_error("the learned smoother runs in the plain FP64 form only");
        return GMG_ERR_UNSUPPORTED;
    }
    if (!(c->omega > 0.0 && c->omega < 2.0)) {
        set_error("omega must lie in (0, 2)");
        return GMG_ERR_ARG;
    }
    if (c->nu1 < 0 || c->nu2 < 0 || c->nu1 > 16 || c->nu2 > 16) {
        set_error("nu1, nu2 must lie in 0..16");
        return GMG_ERR_ARG;
    }
    if (c->cycle != GMG_VCYCLE && c->cycle != GMG_FMG) {
        set_error("cycle must be GMG_VCYCLE or GMG_FMG");
        return GMG_ERR_ARG;
    }
    if (c->cycle == GMG_FMG && (c->precision != GMG_FP64 || c->smoother == GMG_LEARNED)) {
        set_error("GMG_FMG runs in the plain FP64 form with GS or Jacobi smoothing");
        return GMG_ERR_UNSUPPORTED;
    }
    if (c->precision != GMG_FP64 && c->precision != GMG_FP32_IR && c->precision != GMG_BF16_IR &&
        c->precision != GMG_DF_IR) {
        set_error("unknown precision");
        return GMG_ERR_UNSUPPORTED;
    }
    if (c->precision != GMG_FP64 && (c->inner_cycles < 1 || c->inner_cycles > 64)) {
        set_error("inner_cycles must lie in 1..64");
        return GMG_ERR_ARG;
    }
    if (c->maxit < 0 || c->maxit > 100000) {
        set_error("maxit must lie in 0..100000");
        return GMG_ERR_ARG;
    }
    if (c->coarse_sweeps < 0 || c->coarse_sweeps > 100000) {
        set_error("coarse_sweeps must lie in 0..100000");
        return GMG_ERR_ARG;
    }
    return GMG_OK;
}

template <typename T>
gmg_status dev_alloc(gmg_handle h, T** p, int64_t count) {
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return GMG_ERR_ALLOC;
    }
    h->allocs.push_back(*p);
    e = cudaMemsetAsync(*p, 0, sizeof(T) * count, h->stream);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        return GMG_ERR_CUDA;
    }
    return GMG_OK;
}

gmg_status check_device_ptr(const void* p, const char* name) {
    if (!p) {
        set_error(std::string(name) + " is NULL");
        return GMG_ERR_LAYOUT;
    }
    if (((uintptr_t)p) % alignof(double) != 0) {
        set_error(std::string(name) + " is not 8-byte aligned");
        return GMG_ERR_LAYOUT;
    }
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess || (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        set_error(std::string(name) + " is not a device pointer");
        return GMG_ERR_LAYOUT;
    }
    return GMG_OK;
}

int num_levels(const gmg_config& c) { return c.levels > 0 ? c.levels : ilog2(c.n); }

enum Kind {
    K_RB_HALF, K_WJ, K_RESIDUAL, K_RESTRICT, K_PROLONG, K_RESNORM, K_COPY, K_OUTER_RES,
    K_UPDATE, K_MEMSET, K_CONV1, K_CONV2, K_TAIL, K_RB_FUSED, K_MC_SWEEP, K_RESTRICT_PAPER,
    K_PROLONG_PAPER, K_NORM_AHEAD, K_OUTER_RED, K_LEG_DOWN, K_LEG_UP, K_RESTORE, K_COUNT
};
const char* kKindName[K_COUNT] = {"rb_half",     "wj_sweep", "residual", "restrict",
                                  "prolong_add", "resnorm",  "copy",     "outer_residual",
                                  "update",      "memset",   "conv1",    "conv_tc_update", "tail",
                                  "rb_sweep_fused", "mc_sweep", "restrict_paper",
                                  "prolong_paper", "resnorm_red_sweep", "outer_red_update",
                                  "leg_down", "leg_up", "red_restore"};
const char* kPrecSuffix[4] = {"", "_f32", "_bf16", "_df"};

template <typename T>
int prec_of();
template <>
int prec_of<double>() { return 0; }
template <>
int prec_of<float>() { return 1; }
template <>
int prec_of<bf16>() { return 2; }
template <>
int prec_of<df32>() { return 3; }

// Arithmetic model per launch: the operation's algorithmic instruction count
// in the kernel's compute precision (FP64 for double storage and for the
// refinement kernels, FP32 otherwise; a red-black node update counts its
// 2d-1 adds + 1 fma even where the diagonal walkers share one add between
// two nodes) and algorithmic DRAM bytes (each value the operation needs read
// once, each value it produces written once) with w bytes per stored value.
std::pair<double, double> model(int kind, int d, int n, bool red_only, double w, int sweeps) {
    const double N = std::pow((double)(n - 1), d);
    const int nc = n / 2;
    const double Nc = std::pow((double)std::max(nc - 1, 0), d);
    const double cells = std::pow((double)nc, d);
    const bool t = d == 3;
    switch (kind) {
        case K_RB_HALF: return {N / 2 * (t ? 6 : 4), N / 2 * 3 * w};
        case K_WJ: return {N * (t ? 8 : 6), N * 3 * w};
        case K_RESIDUAL:
            return red_only ? std::make_pair(N / 2 * (t ? 7 : 5), N * 2 * w)
                            : std::make_pair(N * (t ? 7 : 5), N * 3 * w);
        case K_RESTRICT:
            return red_only ? std::make_pair(Nc * (t ? 13 : 4), N / 2 * w + Nc * 2 * w)
                            : std::make_pair(Nc * (t ? 27 : 8), N * w + Nc * 2 * w);
        case K_PROLONG:  // red_only here: black fine nodes only
            return red_only ? std::make_pair(cells * (t ? 13 : 4), Nc * w + N * w)
                            : std::make_pair(cells * (t ? 20 : 8), Nc * w + N * 2 * w);
        case K_RESNORM:
            return red_only ? std::make_pair(N / 2 * (t ? 8 : 6), N * 12)
                            : std::make_pair(N * (t ? 8 : 6), N * 16);
        case K_COPY: return {0.0, N * 2 * w};
        case K_OUTER_RES:  // red_only here: also writes the inner iterate (e_init)
            return {N * (t ? 8 : 6), N * (16 + (red_only ? 2 : 1) * w)};
        case K_UPDATE: return {N, N * (16 + w)};
        case K_MEMSET: return {0.0, N * w};
        case K_CONV1: return {N * 8 * (t ? 27 : 9), N * (w + 32)};  // FP32 FMAs
        case K_CONV2: return {N * 16 * (t ? 27 : 9), N * 3 * w};  // both convs, u read+write
        case K_TAIL: return {N * (t ? 40 : 30) * 8.0 / 7.0, N * 2 * w};
        case K_RB_FUSED: return {N * (t ? 6 : 4), N * 3 * w};  // read u, q; write u
        case K_MC_SWEEP:  // one of 2^d colours: the colour's nodes updated
            return {N / (t ? 8 : 4) * (t ? 6 : 4), N / (t ? 8 : 4) * (t ? 8 : 6) * w};
        case K_RESTRICT_PAPER: return {Nc * (t ? 16 : 8), N * w + Nc * 2 * w};
        case K_PROLONG_PAPER: return {cells * (t ? 14 : 6), Nc * w + N * 2 * w};
        case K_NORM_AHEAD:  // red nodes: sigma^2 and the update; read u, q (red); write u, save
            return {N / 2 * (t ? 8 : 6), N * 2.5 * w};
        case K_OUTER_RED:  // black: triple-float GS value into u (3 FP64 adds), e = q_in = 0;
                           // red: u += e, sigma, q_in = e = sigma; u, e read on all nodes
            return {N / 2 * (t ? 14.25 : 13), N * (16 + w) + N / 2 * (8 + 4 * w)};
        case K_LEG_DOWN:  // `sweeps` half sweeps, red residual, restriction: read u, q; write u, q_c, u_c
            return {N / 2 * 6 * sweeps + N / 2 * 7 + Nc * 13, (N * 3 + Nc * 2) * w};
        case K_LEG_UP:  // black prolongation + `sweeps` half sweeps: read u_c, u, q; write u
            return {cells * 13 + N / 2 * 6 * sweeps, (N * 3 + Nc) * w};
        case K_RESTORE:  // red nodes: u -= saved change; read u, r; write u
            return {N / 2, N / 2 * 3 * w};
    }
    return {0.0, 0.0};
}

// Enqueue one kernel (launch() issues it on h->stream), timed when timing
// is on; `kernels` = kernel launches launch() makes.
template <class F>
void timed(gmg_handle h, int kind, int level, int prec, int n, bool red_only, F&& launch,
           int kernels = 1, int sweeps = 0) {
    const double w = prec == 0 || prec == 3 ? 8.0 : prec == 1 ? 4.0 : 2.0;
    auto m = model(kind, h->cfg.d, n, red_only, w, sweeps);
    h->timer.run(h->stream, std::string(kKindName[kind]) + kPrecSuffix[prec], level, m.first,
                 m.second, kernels, launch);
}

// FP32 3D red-black with GMG_FUSED_RB=1: one fused kernel per sweep
// (ping-pong buffers).  Off by default: on GB300 the fused kernel is bound by
// per-node instruction issue and is slower than the two half-sweep kernels.
template <typename T>
bool use_fused_rb(gmg_handle h) {
    return std::is_same<T, float>::value && h->fused_rb && h->cfg.smoother == GMG_RBGS &&
           h->cfg.d == 3;
}

// The next operation on the level is `sweeps` red-black sweeps starting with
// a red half sweep (which overwrites every red node without reading it).
template <typename T>
bool red_sweep_next(gmg_handle h, int sweeps) {
    return h->cfg.smoother == GMG_RBGS && sweeps > 0 && !use_fused_rb<T>(h);
}

bool learned_level(gmg_handle h, int l) {
    return h->cfg.smoother == GMG_LEARNED && l < (int)h->lw.size() && h->lw[l];
}

// One learned smoothing sweep on FP64 level l: sigma = (b - A'u)/(2d),
// u += conv2(relu(conv1(sigma))).  sigma_ready: L.r already holds sigma of
// the current u (level 0 after the stopping-test norm).
void learned_sweep(gmg_handle h, Level<double>& L, int l, bool sigma_ready) {
    const int d = h->cfg.d;
    if (!sigma_ready)
        timed(h, K_RESIDUAL, l, 0, L.n, false,
              [&] { lk::residual<double>(d, L.n, L.u[0], L.q, L.r, false, h->stream); });
    timed(h, K_CONV2, l, 0, L.n, false,
          [&] { learned::conv_tc(d, L.n, L.r, L.u[0], 1, h->lw[l], h->stream); });
}

// Enqueue `sweeps` smoothing sweeps on level l; cur tracks which u buffer
// holds the iterate (weighted Jacobi alternates).
// Level 0 of a plain FP64 handle whose level 0 is learned: the stopping-test
// norm leaves sigma of the cycle's starting iterate in lv[0].r.
bool sigma_carried(gmg_handle h) {
    return h->cfg.precision == GMG_FP64 && learned_level(h, 0) && h->cfg.nu1 > 0;
}

// backward: post-smoothing (Relax_backward), which takes the colours of the
// multi-colour smoother in decreasing order.
// first_red_done: the first red half sweep already ran (fused with the
// previous step's stopping-test norm).
// exact_last: the last half sweep (a black one) uses the unbiased FP64 3D
// Gauss-Seidel value (lk::gs_value), as the level-0 pre-smoothing before the
// unbiased red-only residual must (the black residual then stays exactly 0).
// skip_last_black: the last black half sweep is left to a later kernel
// (mixed::outer_red_update forms it in triple-float).
template <typename T>
void relax(gmg_handle h, std::vector<Level<T>>& lv, int l, int sweeps, int& cur,
           bool sigma_ready = false, bool backward = false, bool first_red_done = false,
           bool exact_last = false, bool skip_last_black = false) {
    Level<T>& L = lv[l];
    const int d = h->cfg.d;
    const int p = prec_of<T>();
    for (int s = 0; s < sweeps; ++s) {
        if constexpr (std::is_same<T, double>::value) {
            if (h->cfg.smoother == GMG_MCGS) {
                const int ncol = d == 3 ? 8 : 4;
                for (int t = 0; t < ncol; ++t) {
                    const int color = backward ? ncol - 1 - t : t;
                    timed(h, K_MC_SWEEP, l, p, L.n, false,
                          [&] { lk::mc_sweep<T>(d, L.lay, L.u[cur], L.q, color, h->stream); });
                }
                continue;
            }
        }
        if constexpr (std::is_same<T, double>::value) {
            if (learned_level(h, l)) {
                learned_sweep(h, L, l, sigma_ready && s == 0);
                continue;
            }
        }
        if constexpr (std::is_same<T, float>::value) {
            if (use_fused_rb<T>(h)) {
                timed(h, K_RB_FUSED, l, p, L.n, false, [&] {
                    fused::rb_sweep3_f32(L.n, L.u[cur], L.u[cur ^ 1], L.q, h->stream);
                });
                cur ^= 1;
                continue;
            }
        }
        if (h->cfg.smoother == GMG_RBGS || h->cfg.smoother == GMG_LEARNED) {
            for (int color = first_red_done && s == 0 ? 1 : 0; color < 2; ++color) {
                if (skip_last_black && s == sweeps - 1 && color == 1) break;
                const bool ex = exact_last && s == sweeps - 1 && color == 1;
                timed(h, K_RB_HALF, l, p, L.n, false,
                      [&] { lk::rb_half<T>(d, L.lay, L.u[cur], L.q, color, h->stream, ex); });
            }
        } else {
            timed(h, K_WJ, l, p, L.n, false, [&] {
                lk::wj_sweep<T>(d, L.lay, L.u[cur], L.u[cur ^ 1], L.q, h->cfg.omega, h->stream);
            });
            cur ^= 1;
        }
    }
}

// The fused leg kernels (legs.cu) run level l of an FP32 / double-float 3D
// red-black hierarchy: ping-pong iterate arrays, a level that legs::applies
// takes, at least GMG_LEG_NMIN intervals.
template <typename T>
bool leg_possible(gmg_handle h, int n) {
    const gmg_config& c = h->cfg;
    const int nmin = h->leg_nmin > 0 ? h->leg_nmin : h->legs_mode == 1 ? 512 : 128;
    const bool type_ok = std::is_same<T, float>::value ||
                         (std::is_same<T, df32>::value && h->legs_mode == 2);
    if constexpr (std::is_same<T, float>::value || std::is_same<T, df32>::value)
        return h->legs_mode > 0 && type_ok && c.d == 3 && c.smoother == GMG_RBGS &&
               c.transfer != GMG_TRANSFER_PAPER && !use_fused_rb<T>(h) && n >= nmin &&
               (h->leg_nmax == 0 || n <= h->leg_nmax) && legs::applies<T>(c.d, n);
    return false;
}
template <typename T>
bool leg_level(gmg_handle h, const std::vector<Level<T>>& lv, int l) {
    return l + 1 < (int)lv.size() && leg_possible<T>(h, lv[l].n) && lv[l].u[1] != nullptr;
}

// First level handled by the persistent tail kernel (L = none): the first
// level with n <= 8 (3D) / 32 (2D) (GMG_TAIL_N overrides) whose tail arrays
// fit in 200 KB of shared memory, below every learned level, leaving at
// least two tail levels.
template <typename T>
int tail_level(gmg_handle h, const std::vector<Level<T>>& lv) {
    const gmg_config& c = h->cfg;
    const int L = (int)lv.size();
    if (c.smoother == GMG_MCGS || c.transfer == GMG_TRANSFER_PAPER) return L;  // grid kernels
    const int nmax = h->tail_max > 0 ? h->tail_max : c.d != 3 ? 32 : 8;
    int lo = 0;
    if (c.smoother == GMG_LEARNED)
        for (int l = 0; l < L && l < (int)h->lw.size(); ++l)
            if (h->lw[l]) lo = l + 1;
    for (int l = lo; l + 1 < L; ++l) {
        const int n = lv[l].n;
        if (n <= nmax && tail::smem_bytes(c.d, n, L - l, c.smoother, sizeof(T)) <= 200 * 1024)
            return l;
    }
    return L;
}

// The grid tail (tail::launch_grid) takes the levels from the first level
// l >= 1 with n <= gtail_nmax down to the coarsest (at least two of them):
// red-black smoothing with full weighting, a device that launches it
// cooperatively, at most 12 levels, dense arrays there, and no fused leg on
// the level above (a leg writes its coarse level in the colour-split layout).
bool grid_tail_ok(gmg_handle h) {
    const gmg_config& c = h->cfg;
    return ((h->gtail_blocks > 0 && h->gtail_bar) || h->gtail_cluster > 0) && h->gtail_nmax > 0 &&
           c.smoother == GMG_RBGS && c.transfer != GMG_TRANSFER_PAPER;
}
// The largest level n it takes.  FP64 3D restrictions from fine n >= 128
// run as z-walkers, which sum the same terms in another order than the
// one-cell kernel (whose order the grid tail follows): FP64 levels up to 64.
template <typename T>
int grid_tail_nmax(gmg_handle h) {
    return std::is_same<T, double>::value && h->cfg.d == 3 ? std::min(h->gtail_nmax, 64)
                                                           : h->gtail_nmax;
}
// At allocation, from the level sizes: the first level stored dense for it.
template <typename T>
int grid_tail_alloc(gmg_handle h, int L) {
    if (!grid_tail_ok(h)) return L;
    const int n0 = h->cfg.n;
    for (int l = 1; l + 1 < L; ++l)
        if ((n0 >> l) <= grid_tail_nmax<T>(h))
            return !leg_possible<T>(h, n0 >> (l - 1)) && L - l <= 12 ? l : L;
    return L;
}
template <typename T>
int grid_tail_level(gmg_handle h, const std::vector<Level<T>>& lv) {
    const int L = (int)lv.size();
    if (!grid_tail_ok(h)) return L;
    for (int l = 1; l + 1 < L; ++l)
        if (lv[l].n <= grid_tail_nmax<T>(h)) {
            bool ok = !leg_level<T>(h, lv, l - 1) && L - l <= 12;
            for (int k = l; k < L && ok; ++k) ok = lv[k].lay.he == 0;
            return ok ? l : L;
        }
    return L;
}

template <typename T>
cudaError_t launch_grid_tail(gmg_handle h, std::vector<Level<T>>& lv, int lg) {
    const gmg_config& c = h->cfg;
    const int L = (int)lv.size();
    int n[12];
    T* u[12];
    T* q[12];
    T* r[12];
    for (int l = lg; l < L; ++l) {
        n[l - lg] = lv[l].n;
        u[l - lg] = lv[l].u[0];
        q[l - lg] = lv[l].q;
        r[l - lg] = lv[l].r;
    }
    h->gtail_used = true;
    return tail::launch_grid<T>(c.d, L - lg, n, u, q, r, c.smoother, c.omega, c.nu1, c.nu2,
                                c.coarse_sweeps, h->gtail_cta_n, h->gtail_bar, h->gtail_blocks,
                                h->stream, h->gtail_cluster);
}

// One cycle of Algorithm 1 on the hierarchy lv (level-0 iterate lv[0].u[0]
// in and out), in stream order.  first_red_done: the cycle's first level-0
// red half sweep already ran (fp64::red_ahead); it starts with the black one.
// skip_last_black0: leave out the last level-0 black half sweep (red-black,
// post-smoothing on grid kernels), which mixed::outer_red_update forms.
template <typename T>
gmg_status enqueue_vcycle(gmg_handle h, std::vector<Level<T>>& lv, bool first_red_done = false,
                          bool skip_last_black0 = false) {
    const gmg_config& c = h->cfg;
    const int d = c.d;
    const int L = (int)lv.size();
    const int p = prec_of<T>();
    std::vector<int> cur(L, 0);
    const int lt = tail_level<T>(h, lv);
    const int lg = lt == 0 ? L : grid_tail_level<T>(h, lv);
    if (lt == 0) {
        // the whole hierarchy is small: one persistent launch
        cudaError_t e = cudaSuccess;
        timed(h, K_TAIL, 0, p, lv[0].n, false, [&] {
            e = tail::launch<T>(d, lv[0].lay, L, lv[0].u[0], lv[0].q, c.smoother, c.omega, c.nu1,
                                c.nu2, c.coarse_sweeps, h->stream, true);
        });
        GMG_CUDA_TRY(e);
    } else if (L == 1) {
        relax(h, lv, 0, c.nu1, cur[0], false, false, first_red_done);
    } else {
        // levels smoothed by grid kernels going down
        const int Ldown = lg < L ? lg : lt < L ? lt : L - 1;
        for (int l = 0; l < Ldown; ++l) {
            // fused down leg: the pre-smoothing half sweeps, the red residual
            // and the restriction in one pass (u ping-pongs)
            const int s_down = 2 * c.nu1 - (l == 0 && first_red_done ? 1 : 0);
            if (leg_level<T>(h, lv, l) && s_down >= 2 && s_down <= 4) {
                Level<T>& F = lv[l];
                Level<T>& C = lv[l + 1];
                cudaError_t e = cudaSuccess;
                timed(
                    h, K_LEG_DOWN, l, p, F.n, true,
                    [&] {
                        e = legs::down<T>(F.lay, C.lay, F.u[cur[l]], F.u[cur[l] ^ 1], F.q, C.q,
                                          C.u[0], s_down, h->stream);
                    },
                    1, s_down);
                GMG_CUDA_TRY(e);
                h->legs_used = true;
                cur[l] ^= 1;
                cur[l + 1] = 0;
                continue;
            }
            // level 0 of the plain FP64 form: the residual of the full
            // iterate, unbiased in 3D (lk::gs_value)
            const bool unbiased = l == 0 && std::is_same<T, double>::value && d == 3;
            relax(h, lv, l, c.nu1, cur[l],
                  l == 0 && std::is_same<T, double>::value && sigma_carried(h), false,
                  l == 0 && first_red_done, unbiased);
            Level<T>& F = lv[l];
            Level<T>& C = lv[l + 1];
            // After a black half sweep the black residual vanishes identically.
            const bool paper = c.transfer == GMG_TRANSFER_PAPER;
            const bool rb = c.smoother == GMG_RBGS ||
                            (c.smoother == GMG_LEARNED && !learned_level(h, l));
            const bool red_only = rb && c.nu1 > 0 && !paper;
            timed(h, K_RESIDUAL, l, p, F.n, red_only, [&] {
                lk::residual<T>(d, F.lay, F.u[cur[l]], F.q, F.r, red_only, h->stream, unbiased);
            });
            const bool exact = C.n == 2;
            bool done = false;
            if constexpr (std::is_same<T, double>::value) {
                if (paper) {
                    timed(h, K_RESTRICT_PAPER, l, p, F.n, false, [&] {
                        lk::restrict_paper<T>(d, F.lay, C.lay, F.r, C.q, C.u[0], exact,
                                              h->stream);
                    });
                    done = true;
                }
            }
            if (!done)
                timed(h, K_RESTRICT, l, p, F.n, red_only, [&] {
                    lk::restrict_fw<T>(d, F.lay, C.lay, F.r, C.q, C.u[0], red_only, exact,
                                       h->stream);
                });
            cur[l + 1] = 0;
        }
        if (lg < L) {
            cudaError_t e = cudaSuccess;
            timed(h, K_TAIL, lg, p, lv[lg].n, false,
                  [&] { e = launch_grid_tail<T>(h, lv, lg); });
            GMG_CUDA_TRY(e);
        } else if (lt < L) {
            cudaError_t e = cudaSuccess;
            timed(h, K_TAIL, lt, p, lv[lt].n, false, [&] {
                e = tail::launch<T>(d, lv[lt].lay, L - lt, lv[lt].u[0], lv[lt].q, c.smoother,
                                    c.omega, c.nu1, c.nu2, c.coarse_sweeps, h->stream);
            });
            GMG_CUDA_TRY(e);
        } else {
            Level<T>& B = lv[L - 1];
            if (B.n > 2) {
                for (int s = 0; s < c.coarse_sweeps; ++s)
                    for (int color = 0; color < 2; ++color)
                        timed(h, K_RB_HALF, L - 1, p, B.n, false,
                              [&] { lk::rb_half<T>(d, B.lay, B.u[0], B.q, color, h->stream); });
            }
        }
        for (int l = Ldown - 1; l >= 0; --l) {
            Level<T>& F = lv[l];
            Level<T>& C = lv[l + 1];
            // fused up leg: black prolongation + correction and the
            // post-smoothing half sweeps in one pass (u ping-pongs)
            const int s_up = 2 * c.nu2 - (skip_last_black0 && l == 0 ? 1 : 0);
            if (leg_level<T>(h, lv, l) && s_up >= 2 && s_up <= 4) {
                cudaError_t e = cudaSuccess;
                timed(
                    h, K_LEG_UP, l, p, F.n, true,
                    [&] {
                        e = legs::up<T>(C.lay, F.lay, C.u[cur[l + 1]], F.u[cur[l]],
                                        F.u[cur[l] ^ 1], F.q, s_up, h->stream);
                    },
                    1, s_up);
                GMG_CUDA_TRY(e);
                h->legs_used = true;
                cur[l] ^= 1;
                continue;
            }
            bool done = false;
            if constexpr (std::is_same<T, double>::value) {
                if (c.transfer == GMG_TRANSFER_PAPER) {
                    timed(h, K_PROLONG_PAPER, l, p, F.n, false, [&] {
                        lk::prolong_paper<T>(d, C.lay, F.lay, C.u[cur[l + 1]], F.u[cur[l]],
                                             h->stream);
                    });
                    done = true;
                }
            }
            if (!done) {
                const bool black = red_sweep_next<T>(h, c.nu2);
                timed(h, K_PROLONG, l, p, F.n, black, [&] {
                    lk::prolong_add<T>(d, C.lay, F.lay, C.u[cur[l + 1]], F.u[cur[l]], h->stream,
                                       black);
                });
            }
            relax(h, lv, l, c.nu2, cur[l], false, true, false, false, skip_last_black0 && l == 0);
        }
    }
    if (cur[0] != 0) {
        cudaError_t e = cudaSuccess;
        timed(h, K_COPY, 0, p, c.n, false, [&] {
            e = cudaMemcpyAsync(lv[0].u[0], lv[0].u[1], sizeof(T) * lv[0].nodes,
                                cudaMemcpyDeviceToDevice, h->stream);
        });
        GMG_CUDA_TRY(e);
    }
    return GMG_OK;
}

// Red-black inner cycles start from e = 0 with a red half sweep, which sets
// e = sigma on the red nodes and reads only black zeros: the outer residual
// writes that iterate directly (mixed::outer_residual's e_init), the first
// inner cycle starts with its black half sweep, and no memset of e is
// needed (boundary entries of e are never written and stay 0).  Same values
// bit for bit: fma(c, 0, q) + nothing else = q in every inner precision.
template <typename T>
bool inner_red_ahead(gmg_handle h) {
    const gmg_config& c = h->cfg;
    return c.smoother == GMG_RBGS && c.nu1 > 0 && !use_fused_rb<T>(h) && h->inner_ahead;
}

// Double-float red-black refinement with pre- and post-smoothing: after the
// inner cycles (a black half sweep last) the black outer residual is zero up
// to the inner rounding, so the update and the next outer residual run as
// mixed::outer_red_update (red residual only; about 40% less FP64 work than
// the update plus the full residual).  FP32 / BF16 inner cycles leave a
// black residual of their own rounding (2^-24 / 2^-8 of e, and fl32(1/6)'s
// bias), which the next step must see: they keep the full residual.
//
// The red-only scheme never corrects the black residual that the FP64
// updates' roundings leave (about eps |u| per step): harmless while |u| stays
// near the solution's size, but from a starting iterate much larger than
// the solution the iterate shrinks and those errors grow relative to it.  So
// a solve uses it only when its starting residual is at most twice the
// residual of u = 0 (step_full decides per solve).
template <typename T>
bool outer_red_possible(gmg_handle h) {
    return std::is_same<T, df32>::value && inner_red_ahead<T>(h) && h->cfg.nu2 > 0 &&
           h->outer_red;
}
template <typename T>
bool outer_red_only(gmg_handle h) {
    return outer_red_possible<T>(h) && !h->step_full;
}

// Refinement step: e = 0, k inner cycles on A'e = sigma, u += e, new sigma.
template <typename T>
gmg_status enqueue_refinement(gmg_handle h, std::vector<Level<T>>& in) {
    const gmg_config& c = h->cfg;
    const int p = prec_of<T>();
    const bool ahead = inner_red_ahead<T>(h);
    if (!ahead) {
        cudaError_t e = cudaSuccess;
        timed(h, K_MEMSET, 0, p, c.n, false, [&] {
            e = cudaMemsetAsync(in[0].u[0], 0, sizeof(T) * in[0].nodes, h->stream);
        });
        GMG_CUDA_TRY(e);
    }
    const bool red_only = outer_red_only<T>(h);
    for (int k = 0; k < c.inner_cycles; ++k) {
        gmg_status st =
            enqueue_vcycle<T>(h, in, ahead && k == 0, red_only && k == c.inner_cycles - 1);
        if (st != GMG_OK) return st;
    }
    if (red_only) {
        timed(
            h, K_OUTER_RED, 0, p, c.n, false,
            [&] {
                mixed::outer_red_update<T>(c.d, in[0].lay, h->lv[0].u[0], h->lv[0].q, in[0].q,
                                           in[0].u[0], h->partial, h->d_res2, h->stream,
                                           h->resid_b, h->resid_flag);
            },
            3);
        return GMG_OK;
    }
    timed(h, K_UPDATE, 0, p, c.n, false,
          [&] { mixed::update<T>(c.d, in[0].lay, h->lv[0].u[0], in[0].u[0], h->stream); });
    timed(
        h, K_OUTER_RES, 0, p, c.n, ahead,
        [&] {
            mixed::outer_residual<T>(c.d, in[0].lay, h->lv[0].u[0], h->lv[0].q, in[0].q, h->partial,
                                     h->d_res2, h->stream, ahead ? in[0].u[0] : nullptr);
        },
        2);
    return GMG_OK;
}

// After a plain red-black V-cycle (or FMG pass) the last operation on level 0
// is a black half sweep, so the stopping-test norm needs the red nodes only.
bool norm_red_only(gmg_handle h) {
    const gmg_config& c = h->cfg;
    return c.precision == GMG_FP64 && c.smoother == GMG_RBGS &&
           (h->lv.size() > 1 ? c.nu2 > 0 : c.nu1 > 0);
}

// The red-only stopping-test norm and the next cycle's first level-0 red half
// sweep read the same operands, and the sweep's change at a red node is that
// norm's sigma: one fused pass (fp64::red_ahead) does both, the cycle graph
// starts with its first black half sweep, and a solve that stops puts the
// red nodes back (fp64::red_restore) -- u and the norm history are those of
// the unfused schedule.  Plain FP64 red-black with grid kernels on level 0,
// pre-smoothing, and a level-0 size the diagonal walkers take.
bool norm_ahead_ok(gmg_handle h) {
    const gmg_config& c = h->cfg;
    return c.precision == GMG_FP64 && c.smoother == GMG_RBGS && c.nu1 > 0 && h->lv.size() > 1 &&
           norm_red_only(h) && fp64::red_ahead_applies(c.d, c.n) &&
           tail_level<double>(h, h->lv) > 0;
}

// The fused norm of the step's (or FMG pass's) result plus the next red half
// sweep; the squared scaled norm lands in h->d_res2.
void enqueue_norm_ahead(gmg_handle h) {
    const gmg_config& c = h->cfg;
    Level<double>& L0 = h->lv[0];
    timed(
        h, K_NORM_AHEAD, 0, 0, c.n, true,
        [&] {
            fp64::red_ahead(c.n, L0.u[0], L0.q, L0.r, h->partial, h->d_res2, true, h->stream);
        },
        2);
}

// Double-float refinement in steps of several cycles.  Each cycle of the
// FP64 V-cycle iteration is still one double-float inner V-cycle, but an
// FP64 step (the triple-float black values, u += e, the red FP64 residual and
// its norm: mixed::outer_red_update) follows only every kmax cycles: the
// inner correction e, and with it the double-float rounding, is then a small
// fraction of u (after a solve's first step, which has one cycle: its
// correction is nearly all of u).  The stopping test still runs after every
// cycle, exactly: after a black half sweep the residual vanishes on the
// black nodes, and on a red node it is the change the next red half sweep
// makes, so that sweep runs right away with the norm folded in
// (mixed::df_red_ahead); if the test stops, the sweep is undone and the step
// ends.  The norm inside a step is that of the inner equation, which is the
// outer one's up to the double-float rounding of sigma (2^-48 relative);
// the step's FP64 norm decides where it ends.  Cycle counts and histories
// are the one-cycle-per-step form's.
bool chain_on(gmg_handle h) {
    const gmg_config& c = h->cfg;
    return h->chain_k > 1 && c.precision == GMG_DF_IR && c.inner_cycles == 1 &&
           c.cycle == GMG_VCYCLE && outer_red_only<df32>(h) && h->lvd.size() > 1 &&
           h->lvd[0].lay.he != 0;
}

// hist holds st->pad entries (the loop state's history capacity).
}  // namespace
namespace gmg {
// The plan of the cycle that runs now: it continues the step (mid) unless the
// step has its cycles or the cap is one cycle away.
__global__ void k_chain_plan(const LoopState* __restrict__ st, ChainState* __restrict__ c) {
    const int k_eff = st->it == c->step_it ? 1 : c->kmax;  // a solve's first step: one cycle
    const bool mid = c->step_it + 1 < k_eff && st->it + 1 < st->cap;
    c->skip_mid = mid ? 0 : 1;
    c->skip_end = mid ? 1 : 0;
    c->restore = 0;
    c->counted = 0;
}

// Inside a step: the norm after the cycle (partials of df_red_ahead, summed
// in k_sum_partials' order), counted as a cycle; if the test stops, the step
// ends here (the red half sweep run ahead is undone first).
__global__ void __launch_bounds__(1024) k_chain_test(const double* __restrict__ partial, int count,
                                                     LoopState* __restrict__ st,
                                                     ChainState* __restrict__ c,
                                                     cudaGraphConditionalHandle cond, int has_cond) {
    __shared__ double warp_sums[32];
    if (c->skip_mid) return;
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partial[i];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double res2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) res2 += warp_sums[w];
    const int it = st->it + 1;
    st->it = it;
    const double res = sqrt(res2);
    st->res = res;
    if (it - 1 < st->pad) st->hist[it - 1] = st->res0 > 0.0 ? res / st->res0 : 0.0;
    c->step_it += 1;
    const bool more = isfinite(res) && (!st->stop || res > st->rtol * st->res0);
    if (!more) {
        c->skip_end = 0;
        c->restore = 1;
        c->counted = 1;
    } else if (has_cond) {
        cudaGraphSetConditional(cond, 1u);
    }
}

// After the step's FP64 update and residual: k_loop_test's test (the cycle
// counted unless the norm inside the step already did), then a new step.
__global__ void k_chain_end_test(const double* __restrict__ res2, LoopState* __restrict__ st,
                                 ChainState* __restrict__ c, cudaGraphConditionalHandle cond,
                                 int has_cond) {
    if (c->skip_end) return;
    int it = st->it;
    if (!c->counted) st->it = ++it;
    const double res = sqrt(res2[0]);
    st->res = res;
    if (it - 1 < st->pad) st->hist[it - 1] = st->res0 > 0.0 ? res / st->res0 : 0.0;
    c->step_it = 0;
    c->counted = 0;
    const bool more = it < st->cap && isfinite(res) && (!st->stop || res > st->rtol * st->res0);
    if (has_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
}
}  // namespace gmg
namespace {

// One cycle of the chained form: the inner V-cycle (its first red half sweep
// already done, its last level-0 black one left to the step's end), then the
// device-side plan's mid part (timer group 1) or end part (group 2; the
// restore, group 3, only after a stop inside the step).  in_loop: inside the
// while node (the test kernels set its condition).
gmg_status enqueue_chain_kernels(gmg_handle h, bool in_loop) {
    const gmg_config& c = h->cfg;
    Level<df32>& I0 = h->lvd[0];
    ChainState* C = h->d_chain;
    const int p = prec_of<df32>();
    k_chain_plan<<<1, 1, 0, h->stream>>>(h->d_loop, C);
    h->timer.graph_kernels += 1;
    gmg_status st = enqueue_vcycle<df32>(h, h->lvd, true, true);
    if (st != GMG_OK) return st;
    h->timer.cur_group = 1;
    timed(h, K_RB_HALF, 0, p, c.n, false, [&] {
        mixed::df_black_half(c.d, I0.lay, I0.u[0], I0.q, &C->skip_mid, h->stream);
    });
    int np = 0;
    timed(h, K_NORM_AHEAD, 0, p, c.n, true, [&] {
        np = mixed::df_red_ahead(c.d, I0.lay, I0.u[0], I0.q, I0.r, h->partial, &C->skip_mid,
                                 h->stream);
    });
    k_chain_test<<<1, 1024, 0, h->stream>>>(h->partial, np, h->d_loop, C, h->loop_cond,
                                            in_loop ? 1 : 0);
    h->timer.graph_kernels += 1;
    h->timer.cur_group = 3;
    timed(h, K_RESTORE, 0, p, c.n, true, [&] {
        mixed::df_red_restore(c.d, I0.lay, I0.u[0], I0.r, &C->restore, h->stream);
    });
    h->timer.cur_group = 2;
    timed(
        h, K_OUTER_RED, 0, p, c.n, false,
        [&] {
            mixed::outer_red_update<df32>(c.d, I0.lay, h->lv[0].u[0], h->lv[0].q, I0.q, I0.u[0],
                                          h->partial, h->d_res2, h->stream, h->resid_b,
                                          h->resid_flag, &C->skip_end);
        },
        3);
    k_chain_end_test<<<1, 1, 0, h->stream>>>(h->d_res2, h->d_loop, C, h->loop_cond,
                                             in_loop ? 1 : 0);
    h->timer.graph_kernels += 1;
    h->timer.cur_group = 0;
    GMG_CUDA_TRY(cudaGetLastError());
    return GMG_OK;
}

// One step of the stopping loop: a plain cycle plus the FP64 norm, or one
// refinement step; the squared scaled norm lands in h->d_res2 (enqueue_step:
// and is copied to h->h_res2).
gmg_status enqueue_step_kernels(gmg_handle h, bool in_loop = false) {
    const gmg_config& c = h->cfg;
    h->timer.begin_capture();
    gmg_status st = GMG_OK;
    if (chain_on(h)) {
        st = enqueue_chain_kernels(h, in_loop);
    } else if (c.precision == GMG_FP64 && h->ahead) {
        st = enqueue_vcycle<double>(h, h->lv, true);
        if (st != GMG_OK) return st;
        enqueue_norm_ahead(h);
    } else if (c.precision == GMG_FP64) {
        st = enqueue_vcycle<double>(h, h->lv);
        if (st != GMG_OK) return st;
        double* keep = sigma_carried(h) ? h->lv[0].r : nullptr;
        timed(
            h, K_RESNORM, 0, 0, c.n, norm_red_only(h),
            [&] {
                fp64::resnorm(c.d, c.n, h->lv[0].u[0], h->lv[0].q, h->partial, h->d_res2,
                              h->stream, keep, norm_red_only(h));
            },
            2);
    } else if (c.precision == GMG_FP32_IR) {
        st = enqueue_refinement<float>(h, h->lvf);
    } else if (c.precision == GMG_DF_IR) {
        st = enqueue_refinement<df32>(h, h->lvd);
    } else {
        st = enqueue_refinement<bf16>(h, h->lvb);
    }
    if (st != GMG_OK) return st;
    GMG_CUDA_TRY(cudaGetLastError());
    return GMG_OK;
}

gmg_status enqueue_step(gmg_handle h) {
    gmg_status st = enqueue_step_kernels(h);
    if (st != GMG_OK) return st;
    if (chain_on(h)) {  // the loop state the step's test kernels keep, and their plan
        GMG_CUDA_TRY(cudaMemcpyAsync(h->h_loop, h->d_loop, kLoopHeader, cudaMemcpyDeviceToHost,
                                     h->stream));
        GMG_CUDA_TRY(cudaMemcpyAsync(h->h_chain, h->d_chain, sizeof(ChainState),
                                     cudaMemcpyDeviceToHost, h->stream));
        GMG_CUDA_TRY(cudaGetLastError());
        return GMG_OK;
    }
    GMG_CUDA_TRY(cudaMemcpyAsync(h->h_res2, h->d_res2, sizeof(double), cudaMemcpyDeviceToHost,
                                 h->stream));
    GMG_CUDA_TRY(cudaGetLastError());
    return GMG_OK;
}

// The stopping test of Algorithm 3 after a cycle, on the device: it counts
// the cycle, records res / res0, and lets the while node run another cycle
// while it < cap, res is finite and (unless stop is off) res > rtol * res0
// (the host loop's test, in the same FP64 operations).
}  // namespace
namespace gmg {
__global__ void k_loop_test(const double* __restrict__ res2, LoopState* __restrict__ st,
                            cudaGraphConditionalHandle cond) {
    const int it = st->it + 1;
    st->it = it;
    const double res = sqrt(res2[0]);
    st->res = res;
    st->hist[it - 1] = st->res0 > 0.0 ? res / st->res0 : 0.0;
    const bool more = it < st->cap && isfinite(res) && (!st->stop || res > st->rtol * st->res0);
    cudaGraphSetConditional(cond, more ? 1u : 0u);
}
}  // namespace gmg
namespace {

// The loop graph: a while node whose body is one step (a cycle and its FP64
// norm) followed by k_loop_test.  On failure the handle keeps the host loop.
void build_loop_graph(gmg_handle h) {
    cudaGraph_t g = nullptr;
    cudaGraph_t body = nullptr;
    bool capturing = false;
    auto give_up = [&] {
        if (capturing) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(h->stream, &tmp);
        }
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        h->loop_graph = nullptr;
    };
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return give_up();
    if (cudaGraphConditionalHandleCreate(&h->loop_cond, g, 1, cudaGraphCondAssignDefault) !=
        cudaSuccess)
        return give_up();
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h->loop_cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) return give_up();
    body = np.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return give_up();
    capturing = true;
    const int step_kernels = h->timer.graph_kernels;
    h->timer.begin_capture();
    if (enqueue_step_kernels(h, true) != GMG_OK) return give_up();
    if (chain_on(h)) {  // the chain's test kernels set the condition
        h->loop_kernels = h->timer.graph_kernels;
    } else {
        k_loop_test<<<1, 1, 0, h->stream>>>(h->d_res2, h->d_loop, h->loop_cond);
        h->loop_kernels = h->timer.graph_kernels + 1;
    }
    h->timer.graph_kernels = step_kernels;
    capturing = false;
    if (cudaStreamEndCapture(h->stream, &body) != cudaSuccess) return give_up();
    if (cudaGraphInstantiate(&h->loop_graph, g, 0) != cudaSuccess) return give_up();
    cudaGraphDestroy(g);
}

// One full-multigrid pass (Algorithm 2) on the plain FP64 hierarchy, then the
// FP64 norm: q restricted to every level (4 FW, the residual's scaling), the
// coarsest solved, then per level u_l = P u_{l+1} and one V-cycle on levels
// l .. L-1.
gmg_status enqueue_fmg(gmg_handle h) {
    const gmg_config& c = h->cfg;
    std::vector<Level<double>>& lv = h->lv;
    const int d = c.d, L = (int)lv.size();
    h->timer.begin_capture();
    for (int l = 0; l + 1 < L; ++l) {
        Level<double>& F = lv[l];
        Level<double>& C = lv[l + 1];
        if (c.transfer == GMG_TRANSFER_PAPER)
            timed(h, K_RESTRICT_PAPER, l, 0, F.n, false, [&] {
                lk::restrict_paper<double>(d, F.lay, C.lay, F.q, C.q, C.u[0], C.n == 2,
                                           h->stream);
            });
        else
            timed(h, K_RESTRICT, l, 0, F.n, false, [&] {
                lk::restrict_fw<double>(d, F.n, F.q, C.q, C.u[0], false, C.n == 2, h->stream);
            });
    }
    if (L > 1 && lv[L - 1].n > 2) {
        Level<double>& B = lv[L - 1];
        for (int s = 0; s < c.coarse_sweeps; ++s)
            for (int color = 0; color < 2; ++color)
                timed(h, K_RB_HALF, L - 1, 0, B.n, false,
                      [&] { lk::rb_half<double>(d, B.n, B.u[0], B.q, color, h->stream); });
    }
    cudaError_t e = cudaMemsetAsync(lv[0].u[0], 0, sizeof(double) * lv[0].nodes, h->stream);
    GMG_CUDA_TRY(e);
    for (int l = L - 2; l >= 0; --l) {
        if (c.transfer == GMG_TRANSFER_PAPER) {
            timed(h, K_PROLONG_PAPER, l, 0, lv[l].n, false, [&] {
                lk::prolong_paper<double>(d, lv[l + 1].lay, lv[l].lay, lv[l + 1].u[0],
                                          lv[l].u[0], h->stream);
            });
        } else {
            const bool black = red_sweep_next<double>(h, c.nu1);
            timed(h, K_PROLONG, l, 0, lv[l].n, black, [&] {
                lk::prolong_add<double>(d, lv[l + 1].n, lv[l + 1].u[0], lv[l].u[0], h->stream,
                                        black);
            });
        }
        std::vector<Level<double>> sub(lv.begin() + l, lv.end());
        gmg_status st = enqueue_vcycle<double>(h, sub);
        if (st != GMG_OK) return st;
    }
    if (L == 1) {
        gmg_status st = enqueue_vcycle<double>(h, lv);
        if (st != GMG_OK) return st;
    }
    if (h->ahead)
        enqueue_norm_ahead(h);
    else
        timed(
            h, K_RESNORM, 0, 0, c.n, norm_red_only(h),
            [&] {
                fp64::resnorm(c.d, c.n, lv[0].u[0], lv[0].q, h->partial, h->d_res2, h->stream,
                              nullptr, norm_red_only(h));
            },
            2);
    GMG_CUDA_TRY(cudaMemcpyAsync(h->h_res2, h->d_res2, sizeof(double), cudaMemcpyDeviceToHost,
                                 h->stream));
    GMG_CUDA_TRY(cudaGetLastError());
    return GMG_OK;
}

gmg_status capture(gmg_handle h, cudaGraphExec_t* out, gmg_status (*enqueue)(gmg_handle)) {
    cudaGraph_t g = nullptr;
    GMG_CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    gmg_status st = enqueue(h);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (st != GMG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) {
        set_error(std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
        return GMG_ERR_CUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        return GMG_ERR_CUDA;
    }
    return GMG_OK;
}

gmg_status ensure_graph(gmg_handle h, double* u) {
    if (h->graph && h->graph_u == u && h->graph_step_full == h->step_full &&
        h->graph_chain == chain_on(h))
        return GMG_OK;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (h->fmg_graph) {
        cudaGraphExecDestroy(h->fmg_graph);
        h->fmg_graph = nullptr;
    }
    if (h->loop_graph) {
        cudaGraphExecDestroy(h->loop_graph);
        h->loop_graph = nullptr;
    }
    h->lv[0].u[0] = u;
    gmg_status st;
    if (h->cfg.cycle == GMG_FMG) {
        if ((st = capture(h, &h->fmg_graph, enqueue_fmg)) != GMG_OK) return st;
        h->fmg_kernels = h->timer.graph_kernels;
        h->fmg_pending = h->timer.pending;
    }
    if ((st = capture(h, &h->graph, enqueue_step)) != GMG_OK) return st;
    if (h->device_loop && h->d_loop && !h->timer.enabled) build_loop_graph(h);
    h->graph_u = u;
    h->graph_step_full = h->step_full;
    h->graph_chain = chain_on(h);
    return GMG_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev)
            cudaSetDevice(dev);
        else
            prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// q_0 = h^2 f/(2d), u's boundary = 0, then the initial squared scaled
// residual norm (and, for refinement, the first inner right-hand side).
gmg_status enqueue_start(gmg_handle h, const double* f, double* u) {
    const gmg_config& c = h->cfg;
    int* unz = c.precision != GMG_FP64 ? h->d_unz : nullptr;
    if (unz) GMG_CUDA_TRY(cudaMemsetAsync(unz, 0, sizeof(int), h->stream));
    fp64::prepare(c.d, c.n, f, h->lv[0].q, u, h->stream, unz);
    if (c.precision == GMG_FP64 && h->ahead && c.cycle != GMG_FMG) {
        // the first norm in two colour halves: the black one from u_0, then
        // the red one fused with the first cycle's first red half sweep
        // (undone if the solve stops before the first cycle)
        fp64::resnorm_black(c.n, u, h->lv[0].q, h->partial, h->d_res2 + 1, h->stream);
        fp64::red_ahead(c.n, u, h->lv[0].q, h->lv[0].r, h->partial, h->d_res2, true, h->stream,
                        h->d_res2 + 1);
        h->timer.launches += 2;
    } else if (c.precision == GMG_FP64) {
        fp64::resnorm(c.d, c.n, u, h->lv[0].q, h->partial, h->d_res2, h->stream,
                      sigma_carried(h) ? h->lv[0].r : nullptr);
    } else if (c.precision == GMG_FP32_IR)
        mixed::outer_residual<float>(c.d, h->lvf[0].lay, u, h->lv[0].q, h->lvf[0].q, h->partial,
                                     h->d_res2, h->stream,
                                     inner_red_ahead<float>(h) ? h->lvf[0].u[0] : nullptr,
                                     nullptr, nullptr, nullptr, unz);
    else if (c.precision == GMG_DF_IR)
        mixed::outer_residual<df32>(c.d, h->lvd[0].lay, u, h->lv[0].q, h->lvd[0].q, h->partial,
                                    h->d_res2, h->stream,
                                    inner_red_ahead<df32>(h) ? h->lvd[0].u[0] : nullptr,
                                    outer_red_possible<df32>(h) ? h->resid_b : nullptr,
                                    outer_red_possible<df32>(h) ? h->resid_flag : nullptr,
                                    outer_red_possible<df32>(h) ? h->d_res2 + 2 : nullptr, unz);
    else
        mixed::outer_residual<bf16>(c.d, h->lvb[0].lay, u, h->lv[0].q, h->lvb[0].q, h->partial,
                                    h->d_res2, h->stream,
                                    inner_red_ahead<bf16>(h) ? h->lvb[0].u[0] : nullptr,
                                    nullptr, nullptr, nullptr, unz);
    h->timer.launches += 3;
    GMG_CUDA_TRY(cudaGetLastError());
    return GMG_OK;
}

gmg_status start(gmg_handle h, const double* f, double* u, double* res0) {
    GMG_CUDA_TRY(cudaEventRecord(h->ev, h->user_stream));
    GMG_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev, 0));
    gmg_status st = enqueue_start(h, f, u);
    if (st != GMG_OK) return st;
    const bool choose = outer_red_possible<df32>(h);
    GMG_CUDA_TRY(cudaMemcpyAsync(h->h_res2, h->d_res2, sizeof(double) * (choose ? 3 : 1),
                                 cudaMemcpyDeviceToHost, h->stream));
    GMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    *res0 = std::sqrt(*h->h_res2);
    if (!std::isfinite(*res0)) {
        set_error("initial residual norm is not finite (NaN/Inf in f or u)");
        return GMG_ERR_NONFINITE;
    }
    if (choose) h->step_full = !(h->h_res2[0] <= 4.0 * h->h_res2[2]);
    return ensure_graph(h, u);
}

// Run steps: until the stopping test (stop = true) or exactly ncycles.
gmg_status run(gmg_handle h, const double* f, double* u, double rtol, int ncycles, bool stop,
               int* iters_out, double* relres_out) {
    gmg_status st = check_device_ptr(f, "f");
    if (st != GMG_OK) return st;
    st = check_device_ptr(u, "u");
    if (st != GMG_OK) return st;
    DeviceGuard guard(h->device);
    h->hist.clear();
    double res0 = 0.0;
    st = start(h, f, u, &res0);
    if (st != GMG_OK) return st;
    double res = res0;
    int it = 0;
    const int cap = stop ? h->cfg.maxit : ncycles;
    // with the fused norm a red half sweep of a cycle that does not run is
    // pending on u whenever the loop ends: undo it
    auto finish = [&]() -> gmg_status {
        if (h->ahead && (it > 0 || !h->fmg_graph)) {
            fp64::red_restore(h->cfg.n, u, h->lv[0].r, h->stream);
            h->timer.launches += 1;
            GMG_CUDA_TRY(cudaGetLastError());
            GMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
        }
        return GMG_OK;
    };
    // chained double-float steps: the plan and the test run on the device in
    // either loop, on the loop state set here
    const bool chain = chain_on(h);
    if (chain) {
        LoopState* L = h->h_loop;
        L->res0 = res0;
        L->rtol = rtol;
        L->res = res;
        L->cap = cap;
        L->stop = stop ? 1 : 0;
        L->it = 0;
        L->pad = h->loop_cap;
        ChainState* C = h->h_chain;
        *C = ChainState{0, h->chain_k, 0, 0, 0, 0};
        GMG_CUDA_TRY(
            cudaMemcpyAsync(h->d_loop, L, kLoopHeader, cudaMemcpyHostToDevice, h->stream));
        GMG_CUDA_TRY(cudaMemcpyAsync(h->d_chain, C, sizeof(ChainState), cudaMemcpyHostToDevice,
                                     h->stream));
    }
    while (it < cap && (!stop || res > rtol * res0)) {
        const bool fmg = it == 0 && h->fmg_graph;
        if (!fmg && h->loop_graph && !h->timer.enabled && cap <= h->loop_cap) {
            // the remaining cycles in one launch, the test on the device
            LoopState* L = h->h_loop;
            L->res0 = res0;
            L->rtol = rtol;
            L->res = res;
            L->cap = cap;
            L->stop = stop ? 1 : 0;
            L->it = it;
            L->pad = h->loop_cap;
            GMG_CUDA_TRY(
                cudaMemcpyAsync(h->d_loop, L, kLoopHeader, cudaMemcpyHostToDevice, h->stream));
            GMG_CUDA_TRY(cudaGraphLaunch(h->loop_graph, h->stream));
            GMG_CUDA_TRY(cudaMemcpyAsync(L, h->d_loop, kLoopHeader + sizeof(double) * cap,
                                         cudaMemcpyDeviceToHost, h->stream));
            GMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
            const int it0 = it;
            it = L->it;
            h->timer.launches += (int64_t)(it - it0) * h->loop_kernels;
            for (int k = it0; k < it; ++k) {
                h->hist.push_back(L->hist[k]);
                if (!stop && relres_out) relres_out[k] = L->hist[k];
            }
            res = L->res;
            if (!std::isfinite(res)) {
                if (iters_out) *iters_out = it;
                if ((st = finish()) != GMG_OK) return st;
                set_error("residual norm became non-finite");
                return GMG_ERR_NONFINITE;
            }
            break;
        }
        GMG_CUDA_TRY(cudaGraphLaunch(fmg ? h->fmg_graph : h->graph, h->stream));
        GMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
        if (chain) {
            // one cycle; the timer leaves out the groups the plan skipped
            const ChainState* C = h->h_chain;
            h->timer.after_graph_run((C->skip_mid ? 2u : 0u) | (C->skip_end ? 4u : 0u) |
                                     (C->restore ? 0u : 8u));
            it = h->h_loop->it;
            res = h->h_loop->res;
            const double rel = res0 > 0.0 ? res / res0 : 0.0;
            h->hist.push_back(rel);
            if (!stop && relres_out) relres_out[it - 1] = rel;
            if (!std::isfinite(res)) {
                if (iters_out) *iters_out = it;
                set_error("residual norm became non-finite");
                return GMG_ERR_NONFINITE;
            }
            continue;
        }
        if (fmg) {
            // the FMG graph's own launch count and (when timing) event pairs
            std::swap(h->timer.pending, h->fmg_pending);
            std::swap(h->timer.graph_kernels, h->fmg_kernels);
            h->timer.after_graph_run();
            std::swap(h->timer.pending, h->fmg_pending);
            std::swap(h->timer.graph_kernels, h->fmg_kernels);
        } else {
            h->timer.after_graph_run();
        }
        res = std::sqrt(*h->h_res2);
        ++it;
        const double rel = res0 > 0.0 ? res / res0 : 0.0;
        h->hist.push_back(rel);
        if (!stop && relres_out) relres_out[it - 1] = rel;
        if (!std::isfinite(res)) {
            if (iters_out) *iters_out = it;
            if ((st = finish()) != GMG_OK) return st;
            set_error("residual norm became non-finite");
            return GMG_ERR_NONFINITE;
        }
    }
    if ((st = finish()) != GMG_OK) return st;
    if (h->gtail_used && h->gtail_bar && h->gtail_cluster == 0 &&
        tail::grid_fault(h->gtail_bar) != 0) {
        set_error("the grid tail gave up waiting at a grid barrier; results are invalid");
        return GMG_ERR_CUDA;
    }
    if (h->legs_used && legs::fault() != 0) {
        set_error("a fused leg kernel gave up waiting for its plane loads; results are invalid");
        return GMG_ERR_CUDA;
    }
    if (iters_out) *iters_out = it;
    if (stop && relres_out) *relres_out = res0 > 0.0 ? res / res0 : 0.0;
    if (stop && res > rtol * res0) {
        set_error("maxit reached before the relative residual fell below rtol");
        return GMG_ERR_NOT_CONVERGED;
    }
    return GMG_OK;
}

template <typename T>
gmg_status alloc_hierarchy(gmg_handle h, std::vector<Level<T>>& lv, int levels, bool alloc_u0) {
    const gmg_config& c = h->cfg;
    gmg_status st;
    lv.resize(levels);
    for (int l = 0; l < levels; ++l) {
        Level<T>& v = lv[l];
        v.n = c.n >> l;
        // FP64 levels keep the caller's dense layout; the FP32/BF16 inner
        // hierarchies are colour-split (dense for the fused FP32 sweep and on
        // the levels of the grid tail)
        const bool dense = std::is_same<T, double>::value || use_fused_rb<T>(h) ||
                           l >= grid_tail_alloc<T>(h, levels);
        v.lay = dense ? dense_lay(c.d, v.n) : split_lay(c.d, v.n);
        v.nodes = lay_elems(c.d, v.lay);
        if (l > 0 || alloc_u0)
            if ((st = dev_alloc(h, &v.u[0], v.nodes)) != GMG_OK) return st;
        const bool pingpong =
            c.smoother == GMG_WJACOBI || use_fused_rb<T>(h) || (l + 1 < levels && leg_possible<T>(h, v.n));
        if (pingpong && (st = dev_alloc(h, &v.u[1], v.nodes)) != GMG_OK) return st;
        if ((st = dev_alloc(h, &v.q, v.nodes)) != GMG_OK) return st;
        const bool need_r = l + 1 < levels || c.smoother == GMG_LEARNED;
        if (need_r && (st = dev_alloc(h, &v.r, v.nodes)) != GMG_OK) return st;
    }
    return GMG_OK;
}

}  // namespace

extern "C" {

int gmg_abi_version(void) { return GMG_ABI_VERSION; }

const char* gmg_last_error(void) { return gmg::last_error().c_str(); }

gmg_status gmg_config_init(gmg_config* cfg, int d, int n) {
    if (!cfg) {
        set_error("config is NULL");
        return GMG_ERR_ARG;
    }
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->d = d;
    cfg->n = n;
    cfg->levels = 0;
    cfg->smoother = GMG_RBGS;
    cfg->omega = 0.8;
    cfg->nu1 = 2;
    cfg->nu2 = 2;
    cfg->cycle = GMG_VCYCLE;
    cfg->precision = GMG_FP64;
    cfg->maxit = 100;
    cfg->inner_cycles = 4;
    cfg->coarse_sweeps = 64;
    cfg->transfer = GMG_TRANSFER_FW;
    return GMG_OK;
}

gmg_status gmg_destroy(gmg_handle h) {
    if (!h) return GMG_OK;
    DeviceGuard guard(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->fmg_graph) cudaGraphExecDestroy(h->fmg_graph);
    if (h->loop_graph) cudaGraphExecDestroy(h->loop_graph);
    if (h->h_loop) cudaFreeHost(h->h_loop);
    if (h->h_chain) cudaFreeHost(h->h_chain);
    h->timer.destroy();
    for (void* p : h->allocs) cudaFree(p);
    if (h->h_res2) cudaFreeHost(h->h_res2);
    if (h->ev) cudaEventDestroy(h->ev);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return GMG_OK;
}

gmg_status gmg_create(const gmg_config* cfg, void* cuda_stream, gmg_handle* out) {
    if (!out) {
        set_error("out is NULL");
        return GMG_ERR_ARG;
    }
    *out = nullptr;
    gmg_status st = check_cfg(cfg);
    if (st != GMG_OK) return st;
    gmg_handle h = new gmg_handle_s();
    h->cfg = *cfg;
    h->user_stream = (cudaStream_t)cuda_stream;
    if (const char* v = std::getenv("GMG_FUSED_RB")) h->fused_rb = std::strcmp(v, "1") == 0;
    if (const char* v = std::getenv("GMG_INNER_AHEAD")) h->inner_ahead = std::strcmp(v, "0") != 0;
    if (const char* v = std::getenv("GMG_OUTER_RED")) h->outer_red = std::strcmp(v, "0") != 0;
    if (const char* v = std::getenv("GMG_TAIL_N")) h->tail_max = std::max(0, std::atoi(v));
    if (const char* v = std::getenv("GMG_DEVICE_LOOP")) h->device_loop = std::strcmp(v, "0") != 0;
    if (const char* v = std::getenv("GMG_FUSED_LEGS")) h->legs_mode = std::strcmp(v, "0") ? 2 : 0;
    if (const char* v = std::getenv("GMG_LEG_NMIN")) h->leg_nmin = std::max(2, std::atoi(v));
    if (const char* v = std::getenv("GMG_LEG_NMAX")) h->leg_nmax = std::max(0, std::atoi(v));
    if (const char* v = std::getenv("GMG_GRID_TAIL_N")) h->gtail_nmax = std::max(0, std::atoi(v));
    if (const char* v = std::getenv("GMG_GRID_TAIL_CTA_N"))
        h->gtail_cta_n = std::max(2, std::atoi(v));
    if (const char* v = std::getenv("GMG_GRID_TAIL_CLUSTER"))
        h->gtail_cluster = std::max(0, std::min(16, std::atoi(v)));
    if (const char* v = std::getenv("GMG_DF_STEP_CYCLES"))
        h->chain_k = std::max(1, std::min(64, std::atoi(v)));
    auto fail = [&](gmg_status s) {
        gmg_destroy(h);
        return s;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        set_error("no CUDA device");
        delete h;
        return GMG_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming) != cudaSuccess) {
        set_error("stream/event creation failed");
        return fail(GMG_ERR_CUDA);
    }
    const int d = cfg->d;
    const int L = num_levels(*cfg);
    if (h->gtail_nmax > 0 && cfg->smoother == GMG_RBGS) {
        h->gtail_blocks = cfg->precision == GMG_FP64      ? tail::grid_blocks<double>(d)
                          : cfg->precision == GMG_FP32_IR ? tail::grid_blocks<float>(d)
                          : cfg->precision == GMG_DF_IR   ? tail::grid_blocks<df32>(d)
                                                          : tail::grid_blocks<bf16>(d);
        if (h->gtail_blocks > 0 &&
            (st = dev_alloc(h, (char**)&h->gtail_bar, (int64_t)tail::grid_bar_bytes())) != GMG_OK)
            return fail(st);
    }
    if (cfg->precision == GMG_FP64) {
        if ((st = alloc_hierarchy<double>(h, h->lv, L, false)) != GMG_OK) return fail(st);
    } else {
        // FP64 level 0: the caller's u and the FP64 scaled right-hand side
        h->lv.resize(1);
        h->lv[0].n = cfg->n;
        h->lv[0].lay = dense_lay(d, cfg->n);
        h->lv[0].nodes = nodes_of(d, cfg->n);
        if ((st = dev_alloc(h, &h->lv[0].q, h->lv[0].nodes)) != GMG_OK) return fail(st);
        st = cfg->precision == GMG_FP32_IR ? alloc_hierarchy<float>(h, h->lvf, L, true)
             : cfg->precision == GMG_DF_IR ? alloc_hierarchy<df32>(h, h->lvd, L, true)
                                           : alloc_hierarchy<bf16>(h, h->lvb, L, true);
        if (st != GMG_OK) return fail(st);
        if ((st = dev_alloc(h, &h->d_unz, 1)) != GMG_OK) return fail(st);
        if (cfg->precision == GMG_DF_IR &&
            ((st = dev_alloc(h, &h->resid_b, h->lvd[0].nodes)) != GMG_OK ||
             (st = dev_alloc(h, &h->resid_flag, 1)) != GMG_OK))
            return fail(st);
    }
    if (cfg->smoother == GMG_LEARNED) {
        h->lw.assign(L, nullptr);
        h->lz.assign(L, nullptr);
        if ((st = dev_alloc(h, &h->lw_scratch, 2 * 8 * 27)) != GMG_OK) return fail(st);
    }
    // partials: the residual's, and (refinement start) those of q^2 after them
    const int np = std::max(fp64::resnorm_partials(d, cfg->n), 2 * mixed::outer_partials(d, cfg->n));
    if ((st = dev_alloc(h, &h->partial, np)) != GMG_OK) return fail(st);
    if ((st = dev_alloc(h, &h->d_res2, 3)) != GMG_OK) return fail(st);
    if (cudaMallocHost((void**)&h->h_res2, 3 * sizeof(double)) != cudaSuccess) {
        set_error("cudaMallocHost failed");
        return fail(GMG_ERR_ALLOC);
    }
    h->loop_cap = std::max(cfg->maxit, 1);
    const size_t loop_bytes = kLoopHeader + sizeof(double) * h->loop_cap;
    if ((st = dev_alloc(h, (char**)&h->d_loop, (int64_t)loop_bytes)) != GMG_OK) return fail(st);
    if (cudaMallocHost((void**)&h->h_loop, loop_bytes) != cudaSuccess) {
        set_error("cudaMallocHost failed");
        return fail(GMG_ERR_ALLOC);
    }
    if ((st = dev_alloc(h, (char**)&h->d_chain, (int64_t)sizeof(ChainState))) != GMG_OK)
        return fail(st);
    if (cudaMallocHost((void**)&h->h_chain, sizeof(ChainState)) != cudaSuccess) {
        set_error("cudaMallocHost failed");
        return fail(GMG_ERR_ALLOC);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        set_error("initialisation failed");
        return fail(GMG_ERR_CUDA);
    }
    h->ahead = norm_ahead_ok(h);
    *out = h;
    return GMG_OK;
}

gmg_status gmg_solve(gmg_handle h, const double* f, double* u, double rtol, int* iters_out,
                     double* relres_out) {
    if (!h) {
        set_error("handle is NULL");
        return GMG_ERR_ARG;
    }
    if (!(rtol >= 0.0) || !std::isfinite(rtol)) {
        set_error("rtol must be finite and >= 0");
        return GMG_ERR_ARG;
    }
    return run(h, f, u, rtol, 0, true, iters_out, relres_out);
}

gmg_status gmg_solve_strided(gmg_handle h, const double* f, double* u, const int64_t strides[3],
                             double rtol, int* iters_out, double* relres_out) {
    if (!h || !strides) {
        set_error("handle / strides is NULL");
        return GMG_ERR_ARG;
    }
    const int d = h->cfg.d;
    const int64_t m = h->cfg.n + 1;
    const int64_t sy = strides[1], sz = d == 3 ? strides[2] : 0;
    if (strides[0] != 1 || sy < m || (d == 3 && sz < sy * m)) {
        set_error("strides must be {1, >= n+1, >= strides[1]*(n+1) (3D)} elements");
        return GMG_ERR_LAYOUT;
    }
    if (sy == m && (d == 2 || sz == m * m)) return gmg_solve(h, f, u, rtol, iters_out, relres_out);
    if (!(rtol >= 0.0) || !std::isfinite(rtol)) {
        set_error("rtol must be finite and >= 0");
        return GMG_ERR_ARG;
    }
    gmg_status st = check_device_ptr(f, "f");
    if (st != GMG_OK) return st;
    if ((st = check_device_ptr(u, "u")) != GMG_OK) return st;
    DeviceGuard guard(h->device);
    const int64_t nodes = h->lv[0].nodes;
    if (!h->f_stage) {
        if ((st = dev_alloc(h, &h->f_stage, nodes)) != GMG_OK) return st;
        if ((st = dev_alloc(h, &h->u_stage, nodes)) != GMG_OK) return st;
    }
    GMG_CUDA_TRY(cudaEventRecord(h->ev, h->user_stream));
    GMG_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev, 0));
    const int64_t dz = d == 3 ? m * m : 0;
    fp64::copy_strided(d, h->cfg.n, f, sy, sz, h->f_stage, m, dz, h->stream);
    fp64::copy_strided(d, h->cfg.n, u, sy, sz, h->u_stage, m, dz, h->stream);
    GMG_CUDA_TRY(cudaGetLastError());
    st = run(h, h->f_stage, h->u_stage, rtol, 0, true, iters_out, relres_out);
    if (st != GMG_OK && st != GMG_ERR_NOT_CONVERGED) return st;
    fp64::copy_strided(d, h->cfg.n, h->u_stage, m, dz, u, sy, sz, h->stream);
    GMG_CUDA_TRY(cudaGetLastError());
    GMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return st;
}

gmg_status gmg_cycles(gmg_handle h, const double* f, double* u, int ncycles, double* relres_out) {
    if (!h) {
        set_error("handle is NULL");
        return GMG_ERR_ARG;
    }
    if (ncycles < 0) {
        set_error("ncycles must be >= 0");
        return GMG_ERR_ARG;
    }
    return run(h, f, u, 0.0, ncycles, false, nullptr, relres_out);
}

gmg_status gmg_solve_host(gmg_handle h, const double* f_host, double* u_host, double rtol,
                          int* iters_out, double* relres_out) {
    if (!h) {
        set_error("handle is NULL");
        return GMG_ERR_ARG;
    }
    if (!f_host || !u_host) {
        set_error("f_host / u_host is NULL");
        return GMG_ERR_LAYOUT;
    }
    DeviceGuard guard(h->device);
    const int64_t m = h->lv[0].nodes;
    gmg_status st;
    if (!h->f_stage) {
        if ((st = dev_alloc(h, &h->f_stage, m)) != GMG_OK) return st;
        if ((st = dev_alloc(h, &h->u_stage, m)) != GMG_OK) return st;
    }
    GMG_CUDA_TRY(cudaEventRecord(h->ev, h->user_stream));
    GMG_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev, 0));
    GMG_CUDA_TRY(cudaMemcpyAsync(h->f_stage, f_host, sizeof(double) * m, cudaMemcpyHostToDevice,
                                 h->stream));
    GMG_CUDA_TRY(cudaMemcpyAsync(h->u_stage, u_host, sizeof(double) * m, cudaMemcpyHostToDevice,
                                 h->stream));
    st = run(h, h->f_stage, h->u_stage, rtol, 0, true, iters_out, relres_out);
    if (st != GMG_OK && st != GMG_ERR_NOT_CONVERGED) return st;
    GMG_CUDA_TRY(cudaMemcpyAsync(u_host, h->u_stage, sizeof(double) * m, cudaMemcpyDeviceToHost,
                                 h->stream));
    GMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return st;
}

gmg_status gmg_residual_norm(gmg_handle h, const double* f, double* u, double* norm_out) {
    if (!h || !norm_out) {
        set_error("handle / norm_out is NULL");
        return GMG_ERR_ARG;
    }
    gmg_status st = check_device_ptr(f, "f");
    if (st != GMG_OK) return st;
    if ((st = check_device_ptr(u, "u")) != GMG_OK) return st;
    DeviceGuard guard(h->device);
    GMG_CUDA_TRY(cudaEventRecord(h->ev, h->user_stream));
    GMG_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev, 0));
    const gmg_config& c = h->cfg;
    fp64::prepare(c.d, c.n, f, h->lv[0].q, u, h->stream);
    fp64::resnorm(c.d, c.n, u, h->lv[0].q, h->partial, h->d_res2, h->stream);
    h->timer.launches += 3;
    GMG_CUDA_TRY(cudaMemcpyAsync(h->h_res2, h->d_res2, sizeof(double), cudaMemcpyDeviceToHost,
                                 h->stream));
    GMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    // sigma = (h^2 f - A'u) / (2d)
    *norm_out = (2.0 * c.d) * std::sqrt(*h->h_res2);
    return GMG_OK;
}

gmg_status gmg_set_learned_weights(gmg_handle h, int level, const float* weights) {
    if (!h) {
        set_error("handle is NULL");
        return GMG_ERR_ARG;
    }
    if (h->cfg.smoother != GMG_LEARNED) {
        set_error("the handle was not created with smoother GMG_LEARNED");
        return GMG_ERR_ARG;
    }
    if (level < 0 || level >= (int)h->lw.size()) {
        set_error("level out of range");
        return GMG_ERR_ARG;
    }
    DeviceGuard guard(h->device);
    GMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (!weights) {
        h->lw[level] = nullptr;
    } else {
        gmg_status st;
        if (!h->lz[level]) {
            float* z = nullptr;
            if ((st = dev_alloc(h, &z, 8 * h->lv[level].nodes)) != GMG_OK) return st;
            h->lz[level] = z;
        }
        // keep a device copy per level (the pointer stays valid until destroy)
        float* w = nullptr;
        if ((st = dev_alloc(h, &w, 2 * 8 * 27)) != GMG_OK) return st;
        learned::upload_weights(h->cfg.d, weights, w, h->lw_scratch, h->stream);
        GMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
        h->lw[level] = w;
    }
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        h->graph_u = nullptr;
    }
    return GMG_OK;
}

gmg_status gmg_set_timing(gmg_handle h, int enable) {
    if (!h) {
        set_error("handle is NULL");
        return GMG_ERR_ARG;
    }
    if ((enable != 0) != h->timer.enabled) {
        DeviceGuard guard(h->device);
        h->timer.enabled = enable != 0;
        if (h->graph) {
            GMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
            cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
            h->graph_u = nullptr;
        }
    }
    return GMG_OK;
}

gmg_status gmg_timing_reset(gmg_handle h) {
    if (!h) {
        set_error("handle is NULL");
        return GMG_ERR_ARG;
    }
    h->timer.reset();
    return GMG_OK;
}

gmg_status gmg_timing_report(gmg_handle h, gmg_kernel_stat* out, int cap, int* count,
                             int64_t* launches_out) {
    if (!h || (!out && cap > 0)) {
        set_error("bad arguments");
        return GMG_ERR_ARG;
    }
    h->timer.report(out, cap, count, launches_out);
    return GMG_OK;
}

gmg_status gmg_history(gmg_handle h, double* relres, int cap, int* count) {
    if (!h || (!relres && cap > 0)) {
        set_error("bad arguments");
        return GMG_ERR_ARG;
    }
    const int m = (int)h->hist.size();
    for (int i = 0; i < m && i < cap; ++i) relres[i] = h->hist[i];
    if (count) *count = m;
    return GMG_OK;
}

gmg_status gmg_smoother_train(gmg_handle h, const gmg_train_config* tc, const float* w_init,
                              double* loss_history) {
    if (!h || !tc) {
        set_error("handle / train config is NULL");
        return GMG_ERR_ARG;
    }
    if (h->cfg.smoother != GMG_LEARNED) {
        set_error("the handle was not created with smoother GMG_LEARNED");
        return GMG_ERR_ARG;
    }
    const int d = h->cfg.d, T = d == 3 ? 27 : 9;
    std::vector<float> w0(2 * 8 * T, 0.f), w(2 * 8 * T, 0.f);
    if (w_init) {
        std::copy(w_init, w_init + 2 * 8 * T, w0.begin());
    } else {
        // weighted Jacobi, N(sigma) = omega * sigma (relu(x) - relu(-x) = x)
        const float om = (float)(tc->omega_init > 0.0 ? tc->omega_init : d == 3 ? 6.0 / 7.0 : 0.8);
        w0[0 * T + T / 2] = 1.f;
        w0[1 * T + T / 2] = -1.f;
        w0[8 * T + 0 * T + T / 2] = om;
        w0[8 * T + 1 * T + T / 2] = -om;
    }
    gmg_status st = gmg_learned_train(d, tc->n, tc->steps, tc->batch, tc->pair_cycles,
                                      tc->coarse_cycles, tc->lr, tc->seed, w0.data(), w.data(),
                                      loss_history, (void*)h->user_stream);
    if (st != GMG_OK) return st;
    if (tc->select_f) {
        // the fallback: keep the trained weights only where they lower the
        // measured contraction on the caller's problem
        std::vector<const float*> cand(h->lw.size(), nullptr);
        for (int l = 0; l < (int)cand.size() && l < 32; ++l)
            if ((tc->level_mask >> l) & 1u) cand[l] = w.data();
        return gmg_smoother_select(h, tc->select_f, cand.data(), (int)cand.size(), 8, 2,
                                   nullptr, nullptr, nullptr);
    }
    for (int l = 0; l < (int)h->lw.size() && l < 32; ++l)
        if ((tc->level_mask >> l) & 1u)
            if ((st = gmg_set_learned_weights(h, l, w.data())) != GMG_OK) return st;
    return GMG_OK;
}

gmg_status gmg_smoother_select(gmg_handle h, const double* f, const float* const* candidates,
                               int count, int cycles, int skip, unsigned* kept_mask_out,
                               double* rho_base_out, double* rho_out) {
    if (!h || (!candidates && count > 0)) {
        set_error("handle / candidates is NULL");
        return GMG_ERR_ARG;
    }
    if (h->cfg.smoother != GMG_LEARNED) {
        set_error("the handle was not created with smoother GMG_LEARNED");
        return GMG_ERR_ARG;
    }
    if (count < 0 || count > (int)h->lw.size() || count > 32) {
        set_error("count must be in [0, levels of the handle] (at most 32)");
        return GMG_ERR_ARG;
    }
    if (skip < 0 || cycles < skip + 2 || cycles > 1000) {
        set_error("need 0 <= skip and skip + 2 <= cycles <= 1000");
        return GMG_ERR_ARG;
    }
    gmg_status st = check_device_ptr(f, "f");
    if (st != GMG_OK) return st;
    DeviceGuard guard(h->device);
    const int64_t m = h->lv[0].nodes;
    if (!h->f_stage) {
        if ((st = dev_alloc(h, &h->f_stage, m)) != GMG_OK) return st;
        if ((st = dev_alloc(h, &h->u_stage, m)) != GMG_OK) return st;
    }
    std::vector<double> rel(cycles);
    // geometric mean of the residual reduction of cycles skip+1 .. cycles-1
    // of a solve from u = 0
    auto contraction = [&](double* rho) -> gmg_status {
        GMG_CUDA_TRY(cudaEventRecord(h->ev, h->user_stream));
        GMG_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev, 0));
        GMG_CUDA_TRY(cudaMemsetAsync(h->u_stage, 0, sizeof(double) * m, h->stream));
        GMG_CUDA_TRY(cudaEventRecord(h->ev, h->stream));
        GMG_CUDA_TRY(cudaStreamWaitEvent(h->user_stream, h->ev, 0));
        gmg_status s = run(h, f, h->u_stage, 0.0, cycles, false, nullptr, rel.data());
        if (s != GMG_OK) return s;
        const double a = rel[cycles - 1], b = rel[skip];
        *rho = (b > 0.0 && a >= 0.0) ? std::pow(a / b, 1.0 / (cycles - 1 - skip))
                                     : std::numeric_limits<double>::infinity();
        if (!std::isfinite(*rho)) *rho = std::numeric_limits<double>::infinity();
        return GMG_OK;
    };
    for (int l = 0; l < (int)h->lw.size(); ++l)
        if ((st = gmg_set_learned_weights(h, l, nullptr)) != GMG_OK) return st;
    double base = 0.0;
    if ((st = contraction(&base)) != GMG_OK) return st;
    double best = base;
    unsigned kept = 0;
    for (int l = 0; l < count; ++l) {
        if (!candidates[l]) continue;
        if ((st = gmg_set_learned_weights(h, l, candidates[l])) != GMG_OK) return st;
        double rho = 0.0;
        if ((st = contraction(&rho)) != GMG_OK) return st;
        if (rho < best) {
            best = rho;
            kept |= 1u << l;
        } else if ((st = gmg_set_learned_weights(h, l, nullptr)) != GMG_OK) {
            return st;
        }
    }
    if (kept_mask_out) *kept_mask_out = kept;
    if (rho_base_out) *rho_base_out = base;
    if (rho_out) *rho_out = best;
    return GMG_OK;
}

gmg_status gmg_smoother_save(gmg_handle h, void* blob, size_t cap, size_t* bytes_out) {
    if (!h || !bytes_out || (!blob && cap > 0)) {
        set_error("bad arguments");
        return GMG_ERR_ARG;
    }
    if (h->cfg.smoother != GMG_LEARNED) {
        set_error("the handle was not created with smoother GMG_LEARNED");
        return GMG_ERR_ARG;
    }
    const int T = h->cfg.d == 3 ? 27 : 9;
    const size_t wbytes = sizeof(float) * 2 * 8 * T;
    size_t need = 0;
    for (float* w : h->lw) need += sizeof(int32_t) + (w ? wbytes : 0);
    *bytes_out = need;
    if (!blob) return GMG_OK;
    if (cap < need) {
        set_error("blob too small");
        return GMG_ERR_ARG;
    }
    DeviceGuard guard(h->device);
    GMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    unsigned char* p = static_cast<unsigned char*>(blob);
    for (float* w : h->lw) {
        const int32_t flag = w ? 1 : 0;
        std::memcpy(p, &flag, sizeof(flag));
        p += sizeof(flag);
        if (w) {
            GMG_CUDA_TRY(cudaMemcpy(p, w, wbytes, cudaMemcpyDeviceToHost));
            p += wbytes;
        }
    }
    return GMG_OK;
}

gmg_status gmg_smoother_load(gmg_handle h, const void* blob, size_t bytes) {
    if (!h || !blob) {
        set_error("handle / blob is NULL");
        return GMG_ERR_ARG;
    }
    if (h->cfg.smoother != GMG_LEARNED) {
        set_error("the handle was not created with smoother GMG_LEARNED");
        return GMG_ERR_ARG;
    }
    const int T = h->cfg.d == 3 ? 27 : 9;
    const size_t wbytes = sizeof(float) * 2 * 8 * T;
    // parse the whole blob before changing any level
    const unsigned char* p = static_cast<const unsigned char*>(blob);
    const unsigned char* end = p + bytes;
    std::vector<const float*> ws;
    for (size_t l = 0; l < h->lw.size(); ++l) {
        int32_t flag = 0;
        if (end - p < (ptrdiff_t)sizeof(flag)) {
            set_error("blob truncated");
            return GMG_ERR_ARG;
        }
        std::memcpy(&flag, p, sizeof(flag));
        p += sizeof(flag);
        if (flag != 0 && flag != 1) {
            set_error("blob: bad level flag");
            return GMG_ERR_ARG;
        }
        if (flag) {
            if (end - p < (ptrdiff_t)wbytes) {
                set_error("blob truncated");
                return GMG_ERR_ARG;
            }
            ws.push_back(reinterpret_cast<const float*>(p));
            p += wbytes;
        } else {
            ws.push_back(nullptr);
        }
    }
    if (p != end) {
        set_error("blob size does not match the handle's levels");
        return GMG_ERR_ARG;
    }
    for (size_t l = 0; l < ws.size(); ++l) {
        std::vector<float> w;
        const float* src = ws[l];
        if (src) {  // the blob need not be float-aligned
            w.resize(2 * 8 * T);
            std::memcpy(w.data(), src, wbytes);
        }
        gmg_status st = gmg_set_learned_weights(h, (int)l, src ? w.data() : nullptr);
        if (st != GMG_OK) return st;
    }
    return GMG_OK;
}

}  // extern "C"
