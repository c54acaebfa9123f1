/*
 * gmg.h -- C ABI of the GB300 geometric multigrid (GMG) library for the
 * finite-difference Poisson equation
 *
 *     -Laplace(u) = f in (0,1)^d,  u = 0 on the boundary,  d = 2 or 3,
 *
 * discretised by the 5-point (2D) / 7-point (3D) central-difference scheme on
 * a uniform grid with n intervals per dimension (h = 1/n), section 2.2 of
 * Feng, Shu, Xu & Zhang, "Numerical Study of Geometric Multigrid Methods on
 * CPU-GPU Heterogeneous Computers" (arXiv:1208.4247).  The solver runs the
 * V-cycle of Algorithm 1 inside the stopping loop of Algorithm 3 (GMGSolve),
 * with every level on the GPU.
 *
 * Array convention for every f / u argument: double precision, all (n+1)^d
 * grid nodes including the boundary, C order with x fastest (element
 * ((k*(n+1)) + j)*(n+1) + i; k = 0 in 2D), densely packed.  f on boundary
 * nodes is ignored; the solver writes 0 to u's boundary nodes.
 *
 * Ownership: the caller owns f and u.  A handle owns the level hierarchy
 * (about 3.3-4 N values, section 4 remark on space complexity) and a CUDA
 * graph of one cycle; it is bound to the CUDA device current at
 * gmg_create and to the stream given there.
 *
 * Errors: every call returns a gmg_status; on failure gmg_last_error()
 * returns a message for the calling thread (valid until its next call).
 * No call aborts the process.  Calls on one handle must not run
 * concurrently from several threads.
 */
#ifndef GMG_H
#define GMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GMG_OK = 0,
    GMG_ERR_ARG = 1,            /* bad argument or configuration */
    GMG_ERR_LAYOUT = 2,         /* pointer not usable (null, host vs device, misaligned) */
    GMG_ERR_ALLOC = 3,          /* device or pinned host allocation failed */
    GMG_ERR_CUDA = 4,           /* a CUDA runtime call failed */
    GMG_ERR_NONFINITE = 5,      /* residual norm became NaN / Inf */
    GMG_ERR_NOT_CONVERGED = 6,  /* maxit reached; u holds the last iterate */
    GMG_ERR_DEVICE_TIMEOUT = 7, /* a bounded device-side wait gave up */
    GMG_ERR_UNSUPPORTED = 8     /* configuration not built in this library */
} gmg_status;

/* GMG_MCGS: the paper's own smoother (Remark 1 of section 3.2): Gauss-Seidel
 * in four colours (2D) or eight (3D), colour (i&1) + 2(j&1) + 4(k&1), in
 * increasing colour order in pre-smoothing and decreasing order in
 * post-smoothing (Relax_forward / Relax_backward of Algorithm 1). */
typedef enum { GMG_WJACOBI = 0, GMG_RBGS = 1, GMG_LEARNED = 2, GMG_MCGS = 3 } gmg_smoother;
/* Grid transfers: full weighting + (bi/tri)linear interpolation, or the
 * paper's own pair -- the 7-point (2D) / 15-point (3D) restriction of eq.
 * Restriction2d (weight 1/2^d at 2I, 1/2^(d+1) at 2I +- delta, delta in
 * {0,1}^d nonzero) and the diagonal-linear prolongation of eq.
 * Prolongation2d (fine 2I + delta takes (e_I + e_{I+delta})/2). */
typedef enum { GMG_TRANSFER_FW = 0, GMG_TRANSFER_PAPER = 1 } gmg_transfer;
/* GMG_DF_IR: FP64 iterative refinement whose inner V-cycles run in
 * double-float arithmetic (each value the unevaluated sum of two FP32
 * numbers, about 48 significant bits, 8 bytes) on the FP32 pipe.  With
 * inner_cycles = 1 a refinement step u <- u + V(b - A'u) equals one FP64
 * V-cycle in exact arithmetic (the cycle is affine in u), and its rounding
 * scales with the correction rather than with u: every step agrees with the
 * plain FP64 cycle to far below 1e-12 (relative), so a solve takes the plain
 * form's cycle count.  FP64 stays on the GPU for the outer residual, its
 * norm and the update u += e. */
typedef enum { GMG_FP64 = 0, GMG_FP32_IR = 1, GMG_BF16_IR = 2, GMG_DF_IR = 3 } gmg_precision;
typedef enum { GMG_VCYCLE = 0, GMG_FMG = 1 } gmg_cycle;

typedef struct {
    int d;             /* 2 or 3 */
    int n;             /* intervals per dimension: a power of two, 2..4096 (2D) / 2..1024 (3D) */
    int levels;        /* grids in the hierarchy (Algorithm 1's L); 0 = down to n = 2,
                          whose single unknown is solved exactly (Remark, coarsest level) */
    int smoother;      /* gmg_smoother: weighted Jacobi or red-black Gauss-Seidel
                          (red = i+j+k even, red before black in pre- and post-smoothing) */
    double omega;      /* weighted-Jacobi weight (ignored by red-black GS) */
    int nu1, nu2;      /* pre- / post-smoothing sweeps (Algorithm 1's mu_f, mu_b), 0..16 */
    int cycle;         /* gmg_cycle: GMG_VCYCLE, or GMG_FMG: the first cycle of a solve is one
                          full-multigrid pass (Algorithm 2: the right-hand side restricted
                          to every level, coarsest solved, then per level interpolation of
                          the coarse solution and one V-cycle; the initial u is ignored),
                          the following ones V-cycles (plain FP64, GS or Jacobi only) */
    int precision;     /* gmg_precision: plain FP64, or FP32 / BF16 / double-float
                          V-cycles inside FP64 iterative refinement */
    int maxit;         /* cap on V-cycles (FP64) or on outer refinement steps */
    int inner_cycles;  /* refinement forms: V-cycles per outer refinement step (double-float:
                          1 gives the plain FP64 cycle) */
    int coarse_sweeps; /* red-black sweeps from zero on a coarsest grid with more than
                          one unknown (truncated hierarchy); unused otherwise */
    int transfer;      /* gmg_transfer.  GMG_MCGS and GMG_TRANSFER_PAPER run in the plain
                          FP64 form (V-cycles or FMG), every level on grid kernels */
} gmg_config;

typedef struct gmg_handle_s* gmg_handle;

/* Fill *cfg with defaults for d, n: all levels, red-black GS, omega = 4/5,
 * V(2,2), plain FP64, maxit 100, 4 inner cycles, 64 coarse sweeps, full-weighting
 * transfers. */
gmg_status gmg_config_init(gmg_config* cfg, int d, int n);

/* Create a solver for *cfg on the current CUDA device: the grid hierarchy of
 * Algorithm 1 (n, n/2, ..., down to the 3^d grid or cfg->levels grids;
 * section 3.1) with its per-level arrays.  cuda_stream is a cudaStream_t
 * (NULL = legacy default stream) on which every later call on the handle is
 * ordered.  Allocates the level hierarchy on the device; *out receives the
 * handle, owned by the caller until gmg_destroy.  Errors: GMG_ERR_ARG for a
 * bad configuration (before any device work), GMG_ERR_ALLOC when device
 * memory runs out (nothing is left allocated), GMG_ERR_CUDA otherwise.
 * Environment: GMG_FUSED_RB=1 makes GMG_FP32_IR handles in 3D with red-black
 * smoothing run each sweep as one fused z-streaming kernel on a dense inner
 * layout instead of two half sweeps on the colour-split one (same results
 * bit for bit; slower on GB300, see the design notes).  GMG_TAIL_N=m sets the
 * largest level n handled by the single-CTA tail launch (default 8 in 3D,
 * 32 in 2D; 1 turns the tail off); results are the same bit for bit.
 * GMG_RB_WALK=0 (read once per process) replaces the diagonal-walker FP64 3D
 * half sweeps, red-only residuals and norms (levels 128 <= n <= 512) by row
 * kernels; results are the same bit for bit.  GMG_NORM_AHEAD=0 (read once
 * per process) keeps the stopping-test norm of the plain red-black form a
 * separate kernel instead of fusing it with the next cycle's first red half
 * sweep (3D levels 128 <= n <= 512; a solve that stops undoes that sweep);
 * u and the cycle count are the same bit for bit, the norms agree to
 * rounding.  GMG_OUTER_RED=0 makes GMG_DF_IR red-black handles update u and
 * form the outer residual on every node (separate kernels) instead of on
 * the red nodes only (the black residual after a black inner half sweep is
 * zero up to the inner rounding); the results agree to that rounding.
 * GMG_INNER_AHEAD=0 makes red-black refinement forms
 * zero the correction and run the first inner red half sweep as kernels of
 * their own instead of having the outer residual write that half sweep's
 * result (sigma on red nodes, 0 on black); results are the same bit for
 * bit.  GMG_DF_STEP_CYCLES=k (default 8) sets, for GMG_DF_IR red-black
 * handles with one inner cycle, the V-cycles per FP64 refinement step after
 * a solve's first step (which has one): the FP64 update, residual and norm
 * follow every k-th cycle, while the stopping test still runs after every
 * cycle (on the inner residual, folded into the next red half sweep, which
 * is undone when the test stops); k = 1 runs the FP64 step after every
 * cycle.  Cycle counts are the same; iterates agree to the double-float
 * rounding of the correction (far below 1e-12 of u per cycle).
 * GMG_FUSED_LEGS=0/1 turns the fused leg kernels off / on for every FP32
 * and double-float level that takes them (default: FP32 levels n >= 512);
 * GMG_LEG_NMIN / GMG_LEG_NMAX bound the level sizes; results are the same bit
 * for bit.  GMG_GRID_TAIL_N=m runs the levels with n <= m (red-black) and
 * all smaller ones as one cooperative launch with grid barriers between the
 * steps, the levels with n <= GMG_GRID_TAIL_CTA_N (default 8) in one CTA of
 * it (default off: slower than the per-level kernels on GB300);
 * GMG_GRID_TAIL_CLUSTER=c (2..16) runs it as one thread-block cluster of c
 * CTAs with the hardware cluster barrier instead; results are the same bit
 * for bit (3D FP64: levels n <= 64). */
gmg_status gmg_create(const gmg_config* cfg, void* cuda_stream, gmg_handle* out);

/* GMGSolve (Algorithm 3, all levels on the device): starting from the initial
 * guess in u, run cycles while ||h^2 f - A'u||_2 > rtol * ||h^2 f - A'u_0||_2
 * (A' the unscaled 5/7-point operator, norm over interior nodes) and fewer
 * than maxit cycles have run.  f, u: device pointers (layout above).
 * iters_out (may be NULL): cycles run.  relres_out (may be NULL): final
 * relative residual.  Returns GMG_ERR_NOT_CONVERGED with a valid u when
 * maxit stops the loop.  The stopping test runs on the device: the cycles
 * after the first run as one graph launch whose while node repeats a cycle
 * and its norm until the test fails, and the host synchronises once per
 * solve (once per cycle while per-kernel timing is on, or with
 * GMG_DEVICE_LOOP=0 at create; results are the same bit for bit). */
gmg_status gmg_solve(gmg_handle h, const double* f, double* u, double rtol,
                     int* iters_out, double* relres_out);

/* Algorithm 3 as gmg_solve, but f and u are HOST pointers: f and the initial
 * u are copied to device buffers owned by the handle, the solve runs, u is
 * copied back.  Errors as gmg_solve. */
gmg_status gmg_solve_host(gmg_handle h, const double* f_host, double* u_host, double rtol,
                          int* iters_out, double* relres_out);

/* Exactly ncycles cycles of Algorithm 1 from the given u (no stopping test),
 * e.g. for per-cycle comparisons.  relres_out (may be NULL, else ncycles
 * entries) receives ||h^2 f - A'u|| / ||h^2 f - A'u_0|| after each cycle.
 * f, u: device pointers. */
gmg_status gmg_cycles(gmg_handle h, const double* f, double* u, int ncycles,
                      double* relres_out);

/* FP64 residual norm ||h^2 f - A'u||_2 over the interior nodes (Algorithm 3's
 * res), written to *norm_out (host).  Writes 0 to u's boundary nodes, as
 * gmg_solve does.  f, u: device pointers.  Synchronises the handle's stream. */
gmg_status gmg_residual_norm(gmg_handle h, const double* f, double* u, double* norm_out);

/* Allocation-free variant of gmg_residual_norm (the paper has no counterpart;
 * this is a library service).  For callers that cannot allocate device memory
 * when they need the residual -- e.g. code running inside a device-allocator
 * or memory-pool callback, or a real-time loop where cudaMalloc/cudaFree
 * (which may synchronise the device) are forbidden -- and so cannot create a
 * gmg_handle.  No handle: d, n as in gmg_config; f, u: device pointers in the
 * layout above (u is read only, its boundary nodes are taken as 0);
 * norm_dev: device pointer to one double that receives ||h^2 f - A'u||_2.
 * The call runs on the current CUDA device: f, u and norm_dev must be 8-byte
 * aligned device memory of that device (or managed memory), else
 * GMG_ERR_LAYOUT before anything is launched.  Stream-ordered on cuda_stream
 * (a cudaStream_t, NULL = legacy default stream); no host synchronisation,
 * no allocation of any kind.  The result equals gmg_residual_norm's to
 * rounding (its own summation order).
 * Scratch: a fixed 512 KiB static device array (65536 partial sums) that each
 * GPU loading the library holds until exit; grids needing more partial sums
 * than that (3D n > 256) are rejected with GMG_ERR_ARG.  Every call looks up
 * the array's device address on the current device (cudaGetSymbolAddress,
 * which allocates nothing, so the address stays right after a
 * cudaDeviceReset); the first call on a device may load the library's device
 * code there, so make that first call before any stream capture.  All calls
 * share the array, so calls that overlap on the GPU race and must be
 * serialised by the caller. */
gmg_status gmg_residual_norm_noalloc(int d, int n, const double* f, const double* u,
                                     double* norm_dev, void* cuda_stream);

/* Relative-residual history of the last solve / cycles call (Algorithm 3's
 * res / res_0 after each cycle): writes up to cap entries to relres (host),
 * the count to *count (count may be NULL).  GMG_ERR_ARG for a NULL handle or
 * a NULL relres with cap > 0. */
gmg_status gmg_history(gmg_handle h, double* relres, int cap, int* count);

/* Per-kernel device timing (diagnostics, the paper's per-function and
 * per-level profiles of section 5.3).  While enabled, every kernel of the
 * cycle graph is bracketed by CUDA events recorded on the handle's stream,
 * and after each cycle its device time is added to a record keyed by
 * (kernel, level).  Enabling or disabling re-captures the cycle graph. */
gmg_status gmg_set_timing(gmg_handle h, int enable);

typedef struct {
    char kernel[24];   /* kernel name, e.g. "rb_half", "restrict", "resnorm" */
    int level;         /* grid level (0 = finest) */
    int64_t launches;  /* launches timed since the last reset */
    double ms;         /* summed device time of those launches */
    double dp_ops;     /* FP64 pipe instructions per launch (arithmetic model) */
    double bytes;      /* algorithmic DRAM bytes per launch (each value read/written once) */
} gmg_kernel_stat;

/* Copy up to cap records to out (host); *count receives the number of
 * records.  *launches_out (may be NULL) receives every kernel launch the
 * handle made since the last reset, timed or not. */
gmg_status gmg_timing_report(gmg_handle h, gmg_kernel_stat* out, int cap, int* count,
                             int64_t* launches_out);

/* Zero the timing records and the launch counter (section 5.3 profiles). */
gmg_status gmg_timing_reset(gmg_handle h);

/* ------------------------------------------------------- learned smoother
 * A per-level convolutional smoother u <- u + N(sigma), sigma = (h^2 f - A'u)
 * / (2d) the scaled residual, N = conv2(ReLU(conv1(sigma))): conv1 maps 1 -> 8
 * channels, conv2 maps 8 -> 1, both 3^d taps over the interior nodes with zero
 * padding at the Dirichlet boundary, no biases; BF16 weights (the library
 * rounds what it is given, round-to-nearest-even), FP32 accumulation.  The
 * paper has no learned component: this replaces one pre- and one post-
 * smoothing sweep of its V-cycle (Algorithm 1) on the levels given weights.
 * Weights: 2 x 8 x T floats (T = 27 in 3D, 9 in 2D), W1[c][t] then W2[c][t],
 * tap t = (c3+1)*9 + (b+1)*3 + (a+1) for the offset (a, b, c3) in {-1,0,1}^d
 * (x fastest). */
#define GMG_LEARNED_HIDDEN 8

/* Use weights (host, layout above; NULL = red-black GS) on `level` of a handle
 * created with smoother GMG_LEARNED (precision GMG_FP64).  Levels without
 * weights smooth with red-black GS.  A learned sweep is the FP64 residual
 * then the fused tensor-core network (gmg_learned_conv, tensor_cores = 1)
 * added to u.  Re-captures the cycle graph. */
gmg_status gmg_set_learned_weights(gmg_handle h, int level, const float* weights);

/* No counterpart in the paper (the learned smoother above).
 * y = N(x) on the interior nodes of a 2D/3D grid of n intervals (x, y:
 * device FP64, all nodes; x zero on the boundary).  tensor_cores = 0: CUDA-
 * core kernels with FP32 activations (the training path); 1: the fused
 * tensor-core kernel the V-cycle uses (BF16 x and hidden activations,
 * mma.sync m16n8k16, FP32 sums).  Synchronises cuda_stream. */
gmg_status gmg_learned_conv(int d, int n, const float* weights, const double* x, double* y,
                            int tensor_cores, void* cuda_stream);

/* No counterpart in the paper (the learned smoother's training loss).
 * Two-grid contraction loss L = ||S(CG(S(e0)))||^2 / ||e0||^2 of the error e0
 * (device FP64, all nodes, zero boundary) on a grid of n intervals, with
 * S e = e - N(A'e/(2d)) and CG e = e - P A_c'^{-1} 4 FW(A'e), the coarse
 * system solved by coarse_cycles red-black V(2,2) cycles.  *loss_out: L;
 * grad_out (host, 2 x 8 x T doubles, may be NULL): dL/dW at the BF16-rounded
 * weights.  Synchronises cuda_stream. */
gmg_status gmg_learned_loss_grad(int d, int n, const float* weights, const double* e0,
                                 int coarse_cycles, double* loss_out, double* grad_out,
                                 void* cuda_stream);

/* No counterpart in the paper (training of the learned smoother).
 * Train the weights on the GPU: `steps` Adam steps (learning rate lr) on the
 * mean two-grid loss over `batch` error samples per step, each sample the
 * error left by pair_cycles plain red-black V(1,1) cycles applied to seeded
 * white noise (seed) on a grid of n intervals.  w_init -> w_out (host, layout
 * above; FP32 master weights); loss_history (host, `steps` doubles, may be
 * NULL): the mean loss of each step's batch.  Synchronises cuda_stream. */
gmg_status gmg_learned_train(int d, int n, int steps, int batch, int pair_cycles,
                             int coarse_cycles, double lr, uint64_t seed, const float* w_init,
                             float* w_out, double* loss_history, void* cuda_stream);

/* ------------------------------------------------------------ FFT solve
 * The paper's comparison method (section 2.3): a direct solve of the same FD
 * system A'u = h^2 f by sine transforms, u = S^-1 diag(1/lambda) S h^2 f with
 * S the DST-I along every axis and lambda_k = sum_m 4 sin^2(pi k_m / (2n))
 * the discrete eigenvalues (the paper writes the continuous symbol), each
 * DST-I done by a length-2n cuFFT D2Z of the odd extension. */
typedef struct gmg_fft_s* gmg_fft;

/* d = 2 or 3, n a power of two (2D up to 8192, 3D up to 1024); allocates
 * about 3 (n+1)^d doubles of work space and two cuFFT plans. */
gmg_status gmg_fft_create(int d, int n, void* cuda_stream, gmg_fft* out);
/* Section 2.3: u = A'^-1 h^2 f on the interior, 0 on the boundary (f, u
 * device pointers, layout above).  Synchronises the handle's stream.
 * Errors: GMG_ERR_ARG for NULL arguments, GMG_ERR_CUDA for a failed
 * transform or launch. */
gmg_status gmg_fft_solve(gmg_fft h, const double* f, double* u);
/* Release the plans and work space of h.  NULL is a no-op. */
gmg_status gmg_fft_destroy(gmg_fft h);

/* ---------------------------------------------------------------- batches
 * Many independent solves of uneven sizes (2D and 3D mixed) advanced
 * together: every step launches one persistent kernel per level index over
 * the whole batch (work items = chunks of one solve's level grid), so the
 * coarse levels of the large solves share launches with the fine levels of
 * the small ones.  Levels are aligned at the coarsest (3^d) grid.  Cycles run
 * in the inner precision of *common (GMG_FP32_IR or GMG_BF16_IR: FP64 outer
 * residual, update and norm; GMG_FP64: plain cycles) with its smoother and
 * sweeps; each solve stops on its own FP64 relative residual (converged
 * solves are masked on the device).  One refinement step of the whole batch
 * is one captured CUDA graph.  No counterpart in the paper: each solve runs
 * Algorithms 1 and 3, the batching is this library's. */
typedef struct gmg_batch_s* gmg_batch;

/* count solves; d[i], n[i] per solve (as in gmg_config); *common gives the
 * smoother, omega, nu1, nu2, precision, inner_cycles and maxit (its d, n,
 * levels are ignored: every solve uses all its levels).  omega = 0 gives the
 * 2D solves weighted Jacobi with 4/5 and the 3D ones 6/7 (the weight with the
 * smaller two-grid contraction in 3D); any other omega in (0, 2) applies to
 * every solve.  chunk: nodes per
 * work item (0 = 1024); ctas: CTAs per launch (0 = 4 x SM count). */
gmg_status gmg_batch_create(int count, const int* d, const int* n, const gmg_config* common,
                            int chunk, int ctas, void* cuda_stream, gmg_batch* out);

/* f[i], u[i]: device pointers of solve i (layout above), u[i] the initial
 * guess.  iters_out[count] (may be NULL): steps each solve ran;
 * relres_out[count] (may be NULL): each final relative residual.
 * *steps_out (may be NULL): batch steps launched.  Returns
 * GMG_ERR_NOT_CONVERGED if any solve hit maxit. */
gmg_status gmg_batch_solve(gmg_batch b, const double* const* f, double* const* u, double rtol,
                           int* iters_out, double* relres_out, int* steps_out);

/* Per-kernel timing of the batch graph, as gmg_set_timing / gmg_timing_report
 * (section 5.3 profiles). */
gmg_status gmg_batch_set_timing(gmg_batch b, int enable);
gmg_status gmg_batch_timing_report(gmg_batch b, gmg_kernel_stat* out, int cap, int* count,
                                   int64_t* launches_out);

/* Release every device and host resource of the batch.  NULL is a no-op. */
gmg_status gmg_batch_destroy(gmg_batch b);

/* ------------------------------------------- the problem statement's names
 * The solver interface as the problem statement names it (Algorithm 3's
 * GMGSolve on caller arrays with row pitches, the batched form, and training
 * and persistence of the learned smoother); wrappers over the calls above. */

/* gmg_solve on arrays with pitches: node (i, j, k) of f and u at
 * k*strides[2] + j*strides[1] + i (elements; strides[0] must be 1,
 * strides[1] >= n+1, 3D: strides[2] >= strides[1]*(n+1); strides[2] unused
 * in 2D).  Dense pitches call gmg_solve directly; any other pitch stages f
 * and u through dense device copies owned by the handle (one gather each way
 * and one scatter of u, about 3 (n+1)^d doubles moved twice).  u's boundary
 * nodes are written as 0, the padding is not touched.  Errors as gmg_solve;
 * GMG_ERR_LAYOUT for bad strides. */
gmg_status gmg_solve_strided(gmg_handle h, const double* f, double* u, const int64_t strides[3],
                             double rtol, int* iters_out, double* relres_out);

/* The batched form from one configuration per solve: cfgs[i].d, cfgs[i].n
 * give solve i's grid; smoother, omega, nu1, nu2, precision, inner_cycles and
 * maxit must be the same in every cfgs[i] (else GMG_ERR_ARG).  Default chunk
 * and CTA count (see gmg_batch_create). */
gmg_status gmg_create_batched(int count, const gmg_config* cfgs, void* cuda_stream,
                              gmg_batch* out);
/* gmg_batch_solve without the per-solve residuals and the step count. */
gmg_status gmg_solve_batched(gmg_batch b, const double* const* f, double* const* u, double rtol,
                             int* iters_out);

typedef struct {
    int n;               /* grid of the training samples (intervals per dimension) */
    int steps;           /* Adam steps */
    int batch;           /* error samples per step */
    int pair_cycles;     /* plain red-black V(1,1) cycles applied to white noise per sample */
    int coarse_cycles;   /* red-black V(2,2) cycles for the coarse solve of the loss */
    double lr;           /* Adam learning rate */
    uint64_t seed;       /* seed of the samples' white noise */
    double omega_init;   /* start at weighted Jacobi with this omega if w_init is NULL
                            (<= 0: 6/7 in 3D, 4/5 in 2D) */
    unsigned level_mask; /* bit l set: the trained weights are a candidate for level l */
    const double* select_f; /* NULL: install the trained weights on every level of
                               level_mask.  Else a device f (layout above) of the target
                               problem: keep them on a level only where they lower the
                               measured contraction (gmg_smoother_select, 8 cycles, skip 2);
                               every other level smooths with red-black GS */
} gmg_train_config;

/* Train the learned smoother of h (smoother GMG_LEARNED) with
 * gmg_learned_train on the handle's dimension and install the result on the
 * levels of tc->level_mask (with tc->select_f: on those of them where it
 * beats red-black GS, see gmg_smoother_select).  w_init: starting weights (host, layout of
 * gmg_set_learned_weights) or NULL.  loss_history: tc->steps doubles or
 * NULL.  Synchronises the handle's stream. */
gmg_status gmg_smoother_train(gmg_handle h, const gmg_train_config* tc, const float* w_init,
                              double* loss_history);

/* The learned smoother's fallback (no counterpart in the paper; red-black GS,
 * the smoother of Algorithm 1's relax steps, is what it falls back to).  On
 * the target problem f (device, layout above) measure the V-cycle
 * contraction rho = (r_{cycles-1} / r_skip)^(1 / (cycles-1-skip)), r_c the
 * relative residual after cycle c+1 of a solve from u = 0, first with
 * red-black GS on every level, then level by level from the finest (l = 0
 * .. count-1): candidates[l] (host weights, layout of gmg_set_learned_weights;
 * NULL = no candidate) is installed and kept only if rho falls below the best
 * so far, else that level goes back to red-black GS.  Levels >= count smooth
 * with red-black GS.  When no level keeps its weights, the cycle is the
 * red-black one of the same handle.  kept_mask_out (may be NULL): bit l set
 * for each level that kept its weights; rho_base_out, rho_out (may be NULL):
 * the contraction with red-black GS everywhere and with the kept weights.
 * Uses a work array owned by the handle (allocated on first use); f is only
 * read.  Synchronises the handle's stream.  Errors: GMG_ERR_ARG (handle not
 * GMG_LEARNED, count outside [0, levels], skip < 0, cycles < skip + 2),
 * GMG_ERR_LAYOUT (f not a device pointer), else as gmg_cycles. */
gmg_status gmg_smoother_select(gmg_handle h, const double* f, const float* const* candidates,
                               int count, int cycles, int skip, unsigned* kept_mask_out,
                               double* rho_base_out, double* rho_out);

/* Persistence of the learned smoother of h (smoother GMG_LEARNED).  Blob
 * layout, for each level of the handle in order: int32 flag (1: weights
 * follow, 0: the level smooths with red-black GS), then, if 1, the level's
 * BF16-rounded weights as 2 x 8 x T floats (layout of
 * gmg_set_learned_weights).  save: *bytes_out = the blob size; the blob is
 * written when blob != NULL and cap is large enough (else GMG_ERR_ARG).
 * load: the blob must match the handle's level count exactly (else
 * GMG_ERR_ARG, no level changed). */
gmg_status gmg_smoother_save(gmg_handle h, void* blob, size_t cap, size_t* bytes_out);
gmg_status gmg_smoother_load(gmg_handle h, const void* blob, size_t bytes);

/* Release every device and host resource of the handle.  NULL is a no-op.
 * (A library service; no counterpart in the paper.) */
gmg_status gmg_destroy(gmg_handle h);

/* Message of the calling thread's last failed call ("" if none); owned by
 * the library, valid until that thread's next call.  A library service; no
 * counterpart in the paper. */
const char* gmg_last_error(void);

/* Measured FP64 pipe rate of the current device (a library service; no
 * counterpart in the paper): FP64 instructions per second of one kind (0:
 * fused multiply-add, 1: add) issued by independent chains on every SM,
 * timed with CUDA events on cuda_stream (NULL = legacy default stream) over
 * five launches after a warm-up, into *inst_per_s.  The roofline peak of the
 * FP64-bound kernels.  Synchronises cuda_stream; allocates nothing.
 * Errors: GMG_ERR_ARG (kind not 0/1, NULL inst_per_s), GMG_ERR_CUDA. */
gmg_status gmg_measure_fp64_rate(int kind, double* inst_per_s, void* cuda_stream);

/* Version of this ABI (GMG_ABI_VERSION).  A library service. */
int gmg_abi_version(void);
#define GMG_ABI_VERSION 2

#ifdef __cplusplus
}
#endif

#endif /* GMG_H */
