/*
 * gmg_oracle.c -- plain CPU FP64 oracle for the geometric multigrid (GMG)
 * V-cycle of Feng, Shu, Xu & Zhang, "Numerical Study of Geometric Multigrid
 * Methods on CPU-GPU Heterogeneous Computers" (arXiv:1208.4247).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg load it; the solver library never does, and
 * the two share no source, header, table or helper.
 *
 * Conventions (the paper's section 2.2 and section 4):
 *   - d = 2 or 3, n = 2^k intervals per dimension, h = 1/n, nodes 0..n.
 *   - Arrays hold all (n+1)^d nodes, x fastest: index ((k*(n+1))+j)*(n+1)+i
 *     (k = 0 in 2D).  Only interior nodes 1..n-1 are unknowns; boundary nodes
 *     are read as zero whatever the array holds (Dirichlet data u = 0).
 *   - Every level works in the unscaled form of the 5-/7-point scheme:
 *         A' u = b,  A' u_p = 2d u_p - sum of the 2d neighbours,  b = h^2 f.
 *     On coarse levels b_{l+1} = 4 * FW(r_l), the factor (h_{l+1}/h_l)^2 = 4
 *     taking the residual of the fine unscaled equation to the right-hand side
 *     of the coarse unscaled equation.  All scalings are powers of two.
 *   - Compiled with -ffp-contract=off: every expression is evaluated as
 *     written, one rounding per operation, no fused multiply-add.
 *
 * Pins (tests/test_oracle_pins.py): sine eigenpairs of A' (section 2.2),
 * dense direct solves, sine-transform (DST-I) direct solves at full workload
 * sizes, the closed-form discretisation error that the paper's FFT error
 * tables print, brute-force dense two-grid spectral radii (2D and 3D), the
 * h-independence of the full V-cycle's contraction, the triangular-solve form
 * of red-black Gauss-Seidel, the adjoint relation FW = P^T / 2^d and exact
 * interpolation of linear functions; for the paper's own variant (multi-colour
 * GS, its restriction and prolongation) the same kinds of dense checks, its
 * whole V-cycle as a dense composition, and the iteration counts of its
 * smoother table.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ grid */

static inline int64_t nodes(int d, int n)
{
    int64_t m = n + 1;
    return d == 2 ? m * m : m * m * m;
}

static inline int64_t IDX(int n, int i, int j, int k)
{
    return ((int64_t)k * (n + 1) + j) * (n + 1) + i;
}

static inline int interior(int d, int n, int i, int j, int k)
{
    if (i <= 0 || i >= n || j <= 0 || j >= n) return 0;
    if (d == 3 && (k <= 0 || k >= n)) return 0;
    return 1;
}

/* Value of a grid function at a node; boundary (and outside) nodes are 0. */
static inline double val(const double* u, int d, int n, int i, int j, int k)
{
    return interior(d, n, i, j, k) ? u[IDX(n, i, j, k)] : 0.0;
}

/* Sum of the 2d axis neighbours in the fixed order x-, x+, y-, y+, z-, z+. */
static inline double nbr_sum(const double* u, int d, int n, int i, int j, int k)
{
    double s = val(u, d, n, i - 1, j, k);
    s = s + val(u, d, n, i + 1, j, k);
    s = s + val(u, d, n, i, j - 1, k);
    s = s + val(u, d, n, i, j + 1, k);
    if (d == 3) {
        s = s + val(u, d, n, i, j, k - 1);
        s = s + val(u, d, n, i, j, k + 1);
    }
    return s;
}

static inline int kmin(int d) { return d == 3 ? 1 : 0; }
static inline int kmax(int d, int n) { return d == 3 ? n - 1 : 0; }

/* ------------------------------------------------------- single operators */

/* out = A' u on interior nodes (section 2.2, 5-point / 7-point scheme without
 * the 1/h^2), boundary entries of out set to 0. */
void orc_apply_stencil(int d, int n, const double* u, double* out)
{
    memset(out, 0, sizeof(double) * nodes(d, n));
#pragma omp parallel for schedule(static)
    for (int k = kmin(d); k <= kmax(d, n); ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i)
                out[IDX(n, i, j, k)] = (2.0 * d) * u[IDX(n, i, j, k)] - nbr_sum(u, d, n, i, j, k);
}

/* r = b - A' u (section 4.1, eq. residual_2D; 3D item (1)). */
void orc_residual(int d, int n, const double* b, const double* u, double* r)
{
    memset(r, 0, sizeof(double) * nodes(d, n));
#pragma omp parallel for schedule(static)
    for (int k = kmin(d); k <= kmax(d, n); ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i) {
                int64_t p = IDX(n, i, j, k);
                r[p] = b[p] - ((2.0 * d) * u[p] - nbr_sum(u, d, n, i, j, k));
            }
}

/* Euclidean norm over interior nodes, summed sequentially in index order
 * (section 4.1 eq. Inner_product2D prints the sum of squares; the square root
 * is taken here, see the readings in the design notes). */
double orc_norm2(int d, int n, const double* r)
{
    double s = 0.0;
    for (int k = kmin(d); k <= kmax(d, n); ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i) {
                double v = r[IDX(n, i, j, k)];
                s = s + v * v;
            }
    return sqrt(s);
}

/* Red-black Gauss-Seidel: per sweep, first every interior node with i+j+k
 * even ("red"), then every node with i+j+k odd ("black"); each update solves
 * its own equation, u_p = (b_p + sum of neighbours) / (2d) (section 4.1,
 * eq. relax_2D; two colours as in the smoother comparison table). */
void orc_rbgs(int d, int n, const double* b, double* u, int sweeps)
{
    for (int s = 0; s < sweeps; ++s)
        for (int color = 0; color < 2; ++color) {
#pragma omp parallel for schedule(static)
            for (int k = kmin(d); k <= kmax(d, n); ++k)
                for (int j = 1; j < n; ++j)
                    for (int i = 1; i < n; ++i) {
                        if (((i + j + k) & 1) != color) continue;
                        int64_t p = IDX(n, i, j, k);
                        u[p] = (b[p] + nbr_sum(u, d, n, i, j, k)) / (2.0 * d);
                    }
        }
}

/* Weighted Jacobi: u <- u + omega * (b - A' u) / (2d), all nodes from the
 * previous iterate (Remark 1 of section 3.2; smoother comparison table). */
void orc_wjacobi(int d, int n, const double* b, double* u, double omega, int sweeps)
{
    int64_t m = nodes(d, n);
    double* old = (double*)malloc(sizeof(double) * m);
    for (int s = 0; s < sweeps; ++s) {
        memcpy(old, u, sizeof(double) * m);
#pragma omp parallel for schedule(static)
        for (int k = kmin(d); k <= kmax(d, n); ++k)
            for (int j = 1; j < n; ++j)
                for (int i = 1; i < n; ++i) {
                    int64_t p = IDX(n, i, j, k);
                    double res = b[p] - ((2.0 * d) * old[p] - nbr_sum(old, d, n, i, j, k));
                    u[p] = old[p] + omega * res / (2.0 * d);
                }
    }
    free(old);
}

/* 1D full-weighting weight for an offset -1, 0, +1: 1/4, 1/2, 1/4. */
static inline double fw1(int delta) { return delta == 0 ? 0.5 : 0.25; }

/* bc = 4 * FW(r): full-weighting restriction from the fine grid (n
 * intervals) to the coarse grid (n/2 intervals), tensor product of
 * [1/4 1/2 1/4], times the (h_c/h)^2 = 4 of the unscaled form (Algorithm 1,
 * f_{l+1} = R r_l; the paper's own 7-point R of eq. Restriction2d is replaced
 * by full weighting). */
void orc_restrict_fw(int d, int n, const double* r, double* bc)
{
    int nc = n / 2;
    memset(bc, 0, sizeof(double) * nodes(d, nc));
    int dz = d == 3 ? 1 : 0;
#pragma omp parallel for schedule(static)
    for (int K = kmin(d); K <= kmax(d, nc); ++K)
        for (int J = 1; J < nc; ++J)
            for (int I = 1; I < nc; ++I) {
                double s = 0.0;
                for (int c = -dz; c <= dz; ++c)
                    for (int b = -1; b <= 1; ++b)
                        for (int a = -1; a <= 1; ++a) {
                            double w = fw1(a) * fw1(b) * (d == 3 ? fw1(c) : 1.0);
                            s = s + w * val(r, d, n, 2 * I + a, 2 * J + b, 2 * K + c);
                        }
                bc[IDX(nc, I, J, K)] = 4.0 * s;
            }
}

/* 1D linear-interpolation weights from coarse index c to fine index i:
 * fine even node i = 2c gets 1, fine odd node gets 1/2 from each side. */
static inline double lin1(int i, int c)
{
    int dd = i - 2 * c;
    if (dd == 0) return 1.0;
    if (dd == 1 || dd == -1) return 0.5;
    return 0.0;
}

/* u += P uc: (bi/tri)linear prolongation of the coarse correction (nc
 * intervals) onto the fine grid (2 nc intervals) and correction of u
 * (Algorithm 1, u_l = u_l + P u_{l+1}; the paper's own interpolation of
 * eq. Prolongation2d is replaced by the tensor-product linear one).  Coarse
 * boundary nodes carry the Dirichlet value 0. */
void orc_prolong_add(int d, int nc, const double* uc, double* u)
{
    int n = 2 * nc;
#pragma omp parallel for schedule(static)
    for (int k = kmin(d); k <= kmax(d, n); ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i) {
                double s = 0.0;
                int c0 = (i - 1) / 2, c1 = (i + 1) / 2;
                int e0 = (j - 1) / 2, e1 = (j + 1) / 2;
                int g0 = d == 3 ? (k - 1) / 2 : 0, g1 = d == 3 ? (k + 1) / 2 : 0;
                for (int C = g0; C <= g1; ++C)
                    for (int B = e0; B <= e1; ++B)
                        for (int A = c0; A <= c1; ++A) {
                            double w = lin1(i, A) * lin1(j, B) * (d == 3 ? lin1(k, C) : 1.0);
                            if (w != 0.0) s = s + w * val(uc, d, nc, A, B, C);
                        }
                u[IDX(n, i, j, k)] = u[IDX(n, i, j, k)] + s;
            }
}

/* The paper's own smoother (Remark 1 of section 3.2): Gauss-Seidel in four
 * colours (2D) or eight (3D), colour (i&1) + 2(j&1) + 4(k&1); each update
 * solves its own equation, u_p = (b_p + sum of neighbours) / (2d) (eq.
 * relax_2D).  Forward sweeps take the colours in increasing order, backward
 * ones in decreasing order (Relax_forward / Relax_backward of Algorithm 1). */
void orc_mcgs(int d, int n, const double* b, double* u, int sweeps, int backward)
{
    int ncol = d == 3 ? 8 : 4;
    for (int s = 0; s < sweeps; ++s)
        for (int t = 0; t < ncol; ++t) {
            int color = backward ? ncol - 1 - t : t;
#pragma omp parallel for schedule(static)
            for (int k = kmin(d); k <= kmax(d, n); ++k)
                for (int j = 1; j < n; ++j)
                    for (int i = 1; i < n; ++i) {
                        if ((i & 1) + 2 * (j & 1) + 4 * (k & 1) != color) continue;
                        int64_t p = IDX(n, i, j, k);
                        u[p] = (b[p] + nbr_sum(u, d, n, i, j, k)) / (2.0 * d);
                    }
        }
}

/* The paper's prolongation (eq. Prolongation2d and its 3D analogue, linear
 * interpolation on the triangulation cut along the main diagonal): fine node
 * 2I + delta, delta in {0,1}^d, gets uc(I) for delta = 0 and
 * (uc(I) + uc(I + delta)) / 2 otherwise; u += that.  Coarse boundary nodes
 * carry 0. */
void orc_prolong_diag(int d, int nc, const double* uc, double* u)
{
    int n = 2 * nc;
#pragma omp parallel for schedule(static)
    for (int k = kmin(d); k <= kmax(d, n); ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i) {
                int I = i / 2, J = j / 2, K = k / 2;
                int a = i & 1, bb = j & 1, c = d == 3 ? (k & 1) : 0;
                double e0 = val(uc, d, nc, I, J, d == 3 ? K : 0);
                double s;
                if (a == 0 && bb == 0 && c == 0)
                    s = e0;
                else
                    s = 0.5 * (e0 + val(uc, d, nc, I + a, J + bb, d == 3 ? K + c : 0));
                u[IDX(n, i, j, k)] = u[IDX(n, i, j, k)] + s;
            }
}

/* The paper's restriction (eq. Restriction2d and its 3D analogue: 7 points
 * in 2D, 15 in 3D), the transpose of the diagonal prolongation over 2^d:
 * weight 1/2^d at 2I and 1/2^(d+1) at 2I +- delta for every delta in
 * {0,1}^d other than 0; times the (h_c/h)^2 = 4 of the unscaled form. */
void orc_restrict_simplex(int d, int n, const double* r, double* bc)
{
    int nc = n / 2;
    memset(bc, 0, sizeof(double) * nodes(d, nc));
    int dz = d == 3 ? 1 : 0;
    double w0 = d == 3 ? 0.125 : 0.25;
#pragma omp parallel for schedule(static)
    for (int K = kmin(d); K <= kmax(d, nc); ++K)
        for (int J = 1; J < nc; ++J)
            for (int I = 1; I < nc; ++I) {
                double s = w0 * val(r, d, n, 2 * I, 2 * J, 2 * K);
                for (int c = 0; c <= dz; ++c)
                    for (int b = 0; b <= 1; ++b)
                        for (int a = 0; a <= 1; ++a) {
                            if (a == 0 && b == 0 && c == 0) continue;
                            s = s + 0.5 * w0 * val(r, d, n, 2 * I + a, 2 * J + b, 2 * K + c);
                            s = s + 0.5 * w0 * val(r, d, n, 2 * I - a, 2 * J - b, 2 * K - c);
                        }
                bc[IDX(nc, I, J, K)] = 4.0 * s;
            }
}

/* Coarsest-level solve.  With one unknown (n = 2) the single equation is
 * solved exactly, u = b / (2d) (Remark on the coarsest-level solver).  A
 * coarsest grid with more unknowns (a truncated hierarchy) is solved
 * approximately by `sweeps` red-black sweeps from zero. */
void orc_coarse_solve(int d, int n, const double* b, double* u, int sweeps)
{
    memset(u, 0, sizeof(double) * nodes(d, n));
    if (n == 2) {
        int64_t p = IDX(n, 1, 1, d == 3 ? 1 : 0);
        u[p] = b[p] / (2.0 * d);
        return;
    }
    orc_rbgs(d, n, b, u, sweeps);
}

/* ---------------------------------------------------------------- V-cycle */

enum { ORC_WJACOBI = 0, ORC_RBGS = 1, ORC_MCGS = 3 };

typedef struct {
    int d;             /* 2 or 3 */
    int n;             /* finest intervals per dimension, a power of two */
    int levels;        /* number of grids, finest = 0 .. coarsest = levels-1 */
    int smoother;      /* ORC_WJACOBI, ORC_RBGS or ORC_MCGS */
    double omega;      /* weighted-Jacobi weight */
    int nu1, nu2;      /* pre- and post-smoothing sweeps */
    int coarse_sweeps; /* red-black sweeps when the coarsest grid has > 1 unknown */
    int transfer;      /* 0: full weighting + multilinear P; 1: the paper's R and P */
} orc_cfg;

/* backward: post-smoothing (Relax_backward), which reverses the colour
 * order of the multi-colour smoother */
static void relax(const orc_cfg* c, int n, const double* b, double* u, int sweeps, int backward)
{
    if (c->smoother == ORC_RBGS)
        orc_rbgs(c->d, n, b, u, sweeps);
    else if (c->smoother == ORC_MCGS)
        orc_mcgs(c->d, n, b, u, sweeps, backward);
    else
        orc_wjacobi(c->d, n, b, u, c->omega, sweeps);
}

static void restrict_(const orc_cfg* c, int n, const double* r, double* bc)
{
    if (c->transfer == 1)
        orc_restrict_simplex(c->d, n, r, bc);
    else
        orc_restrict_fw(c->d, n, r, bc);
}

static void prolong_(const orc_cfg* c, int nc, const double* uc, double* u)
{
    if (c->transfer == 1)
        orc_prolong_diag(c->d, nc, uc, u);
    else
        orc_prolong_add(c->d, nc, uc, u);
}

/* One V-cycle (Algorithm 1) on the right-hand side b0 = h^2 f of the finest
 * level, updating u0 in place.  Coarse iterates start from zero on every
 * descent.  Returns 0, or -1 on a bad configuration / allocation failure. */
int orc_vcycle(const orc_cfg* c, const double* b0, double* u0)
{
    int d = c->d, L = c->levels;
    if (L < 1 || (c->n >> (L - 1)) < 2) return -1;
    double** b = (double**)calloc(L, sizeof(double*));
    double** u = (double**)calloc(L, sizeof(double*));
    double* r = (double*)malloc(sizeof(double) * nodes(d, c->n));
    if (!b || !u || !r) return -1;
    b[0] = (double*)b0;
    u[0] = u0;
    for (int l = 1; l < L; ++l) {
        b[l] = (double*)calloc(nodes(d, c->n >> l), sizeof(double));
        u[l] = (double*)calloc(nodes(d, c->n >> l), sizeof(double));
    }
    /* down: relax, residual, restrict (Algorithm 1, first loop) */
    for (int l = 0; l + 1 < L; ++l) {
        int nl = c->n >> l;
        relax(c, nl, b[l], u[l], c->nu1, 0);
        orc_residual(d, nl, b[l], u[l], r);
        restrict_(c, nl, r, b[l + 1]);
        memset(u[l + 1], 0, sizeof(double) * nodes(d, nl / 2));
    }
    /* coarsest level */
    if (L == 1)
        relax(c, c->n, b[0], u[0], c->nu1, 0);
    else
        orc_coarse_solve(d, c->n >> (L - 1), b[L - 1], u[L - 1], c->coarse_sweeps);
    /* up: prolongate-correct, relax (Algorithm 1, second loop, l = L-2..0) */
    for (int l = L - 2; l >= 0; --l) {
        int nl = c->n >> l;
        prolong_(c, nl / 2, u[l + 1], u[l]);
        relax(c, nl, b[l], u[l], c->nu2, 1);
    }
    for (int l = 1; l < L; ++l) {
        free(b[l]);
        free(u[l]);
    }
    free(b);
    free(u);
    free(r);
    return 0;
}

/* b = h^2 f on interior nodes, 0 on the boundary (section 2.2). */
void orc_scale_rhs(int d, int n, const double* f, double* b)
{
    double h = 1.0 / n;
    memset(b, 0, sizeof(double) * nodes(d, n));
    for (int k = kmin(d); k <= kmax(d, n); ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i) {
                int64_t p = IDX(n, i, j, k);
                b[p] = (h * h) * f[p];
            }
}

/* GMGSolve (Algorithm 3 with every level on one device): from the initial
 * guess u, repeat V-cycles while ||b - A'u|| > rtol * ||b - A'u_initial||
 * and fewer than maxit cycles ran.  relres_hist (may be NULL) receives the
 * relative residual after each cycle.  Returns the cycle count, or -1. */
int orc_solve(const orc_cfg* c, const double* f, double* u, double rtol, int maxit,
              double* relres_hist)
{
    int d = c->d, n = c->n;
    int64_t m = nodes(d, n);
    double* b = (double*)malloc(sizeof(double) * m);
    double* r = (double*)malloc(sizeof(double) * m);
    if (!b || !r) return -1;
    orc_scale_rhs(d, n, f, b);
    for (int k = kmin(d); k <= kmax(d, n); ++k)
        for (int j = 0; j <= n; ++j)
            for (int i = 0; i <= n; ++i)
                if (!interior(d, n, i, j, k)) u[IDX(n, i, j, k)] = 0.0;
    if (d == 3) { /* the k = 0 and k = n planes */
        for (int j = 0; j <= n; ++j)
            for (int i = 0; i <= n; ++i) {
                u[IDX(n, i, j, 0)] = 0.0;
                u[IDX(n, i, j, n)] = 0.0;
            }
    }
    orc_residual(d, n, b, u, r);
    double resinit = orc_norm2(d, n, r), res = resinit;
    int iter = 0;
    while (res > rtol * resinit && iter < maxit) {
        if (orc_vcycle(c, b, u) != 0) {
            iter = -1;
            break;
        }
        orc_residual(d, n, b, u, r);
        res = orc_norm2(d, n, r);
        if (relres_hist) relres_hist[iter] = resinit > 0.0 ? res / resinit : 0.0;
        iter++;
    }
    free(b);
    free(r);
    return iter;
}

/* ------------------------------------------------------- learned smoother
 *
 * A per-level convolutional smoother u <- u + N(sigma), sigma = (b - A'u)/(2d)
 * the scaled residual, N = conv2(ReLU(conv1(sigma))): conv1 maps 1 -> H = 8
 * channels, conv2 maps 8 -> 1, both 3^d-tap correlations over the interior
 * nodes with zero padding at the Dirichlet boundary, no biases.  Weights:
 * W1[c][t], W2[c][t], t = (c3+1)*9 + (b+1)*3 + (a+1) for the tap offset
 * (a, b, c3) in {-1,0,1}^d (x fastest; 9 taps in 2D).  In error form
 * (e = u* - u, sigma = A'e/(2d)) one smoothing step is e <- e - N(A'e/(2d)).
 * The loss is the measured two-grid error contraction
 *     L = ||S(CG(S(e0)))||^2 / ||e0||^2,
 * CG(e) = e - P A_c'^{-1} 4 FW(A'e) with the coarse system solved to
 * round-off. */

#define ORC_HID 8

static inline int ntaps(int d) { return d == 3 ? 27 : 9; }
static inline void tap_off(int d, int t, int* a, int* b, int* c)
{
    *a = t % 3 - 1;
    *b = (t / 3) % 3 - 1;
    *c = d == 3 ? t / 9 - 1 : 0;
}

/* z[ch][p] = sum_t W1[ch][t] x(p + o_t); y[p] = sum_ch sum_t W2[ch][t] relu(z[ch](p + o_t)).
 * z: ORC_HID arrays of nodes(d,n) (may be NULL: then allocated internally). */
void orc_conv_fwd(int d, int n, const float* W1, const float* W2, const double* x, double* z,
                  double* y)
{
    int64_t m = nodes(d, n);
    int T = ntaps(d);
    double* zz = z ? z : (double*)malloc(sizeof(double) * m * ORC_HID);
    memset(zz, 0, sizeof(double) * m * ORC_HID);
    memset(y, 0, sizeof(double) * m);
    for (int ch = 0; ch < ORC_HID; ++ch)
        for (int k = kmin(d); k <= kmax(d, n); ++k)
            for (int j = 1; j < n; ++j)
                for (int i = 1; i < n; ++i) {
                    double s = 0.0;
                    for (int t = 0; t < T; ++t) {
                        int a, b, c;
                        tap_off(d, t, &a, &b, &c);
                        s = s + (double)W1[ch * T + t] * val(x, d, n, i + a, j + b, k + c);
                    }
                    zz[ch * m + IDX(n, i, j, k)] = s;
                }
    for (int k = kmin(d); k <= kmax(d, n); ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i) {
                double s = 0.0;
                for (int ch = 0; ch < ORC_HID; ++ch)
                    for (int t = 0; t < T; ++t) {
                        int a, b, c;
                        tap_off(d, t, &a, &b, &c);
                        double zv = val(zz + ch * m, d, n, i + a, j + b, k + c);
                        s = s + (double)W2[ch * T + t] * (zv > 0.0 ? zv : 0.0);
                    }
                y[IDX(n, i, j, k)] = s;
            }
    if (!z) free(zz);
}

/* Backward of orc_conv_fwd for an upstream gradient gy (interior nodes):
 * gx = dL/dx, dW1, dW2 (accumulated, arrays of ORC_HID*taps doubles). */
void orc_conv_bwd(int d, int n, const float* W1, const float* W2, const double* x,
                  const double* gy, double* gx, double* dW1, double* dW2)
{
    int64_t m = nodes(d, n);
    int T = ntaps(d);
    double* z = (double*)malloc(sizeof(double) * m * ORC_HID);
    double* y = (double*)malloc(sizeof(double) * m);
    double* gz = (double*)calloc(m * ORC_HID, sizeof(double));
    orc_conv_fwd(d, n, W1, W2, x, z, y);
    /* dW2[ch][t] = sum_p gy(p) relu(z_ch(p + o_t));  gh_ch(q) = sum_t W2[ch][t] gy(q - o_t) */
    for (int ch = 0; ch < ORC_HID; ++ch)
        for (int t = 0; t < T; ++t) {
            int a, b, c;
            tap_off(d, t, &a, &b, &c);
            double s = 0.0;
            for (int k = kmin(d); k <= kmax(d, n); ++k)
                for (int j = 1; j < n; ++j)
                    for (int i = 1; i < n; ++i) {
                        double zv = val(z + ch * m, d, n, i + a, j + b, k + c);
                        s = s + gy[IDX(n, i, j, k)] * (zv > 0.0 ? zv : 0.0);
                    }
            dW2[ch * T + t] += s;
        }
    for (int ch = 0; ch < ORC_HID; ++ch)
        for (int k = kmin(d); k <= kmax(d, n); ++k)
            for (int j = 1; j < n; ++j)
                for (int i = 1; i < n; ++i) {
                    double s = 0.0;
                    for (int t = 0; t < T; ++t) {
                        int a, b, c;
                        tap_off(d, t, &a, &b, &c);
                        s = s + (double)W2[ch * T + t] * val(gy, d, n, i - a, j - b, k - c);
                    }
                    int64_t p = IDX(n, i, j, k);
                    gz[ch * m + p] = z[ch * m + p] > 0.0 ? s : 0.0;
                }
    /* dW1[ch][t] = sum_p gz_ch(p) x(p + o_t);  gx(q) = sum_ch sum_t W1[ch][t] gz_ch(q - o_t) */
    for (int ch = 0; ch < ORC_HID; ++ch)
        for (int t = 0; t < T; ++t) {
            int a, b, c;
            tap_off(d, t, &a, &b, &c);
            double s = 0.0;
            for (int k = kmin(d); k <= kmax(d, n); ++k)
                for (int j = 1; j < n; ++j)
                    for (int i = 1; i < n; ++i)
                        s = s + gz[ch * m + IDX(n, i, j, k)] * val(x, d, n, i + a, j + b, k + c);
            dW1[ch * T + t] += s;
        }
    memset(gx, 0, sizeof(double) * m);
    for (int k = kmin(d); k <= kmax(d, n); ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i) {
                double s = 0.0;
                for (int ch = 0; ch < ORC_HID; ++ch)
                    for (int t = 0; t < T; ++t) {
                        int a, b, c;
                        tap_off(d, t, &a, &b, &c);
                        s = s + (double)W1[ch * T + t] * val(gz + ch * m, d, n, i - a, j - b, k - c);
                    }
                gx[IDX(n, i, j, k)] = s;
            }
    free(z);
    free(y);
    free(gz);
}

/* One learned smoothing step in error form: e <- e - N(A'e/(2d)). */
void orc_learned_smooth_error(int d, int n, const float* W1, const float* W2, double* e)
{
    int64_t m = nodes(d, n);
    double* s = (double*)malloc(sizeof(double) * m);
    double* y = (double*)malloc(sizeof(double) * m);
    orc_apply_stencil(d, n, e, s);
    for (int64_t p = 0; p < m; ++p) s[p] = s[p] / (2.0 * d);
    orc_conv_fwd(d, n, W1, W2, s, NULL, y);
    for (int64_t p = 0; p < m; ++p) e[p] = e[p] - y[p];
    free(s);
    free(y);
}

/* Coarse-grid correction in error form with the coarse system solved by
 * `cycles` red-black V(2,2) cycles from zero: e <- e - P A_c'^{-1} 4 FW(A'e). */
void orc_cgc_error(int d, int n, double* e, int cycles)
{
    int nc = n / 2;
    int64_t m = nodes(d, n), mc = nodes(d, nc);
    double* r = (double*)malloc(sizeof(double) * m);
    double* bc = (double*)malloc(sizeof(double) * mc);
    double* uc = (double*)calloc(mc, sizeof(double));
    orc_apply_stencil(d, n, e, r);
    orc_restrict_fw(d, n, r, bc);
    orc_cfg c = {d, nc, 0, ORC_RBGS, 0.8, 2, 2, 1};
    int L = 0;
    while ((2 << L) <= nc) ++L;
    c.levels = L;
    for (int k = 0; k < cycles; ++k) orc_vcycle(&c, bc, uc);
    double* pu = (double*)calloc(m, sizeof(double));
    orc_prolong_add(d, nc, uc, pu);
    for (int64_t p = 0; p < m; ++p) e[p] = e[p] - pu[p];
    free(r);
    free(bc);
    free(uc);
    free(pu);
}

/* Two-grid contraction loss ||S(CG(S(e0)))||^2 / ||e0||^2. */
double orc_learned_loss(int d, int n, const float* W1, const float* W2, const double* e0,
                        int coarse_cycles)
{
    int64_t m = nodes(d, n);
    double* e = (double*)malloc(sizeof(double) * m);
    memcpy(e, e0, sizeof(double) * m);
    orc_learned_smooth_error(d, n, W1, W2, e);
    orc_cgc_error(d, n, e, coarse_cycles);
    orc_learned_smooth_error(d, n, W1, W2, e);
    double num = orc_norm2(d, n, e), den = orc_norm2(d, n, e0);
    free(e);
    return (num * num) / (den * den);
}

/* Round to float (nearest) and then to BF16 (nearest, ties to even). */
static double bf16(double v)
{
    float f = (float)v;
    uint32_t b;
    memcpy(&b, &f, 4);
    b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &b, 4);
    return (double)f;
}

/* The network with BF16 operands: x and relu(z) rounded to BF16 before each
 * convolution (the weights are given BF16-representable), exact sums. */
void orc_conv_fwd_bf16(int d, int n, const float* W1, const float* W2, const double* x,
                       double* y)
{
    int64_t m = nodes(d, n);
    int T = ntaps(d);
    double* xr = (double*)malloc(sizeof(double) * m);
    double* z = (double*)calloc(m * ORC_HID, sizeof(double));
    for (int64_t p = 0; p < m; ++p) xr[p] = bf16(x[p]);
    for (int ch = 0; ch < ORC_HID; ++ch)
        for (int k = kmin(d); k <= kmax(d, n); ++k)
            for (int j = 1; j < n; ++j)
                for (int i = 1; i < n; ++i) {
                    double s = 0.0;
                    for (int t = 0; t < T; ++t) {
                        int a, b, c;
                        tap_off(d, t, &a, &b, &c);
                        s = s + (double)W1[ch * T + t] * val(xr, d, n, i + a, j + b, k + c);
                    }
                    z[ch * m + IDX(n, i, j, k)] = bf16(s > 0.0 ? s : 0.0);
                }
    memset(y, 0, sizeof(double) * m);
    for (int k = kmin(d); k <= kmax(d, n); ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i) {
                double s = 0.0;
                for (int ch = 0; ch < ORC_HID; ++ch)
                    for (int t = 0; t < T; ++t) {
                        int a, b, c;
                        tap_off(d, t, &a, &b, &c);
                        s = s + (double)W2[ch * T + t] * val(z + ch * m, d, n, i + a, j + b, k + c);
                    }
                y[IDX(n, i, j, k)] = s;
            }
    free(xr);
    free(z);
}

/* One learned smoothing step on a level: u <- u + N((b - A'u)/(2d)). */
static int g_bf16_act = 0;
void orc_set_bf16_activations(int on) { g_bf16_act = on; }

void orc_learned_relax(int d, int n, const float* W1, const float* W2, const double* b,
                       double* u)
{
    int64_t m = nodes(d, n);
    double* r = (double*)malloc(sizeof(double) * m);
    double* y = (double*)malloc(sizeof(double) * m);
    orc_residual(d, n, b, u, r);
    for (int64_t p = 0; p < m; ++p) r[p] = r[p] / (2.0 * d);
    if (g_bf16_act)
        orc_conv_fwd_bf16(d, n, W1, W2, r, y);
    else
        orc_conv_fwd(d, n, W1, W2, r, NULL, y);
    for (int64_t p = 0; p < m; ++p) u[p] = u[p] + y[p];
    free(r);
    free(y);
}

/* Algorithm 1 with the learned smoother on the levels whose weights are
 * given: W[l] points at 2 x 8 x taps floats (W1 then W2) or is NULL, in which
 * case level l relaxes with red-black GS.  Sweeps nu1 / nu2 per level. */
int orc_vcycle_learned(const orc_cfg* c, const float* const* W, const double* b0, double* u0)
{
    int d = c->d, L = c->levels, T = ntaps(d);
    if (L < 2 || (c->n >> (L - 1)) != 2) return -1;
    double** b = (double**)calloc(L, sizeof(double*));
    double** u = (double**)calloc(L, sizeof(double*));
    double* r = (double*)malloc(sizeof(double) * nodes(d, c->n));
    b[0] = (double*)b0;
    u[0] = u0;
    for (int l = 1; l < L; ++l) {
        b[l] = (double*)calloc(nodes(d, c->n >> l), sizeof(double));
        u[l] = (double*)calloc(nodes(d, c->n >> l), sizeof(double));
    }
#define ORC_RELAX(l, sweeps)                                                         \
    for (int s_ = 0; s_ < (sweeps); ++s_) {                                          \
        if (W[l])                                                                    \
            orc_learned_relax(d, c->n >> (l), W[l], W[l] + ORC_HID * T, b[l], u[l]); \
        else                                                                         \
            orc_rbgs(d, c->n >> (l), b[l], u[l], 1);                                 \
    }
    for (int l = 0; l + 1 < L; ++l) {
        int nl = c->n >> l;
        ORC_RELAX(l, c->nu1);
        orc_residual(d, nl, b[l], u[l], r);
        orc_restrict_fw(d, nl, r, b[l + 1]);
        memset(u[l + 1], 0, sizeof(double) * nodes(d, nl / 2));
    }
    orc_coarse_solve(d, 2, b[L - 1], u[L - 1], 1);
    for (int l = L - 2; l >= 0; --l) {
        orc_prolong_add(d, (c->n >> l) / 2, u[l + 1], u[l]);
        ORC_RELAX(l, c->nu2);
    }
#undef ORC_RELAX
    for (int l = 1; l < L; ++l) {
        free(b[l]);
        free(u[l]);
    }
    free(b);
    free(u);
    free(r);
    return 0;
}

/* Full multigrid FMG-V (Algorithm 2): the right-hand side restricted to every
 * level, b_{l+1} = 4 FW(b_l) (the scaling of the residual restriction); the
 * coarsest level solved; then for l = L-2 .. 0: u_l = P u_{l+1} (interpolation
 * of the coarse solution) followed by one V-cycle (Algorithm 1) on levels
 * l .. L-1 with right-hand side b_l.  The initial u0 is ignored.  Returns 0
 * or -1. */
int orc_fmg(const orc_cfg* c, const double* b0, double* u0)
{
    int d = c->d, L = c->levels;
    if (L < 1 || (c->n >> (L - 1)) < 2) return -1;
    double** b = (double**)calloc(L, sizeof(double*));
    double** u = (double**)calloc(L, sizeof(double*));
    b[0] = (double*)b0;
    u[0] = u0;
    for (int l = 1; l < L; ++l) {
        b[l] = (double*)calloc(nodes(d, c->n >> l), sizeof(double));
        u[l] = (double*)calloc(nodes(d, c->n >> l), sizeof(double));
    }
    for (int l = 0; l + 1 < L; ++l) restrict_(c, c->n >> l, b[l], b[l + 1]);
    if (L == 1) {
        memset(u0, 0, sizeof(double) * nodes(d, c->n));
        orc_vcycle(c, b0, u0);
    } else {
        orc_coarse_solve(d, c->n >> (L - 1), b[L - 1], u[L - 1], c->coarse_sweeps);
        for (int l = L - 2; l >= 0; --l) {
            int nl = c->n >> l;
            memset(u[l], 0, sizeof(double) * nodes(d, nl));
            prolong_(c, nl / 2, u[l + 1], u[l]);
            orc_cfg cl = *c;
            cl.n = nl;
            cl.levels = L - l;
            orc_vcycle(&cl, b[l], u[l]);
        }
    }
    for (int l = 1; l < L; ++l) {
        free(b[l]);
        free(u[l]);
    }
    free(b);
    free(u);
    return 0;
}
