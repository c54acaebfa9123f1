// Batched form: many independent Poisson solves of uneven sizes (2D and 3D
// mixed) advanced together, FP32 or BF16-storage cycles inside FP64
// iterative refinement, one persistent kernel per level index over the whole
// batch.
//
// Work items are chunks of one solve's level grid (interior nodes, coarse
// interior nodes or coarse cells, by operation).  Levels are aligned at the
// coarsest 3^d grid: level step g processes, for every solve with at least
// g+1 grids, its level L_s - 1 - g.  The small solves' fine levels thus share
// launches with the large solves' coarse levels.  Each kernel's CTAs stride
// over the items of its launch; items of converged solves are skipped
// (per-solve active flags, written only by the step's final kernel).
// One refinement step of the whole batch is captured into one CUDA graph;
// the host reads one counter (solves still active) per step.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gmg_internal.cuh"
#include "level_kernels.cuh"
#include "timing.cuh"

namespace gmg {
namespace batch {

using lk::fastdiv;
using lk::FastDiv;
using lk::fastdiv_make;

struct BLevel {
    int d, n;
    int64_t u0, u1, q, r;  // element offsets into the inner pool (-1: none)
    int64_t sy, sz;        // inner pool row / plane pitch
    int lgG;               // log2 of the 16-byte groups per row the vector kernels take
    FastDiv rows;          // division by n - 1 (interior nodes per row)
};
struct BSolve {
    int d, n, levels, lev0;  // lev0: index of level 0 in the level table
    int64_t q64;             // offset of the FP64 scaled right-hand side
    int item0, item1;        // its items in the level-0 item list
    const double* f;
    double* u;
};
struct Item {
    int solve, level;
    int64_t start;
    int count;
};

using lk::Num;

// Node (i, j, k) of interior index idx (x fastest over the (n-1)^d interior
// nodes of level L) and its offset in the level's inner-pool array; no
// integer division (interior counts stay below 2^32).
__device__ inline int64_t node_of(const BLevel& L, uint32_t idx, int& i, int& j, int& k) {
    const uint32_t m = L.rows.d;
    const uint32_t t = fastdiv(idx, L.rows);
    i = (int)(idx - t * m) + 1;
    if (L.d == 3) {
        const uint32_t kk = fastdiv(t, L.rows);
        j = (int)(t - kk * m) + 1;
        k = (int)kk + 1;
    } else {
        j = (int)t + 1;
        k = 0;
    }
    return (int64_t)k * L.sz + (int64_t)j * L.sy + i;
}
// offset of node (i, j, k) in the solve's dense FP64 arrays
__device__ inline int64_t dense_of(const BLevel& L, int i, int j, int k) {
    return ((int64_t)k * (L.n + 1) + j) * (L.n + 1) + i;
}
__device__ inline int64_t node_of(const BLevel& L, uint32_t idx) {
    int i, j, k;
    return node_of(L, idx, i, j, k);
}

__device__ inline int64_t off_u(const BLevel& L, int which) { return which ? L.u1 : L.u0; }

// V = 16 bytes of inner-pool values (4 FP32, 8 BF16) as floats, and back
template <typename T>
__device__ inline void ldv(const T* p, float* v);
template <>
__device__ inline void ldv<float>(const float* p, float* v) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}
template <>
__device__ inline void ldv<__nv_bfloat16>(const __nv_bfloat16* p, float* v) {
    const uint4 a = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&w[h]);
        v[2 * h] = __low2float(b);
        v[2 * h + 1] = __high2float(b);
    }
}
template <typename T>
__device__ inline void stv(T* p, const float* v);
template <>
__device__ inline void stv<float>(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ inline void stv<__nv_bfloat16>(__nv_bfloat16* p, const float* v) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h)
        *reinterpret_cast<__nv_bfloat162*>(&w[h]) = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

// Vector items: index gid over (interior row) x (16-byte group of the row),
// 2^lgG groups per row (x = V g .. V g + V - 1 covers 0 .. n - 1); the group's
// offset in the level's inner-pool array and its first x.
template <int V>
__device__ inline int64_t group_of(const BLevel& L, uint32_t gid, int& x0, int& j, int& k) {
    const uint32_t row = gid >> L.lgG;
    x0 = V * (int)(gid & ((1u << L.lgG) - 1u));
    if (L.d == 3) {
        const uint32_t m = L.rows.d;
        const uint32_t kk = fastdiv(row, L.rows);
        j = (int)(row - kk * m) + 1;
        k = (int)kk + 1;
    } else {
        j = (int)row + 1;
        k = 0;
    }
    return (int64_t)k * L.sz + (int64_t)j * L.sy + x0;
}

// Smoothing sweep over the items' groups: weighted Jacobi (src -> dst) or one
// colour of red-black Gauss-Seidel (in place, src == dst; the group's other
// nodes are written back unchanged, and no other thread writes them).  Per
// group: one 16-byte load each of the row, its y and z neighbour rows and q,
// the two x neighbours beyond the group as single loads, one 16-byte store;
// nodes outside 1..n-1 are written as 0 (Jacobi) or left unchanged.  The
// neighbour sum is ((x- + x+) + y- + y+) + z- + z+ in this order.  pool_in and pool_out are the
// same pool: what a launch reads through pool_in is never written during the
// launch (the Jacobi source, q; in red-black the other colour).
template <typename T>
__global__ void __launch_bounds__(256) k_smooth(const Item* __restrict__ items, int nitems,
                                                const BSolve* __restrict__ sv,
                                                const BLevel* __restrict__ lv,
                                                const T* __restrict__ pool_in,
                                                T* __restrict__ pool_out,
                                                const int* __restrict__ active, int src, int dst,
                                                int color, float omega2, float omega3) {
    constexpr int V = 16 / (int)sizeof(T);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const Item w = items[it];
        if (!active[w.solve]) continue;
        const BLevel L = lv[sv[w.solve].lev0 + w.level];
        const bool three = L.d == 3;
        const float c = three ? 1.f / 6.f : 0.25f;
        const float omega = three ? omega3 : omega2;
        const T* u = pool_in + off_u(L, src);
        T* uo = pool_out + off_u(L, dst);
        const T* q = pool_in + L.q;
        for (int t = threadIdx.x; t < w.count; t += blockDim.x) {
            int x0, j, k;
            const int64_t p = group_of<V>(L, (uint32_t)(w.start + t), x0, j, k);
            float x[V], ym[V], yp[V], zm[V], zp[V], qv[V], out[V];
            ldv(u + p, x);
            const float xl = Num<T>::ld(u[p - 1]), xr = Num<T>::ld(u[p + V]);
            ldv(u + p - L.sy, ym);
            ldv(u + p + L.sy, yp);
            if (three) {
                ldv(u + p - L.sz, zm);
                ldv(u + p + L.sz, zp);
            }
            ldv(q + p, qv);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float s = (v > 0 ? x[v - 1] : xl) + (v < V - 1 ? x[v + 1] : xr);
                s += ym[v];
                s += yp[v];
                if (three) {
                    s += zm[v];
                    s += zp[v];
                }
                const float g = fmaf(c, s, qv[v]);
                const int xi = x0 + v;
                const bool in = xi >= 1 && xi <= L.n - 1;
                if (color >= 0)
                    out[v] = in && ((xi + j + k) & 1) == color ? g : x[v];
                else
                    out[v] = in ? fmaf(omega, g - x[v], x[v]) : 0.f;
            }
            stv(uo + p, out);
        }
    }
}

// r = sigma over the items' groups (0 outside the interior); pool_in /
// pool_out: the same pool, as in k_smooth (u and q are not written here)
template <typename T>
__global__ void __launch_bounds__(256) k_residual(const Item* __restrict__ items, int nitems,
                                                  const BSolve* __restrict__ sv,
                                                  const BLevel* __restrict__ lv,
                                                  const T* __restrict__ pool_in,
                                                  T* __restrict__ pool_out,
                                                  const int* __restrict__ active, int src) {
    constexpr int V = 16 / (int)sizeof(T);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const Item w = items[it];
        if (!active[w.solve]) continue;
        const BLevel L = lv[sv[w.solve].lev0 + w.level];
        const bool three = L.d == 3;
        const float c = three ? 1.f / 6.f : 0.25f;
        const T* u = pool_in + off_u(L, src);
        const T* q = pool_in + L.q;
        T* r = pool_out + L.r;
        for (int t = threadIdx.x; t < w.count; t += blockDim.x) {
            int x0, j, k;
            const int64_t p = group_of<V>(L, (uint32_t)(w.start + t), x0, j, k);
            float x[V], ym[V], yp[V], zm[V], zp[V], qv[V], out[V];
            ldv(u + p, x);
            const float xl = Num<T>::ld(u[p - 1]), xr = Num<T>::ld(u[p + V]);
            ldv(u + p - L.sy, ym);
            ldv(u + p + L.sy, yp);
            if (three) {
                ldv(u + p - L.sz, zm);
                ldv(u + p + L.sz, zp);
            }
            ldv(q + p, qv);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float s = (v > 0 ? x[v - 1] : xl) + (v < V - 1 ? x[v + 1] : xr);
                s += ym[v];
                s += yp[v];
                if (three) {
                    s += zm[v];
                    s += zp[v];
                }
                const int xi = x0 + v;
                out[v] = xi >= 1 && xi <= L.n - 1 ? fmaf(c, s, qv[v]) - x[v] : 0.f;
            }
            stv(r + p, out);
        }
    }
}

// q_c = 4 FW(r) on the items' coarse interior nodes (item level = fine
// level); u_c = 0, or u_c = q_c on a one-unknown coarsest grid.  pool_in /
// pool_out: the same pool, as in k_smooth (r is not written here).
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(const Item* __restrict__ items, int nitems,
                                                  const BSolve* __restrict__ sv,
                                                  const BLevel* __restrict__ lv,
                                                  const T* __restrict__ pool_in,
                                                  T* __restrict__ pool_out,
                                                  const int* __restrict__ active) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const Item w = items[it];
        if (!active[w.solve]) continue;
        const BLevel F = lv[sv[w.solve].lev0 + w.level];
        const BLevel C = lv[sv[w.solve].lev0 + w.level + 1];
        const bool three = F.d == 3;
        const int64_t sy = F.sy, sz = three ? F.sz : 0;
        const T* r = pool_in + F.r;
        for (int t = threadIdx.x; t < w.count; t += blockDim.x) {
            int I, J, K;
            const int64_t P = node_of(C, (uint32_t)(w.start + t), I, J, K);
            const int64_t p = (2 * K) * sz + (2 * J) * sy + 2 * I;
            float v = 0.f;
            for (int dz = three ? -1 : 0; dz <= (three ? 1 : 0); ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        // 4 x [1/4 1/2 1/4]^d: 2^(1 - zeros... ) as a power of two
                        const int nz = (dx == 0) + (dy == 0) + (three ? (dz == 0) : 0);
                        const int odd = (three ? 3 : 2) - nz;
                        const float wgt = (three ? 0.5f : 1.f) * ldexpf(1.f, -odd);
                        v = fmaf(wgt, Num<T>::ld(r[p + dz * sz + dy * sy + dx]), v);
                    }
            T* qc = pool_out + C.q;
            T* uc = pool_out + C.u0;
            qc[P] = Num<T>::st(v);
            uc[P] = C.n == 2 ? Num<T>::st(v) : Num<T>::st(0.f);
        }
    }
}

// u_fine += P u_coarse, one thread per coarse cell (item level = fine level):
// the cell's 2^d corners are loaded once, the corrections of its 2^d fine
// nodes formed from them (weight 2^-(number of odd offsets) times the sum of
// the corners the fine node lies between), then every fine operand is
// loaded before the first store.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(const Item* __restrict__ items, int nitems,
                                                 const BSolve* __restrict__ sv,
                                                 const BLevel* __restrict__ lv, T* pool,
                                                 const int* __restrict__ active, int fcur,
                                                 int ccur) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const Item w = items[it];
        if (!active[w.solve]) continue;
        const BLevel F = lv[sv[w.solve].lev0 + w.level];
        const BLevel C = lv[sv[w.solve].lev0 + w.level + 1];
        const bool three = F.d == 3;
        const int nc = C.n;
        const int64_t sy = F.sy, sz = three ? F.sz : 0;
        const int64_t cy = C.sy, cz = three ? C.sz : 0;
        const T* uc = pool + off_u(C, ccur);
        T* u = pool + off_u(F, fcur);
        const int lg = __ffs(nc) - 1;  // nc is a power of two
        for (int t = threadIdx.x; t < w.count; t += blockDim.x) {
            const uint32_t cell = (uint32_t)(w.start + t);
            const int I = (int)(cell & (nc - 1)), J = (int)((cell >> lg) & (nc - 1)),
                      K = three ? (int)(cell >> (2 * lg)) : 0;
            const int64_t P = K * cz + J * cy + I;
            const int64_t p = (2 * K) * sz + (2 * J) * sy + 2 * I;
            // corners c[a + 2b + 4c'] = u_c(I + a, J + b, K + c')
            float cv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e)
                cv[e] = (three || e < 4)
                            ? Num<T>::ld(uc[P + ((e >> 2) & 1) * cz + ((e >> 1) & 1) * cy + (e & 1)])
                            : 0.f;
            // the fine node (2I + a, 2J + b, 2K + c') gets 2^-(a+b+c') times the
            // sum of the corners (I + a', J + b', K + c'') with a' <= a, ...
            float corr[8], fv[8];
            bool on[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int a = e & 1, b = (e >> 1) & 1, cc = (e >> 2) & 1;
                on[e] = (three || cc == 0) && !(a == 0 && I == 0) && !(b == 0 && J == 0) &&
                        !(three && cc == 0 && K == 0);
                float sum = 0.f;
#pragma unroll
                for (int g = 0; g < 8; ++g)
                    if ((g & ~e) == 0) sum += cv[g];
                corr[e] = ldexpf(sum, -(a + b + cc));
            }
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (on[e]) fv[e] = Num<T>::ld(u[p + ((e >> 2) & 1) * sz + ((e >> 1) & 1) * sy + (e & 1)]);
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (on[e])
                    u[p + ((e >> 2) & 1) * sz + ((e >> 1) & 1) * sy + (e & 1)] =
                        Num<T>::st(fv[e] + corr[e]);
        }
    }
}

// e = 0 on the items' interior nodes (level 0)
template <typename T>
__global__ void __launch_bounds__(256) k_zero(const Item* __restrict__ items, int nitems,
                                              const BSolve* __restrict__ sv,
                                              const BLevel* __restrict__ lv, T* pool,
                                              const int* __restrict__ active) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const Item w = items[it];
        if (!active[w.solve]) continue;
        const BLevel L = lv[sv[w.solve].lev0];
        T* e = pool + L.u0;
        for (int t = threadIdx.x; t < w.count; t += blockDim.x)
            e[node_of(L, (uint32_t)(w.start + t))] = Num<T>::st(0.f);
    }
}

// u += e in FP64 on the items' interior nodes (level 0)
template <typename T>
__global__ void __launch_bounds__(256) k_update(const Item* __restrict__ items, int nitems,
                                                const BSolve* __restrict__ sv,
                                                const BLevel* __restrict__ lv, const T* pool,
                                                const int* __restrict__ active) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const Item w = items[it];
        if (!active[w.solve]) continue;
        const BSolve S = sv[w.solve];
        const BLevel L = lv[S.lev0];
        const T* e = pool + L.u0;
        for (int t = threadIdx.x; t < w.count; t += blockDim.x) {
            int i, j, k;
            const int64_t p = node_of(L, (uint32_t)(w.start + t), i, j, k);
            S.u[dense_of(L, i, j, k)] += (double)Num<T>::ld(e[p]);
        }
    }
}

// FP64 scaled right-hand side q64 = h^2 f / (2d) on interior nodes; zero
// u's boundary is the caller's layout contract, enforced here on faces
template <typename T>
__global__ void __launch_bounds__(256) k_prepare(const Item* __restrict__ items, int nitems,
                                                 const BSolve* __restrict__ sv,
                                                 const BLevel* __restrict__ lv, double* pool64) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const Item w = items[it];
        const BSolve S = sv[w.solve];
        const BLevel L = lv[S.lev0];
        const double h = 1.0 / S.n;
        const double scale = h * h / (2.0 * S.d);
        double* q = pool64 + S.q64;
        for (int t = threadIdx.x; t < w.count; t += blockDim.x) {
            int i, j, k;
            node_of(L, (uint32_t)(w.start + t), i, j, k);
            const int64_t p = dense_of(L, i, j, k);
            q[p] = scale * S.f[p];
        }
    }
}

__global__ void k_fill_int(int* a, int count, int v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        a[i] = v;
}

__global__ void k_zero_boundary(const BSolve* __restrict__ sv, int count) {
    for (int s = blockIdx.x; s < count; s += gridDim.x) {
        const BSolve S = sv[s];
        const int64_t m = S.n + 1;
        const int64_t nodes = S.d == 3 ? m * m * m : m * m;
        for (int64_t p = threadIdx.x; p < nodes; p += blockDim.x) {
            const int i = (int)(p % m), j = (int)((p / m) % m), k = S.d == 3 ? (int)(p / (m * m)) : 1;
            if (i == 0 || i == S.n || j == 0 || j == S.n || k == 0 || k == (S.d == 3 ? S.n : 2))
                S.u[p] = 0.0;
        }
    }
}

// sigma = q64 + c sum(u) - u in FP64 on the items' interior nodes, stored to
// the inner right-hand side; one partial sum of sigma^2 per item
template <typename T>
__global__ void __launch_bounds__(256) k_outer(const Item* __restrict__ items, int nitems,
                                               const BSolve* __restrict__ sv,
                                               const BLevel* __restrict__ lv, T* pool,
                                               const double* __restrict__ pool64,
                                               const int* __restrict__ active,
                                               double* __restrict__ partial) {
    __shared__ double warp_sums[8];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const Item w = items[it];
        if (!active[w.solve]) continue;
        const BSolve S = sv[w.solve];
        const BLevel L = lv[S.lev0];
        const bool three = L.d == 3;
        const double c = three ? 1.0 / 6.0 : 0.25;
        const int64_t sy = L.n + 1, sz = three ? sy * sy : 0;
        const double* u = S.u;
        const double* q = pool64 + S.q64;
        T* qin = pool + L.q;
        double acc = 0.0;
        for (int t = threadIdx.x; t < w.count; t += blockDim.x) {
            int i, j, k;
            const int64_t pin = node_of(L, (uint32_t)(w.start + t), i, j, k);
            const int64_t p = dense_of(L, i, j, k);
            double s = u[p - 1] + u[p + 1];
            s += u[p - sy];
            s += u[p + sy];
            if (three) {
                s += u[p - sz];
                s += u[p + sz];
            }
            const double sig = fma(c, s, q[p]) - u[p];
            qin[pin] = Num<T>::st((float)sig);
            acc = fma(sig, sig, acc);
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int k = 0; k < (int)(blockDim.x / 32); ++k) s += warp_sums[k];
            partial[it] = s;
        }
        __syncthreads();
    }
}

// per solve: sum its partials in order; start (first != 0): res0; otherwise
// count the step, record the relative residual and retire converged solves
__global__ void __launch_bounds__(1024) k_finalize(const BSolve* __restrict__ sv, int count,
                                                   const double* __restrict__ partial,
                                                   double* res0_2, int* active, int* iters,
                                                   double* relres, double rtol2, int maxit,
                                                   int first, int* num_active) {
    __shared__ int warp_cnt[32];
    int cnt = 0;
    for (int s = threadIdx.x; s < count; s += blockDim.x) {
        const BSolve S = sv[s];
        if (first || active[s]) {
            double sum = 0.0;
            for (int i = S.item0; i < S.item1; ++i) sum += partial[i];
            if (first) {
                res0_2[s] = sum;
                iters[s] = 0;
                relres[s] = sum > 0.0 ? 1.0 : 0.0;
                active[s] = (sum > 0.0 && maxit > 0) ? 1 : 0;
            } else {
                iters[s] += 1;
                relres[s] = sqrt(sum / res0_2[s]);
                if (!(sum > rtol2 * res0_2[s]) || iters[s] >= maxit) active[s] = 0;
            }
        }
        cnt += active[s];
    }
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    if ((threadIdx.x & 31) == 0) warp_cnt[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += warp_cnt[w];
        *num_active = t;
    }
}

}  // namespace batch
}  // namespace gmg

using namespace gmg;
using namespace gmg::batch;

namespace {

enum Op { OP_FINE, OP_COARSE, OP_CELLS, OP_COUNT };

struct Range {
    int off = 0, count = 0;
};

}  // namespace

struct gmg_batch_s {
    gmg_config cfg{};
    int count = 0, chunk = 1024, ctas = 608, device = 0, G = 0, elem = 4;
    cudaStream_t user_stream = nullptr, stream = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<BSolve> hs;
    std::vector<BLevel> hl;
    std::vector<Item> items;
    std::vector<Range> fine, coarse, cells;  // per level step g
    Range level0;                            // level-0 interior items (all solves)
    BSolve* ds = nullptr;
    BLevel* dl = nullptr;
    Item* di = nullptr;
    void* pool = nullptr;
    double* pool64 = nullptr;
    double* partial = nullptr;
    double* res0_2 = nullptr;
    double* relres = nullptr;
    int* active = nullptr;
    int* iters = nullptr;
    int* num_active = nullptr;
    int* h_active = nullptr;  // pinned
    cudaGraphExec_t graph = nullptr;
    double graph_rtol2 = -1.0;  // the stopping tolerance baked into the graph
    KernelTimer timer;
};

namespace {

template <typename T>
struct PrecName;
template <>
struct PrecName<float> {
    static constexpr const char* s = "_f32";
};
template <>
struct PrecName<__nv_bfloat16> {
    static constexpr const char* s = "_bf16";
};

template <typename T, class F>
void launch_op(gmg_batch b, const char* name, int g, const Range& r, double bytes_per_item_node,
               double ops_per_node, int64_t nodes, F&& body) {
    if (r.count == 0) return;
    const int grid = std::min(r.count, b->ctas);
    b->timer.run(b->stream, std::string(name) + PrecName<T>::s, g, ops_per_node * nodes,
                 bytes_per_item_node * nodes, 1, [&] { body(grid, b->di + r.off, r.count); });
}

int64_t range_nodes(gmg_batch b, const Range& r) {
    int64_t s = 0;
    for (int i = r.off; i < r.off + r.count; ++i) s += b->items[i].count;
    return s;
}

// One refinement step of the whole batch (captured): e = 0, k inner
// cycles, u += e, new sigma and per-solve norms, retire converged solves.
template <typename T>
gmg_status enqueue_step(gmg_batch b, double rtol2) {
    const gmg_config& c = b->cfg;
    T* pool = static_cast<T*>(b->pool);
    const double w = sizeof(T);
    const bool rbgs = c.smoother == GMG_RBGS;
    // weighted-Jacobi weight per dimension: the configured one, or with
    // omega = 0 the defaults 4/5 (2D) and 6/7 (3D)
    const float omega2 = c.omega > 0.0 ? (float)c.omega : 0.8f;
    const float omega3 = c.omega > 0.0 ? (float)c.omega : (float)(6.0 / 7.0);
    b->timer.begin_capture();
    const int64_t n0 = range_nodes(b, b->level0);
    launch_op<T>(b, "b_zero", 0, b->level0, w, 0, n0, [&](int grid, const Item* it, int ni) {
        k_zero<T><<<grid, 256, 0, b->stream>>>(it, ni, b->ds, b->dl, pool, b->active);
    });
    std::vector<int> cur(b->G + 1, 0);  // which u buffer holds each level step's iterate
    auto relax = [&](int g, int sweeps) {
        const Range& r = b->fine[g];
        const int64_t nn = range_nodes(b, r) * (16 / b->elem);  // groups x V nodes
        for (int s = 0; s < sweeps; ++s) {
            if (rbgs) {
                for (int color = 0; color < 2; ++color)
                    launch_op<T>(b, "b_rb_half", g, r, 1.5 * w, 3.0, nn,
                                 [&](int grid, const Item* it, int ni) {
                                     k_smooth<T><<<grid, 256, 0, b->stream>>>(
                                         it, ni, b->ds, b->dl, pool, pool, b->active, cur[g],
                                         cur[g], color, omega2, omega3);
                                 });
            } else {
                launch_op<T>(b, "b_wj_sweep", g, r, 3 * w, 8.0, nn,
                             [&](int grid, const Item* it, int ni) {
                                 k_smooth<T><<<grid, 256, 0, b->stream>>>(
                                     it, ni, b->ds, b->dl, pool, pool, b->active, cur[g],
                                     cur[g] ^ 1, -1, omega2, omega3);
                             });
                cur[g] ^= 1;
            }
        }
    };
    for (int k = 0; k < c.inner_cycles; ++k) {
        std::fill(cur.begin(), cur.end(), 0);
        // down: level steps g = G..1 (fine levels of the deepest solves first)
        for (int g = b->G; g >= 1; --g) {
            relax(g, c.nu1);
            const int64_t nn = range_nodes(b, b->fine[g]) * (16 / b->elem);
            launch_op<T>(b, "b_residual", g, b->fine[g], 3 * w, 7.0, nn,
                         [&](int grid, const Item* it, int ni) {
                             k_residual<T><<<grid, 256, 0, b->stream>>>(
                                 it, ni, b->ds, b->dl, pool, pool, b->active, cur[g]);
                         });
            const int64_t nc = range_nodes(b, b->coarse[g]);
            launch_op<T>(b, "b_restrict", g, b->coarse[g], 10 * w, 27.0, nc,
                         [&](int grid, const Item* it, int ni) {
                             k_restrict<T><<<grid, 256, 0, b->stream>>>(it, ni, b->ds, b->dl,
                                                                        pool, pool, b->active);
                         });
            cur[g - 1] = 0;
        }
        // up: g = 1..G
        for (int g = 1; g <= b->G; ++g) {
            const int64_t ncell = range_nodes(b, b->cells[g]);
            const int fc = cur[g], cc = cur[g - 1];
            launch_op<T>(b, "b_prolong_add", g, b->cells[g], 17 * w, 20.0, ncell,
                         [&](int grid, const Item* it, int ni) {
                             k_prolong<T><<<grid, 256, 0, b->stream>>>(it, ni, b->ds, b->dl, pool,
                                                                       b->active, fc, cc);
                         });
            relax(g, c.nu2);
        }
        if (cur[b->G] != 0) {
            set_error("batched weighted Jacobi needs an even nu1 + nu2 on the finest levels");
            return GMG_ERR_UNSUPPORTED;
        }
    }
    launch_op<T>(b, "b_update", 0, b->level0, 16 + w, 1.0, n0,
                 [&](int grid, const Item* it, int ni) {
                     k_update<T><<<grid, 256, 0, b->stream>>>(it, ni, b->ds, b->dl, pool,
                                                              b->active);
                 });
    launch_op<T>(b, "b_outer_residual", 0, b->level0, 16 + w, 8.0, n0,
                 [&](int grid, const Item* it, int ni) {
                     k_outer<T><<<grid, 256, 0, b->stream>>>(it, ni, b->ds, b->dl, pool,
                                                             b->pool64, b->active, b->partial);
                 });
    b->timer.run(b->stream, "b_finalize", 0, 0, 0, 1, [&] {
        k_finalize<<<1, 1024, 0, b->stream>>>(b->ds, b->count, b->partial, b->res0_2, b->active,
                                              b->iters, b->relres, rtol2, c.maxit, 0,
                                              b->num_active);
    });
    GMG_CUDA_TRY(cudaMemcpyAsync(b->h_active, b->num_active, sizeof(int), cudaMemcpyDeviceToHost,
                                 b->stream));
    GMG_CUDA_TRY(cudaGetLastError());
    return GMG_OK;
}

template <typename T>
void enqueue_start(gmg_batch b) {
    T* pool = static_cast<T*>(b->pool);
    const int grid0 = std::min(b->level0.count, b->ctas);
    const Item* it0 = b->di + b->level0.off;
    k_zero_boundary<<<std::min(b->count, 1024), 256, 0, b->stream>>>(b->ds, b->count);
    k_prepare<T><<<grid0, 256, 0, b->stream>>>(it0, b->level0.count, b->ds, b->dl, b->pool64);
    // every solve counts as active for the initial residual
    k_fill_int<<<(b->count + 255) / 256, 256, 0, b->stream>>>(b->active, b->count, 1);
    k_outer<T><<<grid0, 256, 0, b->stream>>>(it0, b->level0.count, b->ds, b->dl, pool, b->pool64,
                                             b->active, b->partial);
    k_finalize<<<1, 1024, 0, b->stream>>>(b->ds, b->count, b->partial, b->res0_2, b->active,
                                          b->iters, b->relres, 0.0, b->cfg.maxit, 1,
                                          b->num_active);
    b->timer.launches += 5;
}

bool dev_ptr_ok(const void* p) {
    if (!p || ((uintptr_t)p) % 8) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

gmg_status gmg_batch_destroy(gmg_batch b) {
    if (!b) return GMG_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->timer.destroy();
    for (void* p : {(void*)b->ds, (void*)b->dl, (void*)b->di, b->pool, (void*)b->pool64,
                    (void*)b->partial, (void*)b->res0_2, (void*)b->relres, (void*)b->active,
                    (void*)b->iters, (void*)b->num_active})
        if (p) cudaFree(p);
    if (b->h_active) cudaFreeHost(b->h_active);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    if (prev >= 0) cudaSetDevice(prev);
    return GMG_OK;
}

gmg_status gmg_batch_create(int count, const int* d, const int* n, const gmg_config* common,
                            int chunk, int ctas, void* cuda_stream, gmg_batch* out) {
    if (!out || !common || !d || !n || count < 1 || count > (1 << 20)) {
        set_error("gmg_batch_create: bad arguments");
        return GMG_ERR_ARG;
    }
    *out = nullptr;
    if (common->precision != GMG_FP32_IR && common->precision != GMG_BF16_IR) {
        set_error("gmg_batch_create: precision must be GMG_FP32_IR or GMG_BF16_IR");
        return GMG_ERR_UNSUPPORTED;
    }
    if (common->smoother != GMG_WJACOBI && common->smoother != GMG_RBGS) {
        set_error("gmg_batch_create: smoother must be weighted Jacobi or red-black GS");
        return GMG_ERR_ARG;
    }
    if (common->transfer != GMG_TRANSFER_FW) {
        set_error("gmg_batch_create: the batch uses full-weighting transfers");
        return GMG_ERR_UNSUPPORTED;
    }
    if (common->smoother == GMG_WJACOBI && ((common->nu1 + common->nu2) % 2 != 0)) {
        set_error("gmg_batch_create: weighted Jacobi needs nu1 + nu2 even");
        return GMG_ERR_UNSUPPORTED;
    }
    if (common->nu1 < 0 || common->nu2 < 0 || common->nu1 > 16 || common->nu2 > 16 ||
        common->inner_cycles < 1 || common->inner_cycles > 64 || common->maxit < 0 ||
        !(common->omega >= 0.0 && common->omega < 2.0)) {
        set_error("gmg_batch_create: nu1, nu2, inner_cycles, maxit or omega out of range");
        return GMG_ERR_ARG;
    }
    if (chunk < 0 || chunk > (1 << 20) || ctas < 0 || ctas > (1 << 16)) {
        set_error("gmg_batch_create: chunk / ctas out of range");
        return GMG_ERR_ARG;
    }
    for (int s = 0; s < count; ++s) {
        const int nmax = d[s] == 2 ? 16384 : 1024;
        if ((d[s] != 2 && d[s] != 3) || n[s] < 2 || n[s] > nmax || (n[s] & (n[s] - 1))) {
            set_error("gmg_batch_create: solve " + std::to_string(s) +
                      ": d must be 2 or 3 and n a power of two within limits");
            return GMG_ERR_ARG;
        }
    }
    gmg_batch b = new gmg_batch_s();
    b->cfg = *common;
    b->count = count;
    b->chunk = chunk > 0 ? chunk : 1024;
    b->user_stream = (cudaStream_t)cuda_stream;
    b->elem = common->precision == GMG_FP32_IR ? 4 : 2;
    auto fail = [&](gmg_status st, const std::string& msg) {
        set_error("gmg_batch_create: " + msg);
        gmg_batch_destroy(b);
        return st;
    };
    if (cudaGetDevice(&b->device) != cudaSuccess) return fail(GMG_ERR_CUDA, "no device");
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    b->ctas = ctas > 0 ? ctas : 4 * sms;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess)
        return fail(GMG_ERR_CUDA, "stream/event creation failed");
    // layout: per solve, per level: u0 [u1] q [r] in the inner pool (256-byte
    // aligned regions); FP64 q64 per solve
    const int64_t align = 256 / b->elem;
    auto up = [&](int64_t v, int64_t a) { return (v + a - 1) / a * a; };
    int64_t poff = 0, off64 = 0;
    for (int s = 0; s < count; ++s) {
        BSolve S{};
        S.d = d[s];
        S.n = n[s];
        int L = 0;
        while ((2 << L) <= n[s]) ++L;  // log2(n) grids: n, n/2, ..., 2
        S.levels = L;
        S.lev0 = (int)b->hl.size();
        const int64_t m0 = n[s] + 1;
        S.q64 = off64;
        off64 = up(off64 + (d[s] == 3 ? m0 * m0 * m0 : m0 * m0), 32);
        for (int l = 0; l < L; ++l) {
            BLevel lv{};
            lv.d = d[s];
            lv.n = n[s] >> l;
            lv.rows = fastdiv_make((uint32_t)(lv.n - 1));
            // rows padded to a multiple of 8 elements (16 bytes in BF16, 32 in FP32)
            const int64_t m = lv.n + 1;
            lv.sy = up(m, 8);
            lv.sz = d[s] == 3 ? lv.sy * m : 0;
            const int V = 16 / b->elem;
            int lg = 0;
            while ((V << (lg + 1)) <= lv.n) ++lg;  // 2^lg groups of V cover x = 0 .. n-1
            lv.lgG = lg;
            const int64_t nodes = d[s] == 3 ? lv.sz * m : lv.sy * m;
            lv.u0 = poff;
            poff = up(poff + nodes, align);
            lv.u1 = -1;
            if (common->smoother == GMG_WJACOBI) {
                lv.u1 = poff;
                poff = up(poff + nodes, align);
            }
            lv.q = poff;
            poff = up(poff + nodes, align);
            lv.r = -1;
            if (l + 1 < L) {
                lv.r = poff;
                poff = up(poff + nodes, align);
            }
            b->hl.push_back(lv);
        }
        b->G = std::max(b->G, L - 1);
        b->hs.push_back(S);
    }
    // work items
    auto add_items = [&](int s, int level, int64_t total, std::vector<Item>& dst) {
        for (int64_t st = 0; st < total; st += b->chunk)
            dst.push_back({s, level, st, (int)std::min<int64_t>(b->chunk, total - st)});
    };
    auto pw = [](int64_t v, int d_) { return d_ == 3 ? v * v * v : v * v; };
    b->fine.resize(b->G + 1);
    b->coarse.resize(b->G + 1);
    b->cells.resize(b->G + 1);
    std::vector<Item> tmp;
    {  // level 0 interior items, grouped by solve (the finalize sums them in order)
        b->level0.off = (int)b->items.size();
        for (int s = 0; s < count; ++s) {
            b->hs[s].item0 = (int)b->items.size() - b->level0.off;
            add_items(s, 0, pw(b->hs[s].n - 1, b->hs[s].d), b->items);
            b->hs[s].item1 = (int)b->items.size() - b->level0.off;
        }
        b->level0.count = (int)b->items.size() - b->level0.off;
    }
    for (int g = 1; g <= b->G; ++g) {
        for (int kind = 0; kind < OP_COUNT; ++kind) {
            Range r;
            r.off = (int)b->items.size();
            for (int s = 0; s < count; ++s) {
                const BSolve& S = b->hs[s];
                const int l = S.levels - 1 - g;
                if (l < 0) continue;
                const int nl = S.n >> l, nc = nl / 2;
                if (kind == OP_FINE) {
                    // the vector kernels' items: (interior row, 16-byte group)
                    // pairs, chunk / V groups per item
                    const int V = 16 / b->elem;
                    const int64_t groups = (int64_t)(S.d == 3 ? (nl - 1) * (nl - 1) : nl - 1)
                                           << b->hl[S.lev0 + l].lgG;
                    const int64_t gchunk = std::max<int64_t>(1, b->chunk / V);
                    for (int64_t st = 0; st < groups; st += gchunk)
                        b->items.push_back({s, l, st, (int)std::min<int64_t>(gchunk, groups - st)});
                    continue;
                }
                const int64_t total = kind == OP_COARSE ? pw(nc - 1, S.d) : pw(nc, S.d);
                add_items(s, l, total, b->items);
            }
            r.count = (int)b->items.size() - r.off;
            (kind == OP_FINE ? b->fine : kind == OP_COARSE ? b->coarse : b->cells)[g] = r;
        }
    }
    cudaError_t e = cudaSuccess;
    auto al = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(bytes, 8));
        if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, std::max<size_t>(bytes, 8), b->stream);
    };
    al((void**)&b->ds, sizeof(BSolve) * count);
    al((void**)&b->dl, sizeof(BLevel) * b->hl.size());
    al((void**)&b->di, sizeof(Item) * b->items.size());
    al(&b->pool, (size_t)b->elem * poff);
    al((void**)&b->pool64, sizeof(double) * off64);
    al((void**)&b->partial, sizeof(double) * b->level0.count);
    al((void**)&b->res0_2, sizeof(double) * count);
    al((void**)&b->relres, sizeof(double) * count);
    al((void**)&b->active, sizeof(int) * count);
    al((void**)&b->iters, sizeof(int) * count);
    al((void**)&b->num_active, sizeof(int));
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? GMG_ERR_ALLOC : GMG_ERR_CUDA,
                    cudaGetErrorString(e));
    if (cudaMallocHost((void**)&b->h_active, sizeof(int)) != cudaSuccess)
        return fail(GMG_ERR_ALLOC, "cudaMallocHost failed");
    e = cudaMemcpyAsync(b->dl, b->hl.data(), sizeof(BLevel) * b->hl.size(), cudaMemcpyHostToDevice,
                        b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->di, b->items.data(), sizeof(Item) * b->items.size(),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail(GMG_ERR_CUDA, cudaGetErrorString(e));
    *out = b;
    return GMG_OK;
}

gmg_status gmg_batch_solve(gmg_batch b, const double* const* f, double* const* u, double rtol,
                           int* iters_out, double* relres_out, int* steps_out) {
    if (!b || !f || !u || !(rtol >= 0.0) || !std::isfinite(rtol)) {
        set_error("gmg_batch_solve: bad arguments");
        return GMG_ERR_ARG;
    }
    for (int s = 0; s < b->count; ++s) {
        if (!dev_ptr_ok(f[s]) || !dev_ptr_ok(u[s])) {
            set_error("gmg_batch_solve: f/u of solve " + std::to_string(s) +
                      " is not an aligned device pointer");
            return GMG_ERR_LAYOUT;
        }
        b->hs[s].f = f[s];
        b->hs[s].u = u[s];
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    struct Restore {
        int p, d;
        ~Restore() {
            if (p >= 0 && p != d) cudaSetDevice(p);
        }
    } restore{prev, b->device};
    const double rtol2 = rtol * rtol;
    GMG_CUDA_TRY(cudaEventRecord(b->ev, b->user_stream));
    GMG_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev, 0));
    GMG_CUDA_TRY(cudaMemcpyAsync(b->ds, b->hs.data(), sizeof(BSolve) * b->count,
                                 cudaMemcpyHostToDevice, b->stream));
    if (b->elem == 4)
        enqueue_start<float>(b);
    else
        enqueue_start<__nv_bfloat16>(b);
    GMG_CUDA_TRY(cudaGetLastError());
    if (b->graph && b->graph_rtol2 != rtol2) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (!b->graph) {
        cudaGraph_t g = nullptr;
        GMG_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        gmg_status st = b->elem == 4 ? enqueue_step<float>(b, rtol2)
                                     : enqueue_step<__nv_bfloat16>(b, rtol2);
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (st != GMG_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        GMG_CUDA_TRY(e);
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        GMG_CUDA_TRY(e);
        b->graph_rtol2 = rtol2;
    }
    GMG_CUDA_TRY(cudaMemcpyAsync(b->h_active, b->num_active, sizeof(int), cudaMemcpyDeviceToHost,
                                 b->stream));
    GMG_CUDA_TRY(cudaStreamSynchronize(b->stream));
    int steps = 0;
    while (*b->h_active > 0 && steps < b->cfg.maxit) {
        GMG_CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
        GMG_CUDA_TRY(cudaStreamSynchronize(b->stream));
        b->timer.after_graph_run();
        ++steps;
    }
    if (steps_out) *steps_out = steps;
    std::vector<int> it(b->count);
    std::vector<double> rel(b->count);
    GMG_CUDA_TRY(cudaMemcpy(it.data(), b->iters, sizeof(int) * b->count, cudaMemcpyDeviceToHost));
    GMG_CUDA_TRY(cudaMemcpy(rel.data(), b->relres, sizeof(double) * b->count,
                            cudaMemcpyDeviceToHost));
    bool all = true;
    for (int s = 0; s < b->count; ++s) {
        if (iters_out) iters_out[s] = it[s];
        if (relres_out) relres_out[s] = rel[s];
        if (!std::isfinite(rel[s])) {
            set_error("gmg_batch_solve: non-finite residual in solve " + std::to_string(s));
            return GMG_ERR_NONFINITE;
        }
        if (rel[s] > rtol) all = false;
    }
    if (!all) {
        set_error("gmg_batch_solve: some solves reached maxit above rtol");
        return GMG_ERR_NOT_CONVERGED;
    }
    return GMG_OK;
}

gmg_status gmg_batch_set_timing(gmg_batch b, int enable) {
    if (!b) {
        set_error("batch is NULL");
        return GMG_ERR_ARG;
    }
    if ((enable != 0) != b->timer.enabled) {
        b->timer.enabled = enable != 0;
        if (b->graph) {
            GMG_CUDA_TRY(cudaStreamSynchronize(b->stream));
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
    }
    b->timer.reset();
    return GMG_OK;
}

gmg_status gmg_batch_timing_report(gmg_batch b, gmg_kernel_stat* out, int cap, int* count,
                                   int64_t* launches_out) {
    if (!b || (!out && cap > 0)) {
        set_error("bad arguments");
        return GMG_ERR_ARG;
    }
    b->timer.report(out, cap, count, launches_out);
    return GMG_OK;
}

gmg_status gmg_create_batched(int count, const gmg_config* cfgs, void* cuda_stream,
                              gmg_batch* out) {
    if (!out || !cfgs || count < 1 || count > (1 << 20)) {
        set_error("gmg_create_batched: bad arguments");
        return GMG_ERR_ARG;
    }
    *out = nullptr;
    const gmg_config& c0 = cfgs[0];
    std::vector<int> d(count), n(count);
    for (int i = 0; i < count; ++i) {
        const gmg_config& c = cfgs[i];
        if (c.smoother != c0.smoother || c.omega != c0.omega || c.nu1 != c0.nu1 ||
            c.nu2 != c0.nu2 || c.precision != c0.precision || c.inner_cycles != c0.inner_cycles ||
            c.maxit != c0.maxit) {
            set_error("gmg_create_batched: solves differ in smoother, sweeps, precision, "
                      "inner_cycles or maxit");
            return GMG_ERR_ARG;
        }
        d[i] = c.d;
        n[i] = c.n;
    }
    return gmg_batch_create(count, d.data(), n.data(), &c0, 0, 0, cuda_stream, out);
}

gmg_status gmg_solve_batched(gmg_batch b, const double* const* f, double* const* u, double rtol,
                             int* iters_out) {
    return gmg_batch_solve(b, f, u, rtol, iters_out, nullptr, nullptr);
}

}  // extern "C"
