// Fused red-black Gauss-Seidel sweep for the FP32 / BF16 inner cycles (3D):
// the red and the black half sweep in one pass over memory.
//
// A CTA owns a TX x TY column of interior nodes and a chunk of z planes, and
// streams the planes through a four-plane window in shared memory:
//   step k:  load plane k+1 (old values) and q of plane k;
//            red half sweep on plane k over the tile plus a one-node ring
//            (the ring's red values are what the tile's black nodes need from
//            the neighbouring columns; they are recomputed, not exchanged);
//            black half sweep on plane k-1 over the tile (its z neighbours
//            k-2 and k are red-updated by now);
//            store plane k-1 of the tile.
// Each node's update uses exactly the neighbour values of the two-kernel
// sweep (red from old black, black from new red, every value rounded to the
// storage type as it is stored), so the result is the same sweep.  The
// sweep reads u_in and writes u_out (u_in is not modified): CTAs read halo
// columns and chunk-boundary planes of other CTAs, which must stay the old
// values.  HBM traffic per sweep: u and q read once, u written once (12
// bytes/node in FP32), against two full passes for the two half sweeps.
#include "level_kernels.cuh"

namespace gmg {
namespace fused {
namespace {

using lk::Num;

constexpr int TX = 32, TY = 8, NT = TX * TY, CHUNK = 16;
constexpr int PX = TX + 4, PY = TY + 4, PL = PX * PY;

template <typename T>
__global__ void __launch_bounds__(NT) k_rb_sweep3(const T* __restrict__ uin, T* __restrict__ uout,
                                                  const T* __restrict__ q, int n) {
    using N = Num<T>;
    __shared__ float su[4][PL];
    __shared__ float sq[2][PL];
    const float c = 1.f / 6.f;
    const int tid = threadIdx.x;
    const int i0 = 1 + TX * blockIdx.x, j0 = 1 + TY * blockIdx.y;
    const int ks = 1 + CHUNK * blockIdx.z;
    const int ke = min(ks + CHUNK, n);  // black + store for planes ks .. ke-1
    const int64_t sy = (int64_t)n + 1, sz = sy * sy;

    auto load = [&](const T* src, float* dst, int k) {
        for (int m = tid; m < PL; m += NT) {
            const int i = i0 - 2 + m % PX, j = j0 - 2 + m / PX;
            float v = 0.f;
            if (k >= 0 && k <= n && i >= 0 && i <= n && j >= 0 && j <= n)
                v = N::ld(src[k * sz + j * sy + i]);
            dst[m] = v;
        }
    };
    // one colour of plane k over the window region [lo, PX-lo) x [lo, PY-lo):
    // lo = 1 is the tile plus its ring, lo = 2 the tile
    auto half = [&](int k, int color, int lo) {
        if (k < 1 || k > n - 1) return;
        float* uc = su[k & 3];
        const float* um = su[(k - 1) & 3];
        const float* up = su[(k + 1) & 3];
        const float* qk = sq[k & 1];
        const int w = PX - 2 * lo, h = PY - 2 * lo;
        for (int t = tid; t < w * h; t += NT) {
            const int sx = lo + t % w, syy = lo + t / w;
            const int i = i0 - 2 + sx, j = j0 - 2 + syy;
            if (i < 1 || i > n - 1 || j < 1 || j > n - 1 || ((i + j + k) & 1) != color) continue;
            const int m = syy * PX + sx;
            const float s = ((uc[m - 1] + uc[m + 1]) + (uc[m - PX] + uc[m + PX])) + (um[m] + up[m]);
            uc[m] = N::ld(N::st(fmaf(c, s, qk[m])));
        }
    };

    // prologue: planes ks-2 .. ks+1, q of ks-1; red on plane ks-1 over the tile
    for (int k = ks - 2; k <= ks + 1; ++k) load(uin, su[k & 3], k);
    load(q, sq[(ks - 1) & 1], ks - 1);
    __syncthreads();
    half(ks - 1, 0, 2);
    __syncthreads();
    for (int k = ks; k <= ke; ++k) {
        if (k > ks) load(uin, su[(k + 1) & 3], k + 1);
        load(q, sq[k & 1], k);
        __syncthreads();
        half(k, 0, 1);  // red, tile + ring
        __syncthreads();
        if (k - 1 >= ks) {
            half(k - 1, 1, 2);  // black, tile
            __syncthreads();
            const float* done = su[(k - 1) & 3];
            for (int m = tid; m < TX * TY; m += NT) {
                const int sx = 2 + m % TX, syy = 2 + m / TX;
                const int i = i0 - 2 + sx, j = j0 - 2 + syy;
                if (i <= n - 1 && j <= n - 1)
                    uout[(int64_t)(k - 1) * sz + j * sy + i] = N::st(done[syy * PX + sx]);
            }
        }
        __syncthreads();
    }
}

}  // namespace

template <typename T>
void rb_sweep3(int n, const T* uin, T* uout, const T* q, cudaStream_t s) {
    dim3 grid((n - 1 + TX - 1) / TX, (n - 1 + TY - 1) / TY, (n - 1 + CHUNK - 1) / CHUNK);
    k_rb_sweep3<T><<<grid, NT, 0, s>>>(uin, uout, q, n);
}

template void rb_sweep3<float>(int, const float*, float*, const float*, cudaStream_t);
template void rb_sweep3<__nv_bfloat16>(int, const __nv_bfloat16*, __nv_bfloat16*,
                                       const __nv_bfloat16*, cudaStream_t);

}  // namespace fused
}  // namespace gmg
