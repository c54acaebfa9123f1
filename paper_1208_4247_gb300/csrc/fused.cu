// Fused red-black Gauss-Seidel sweep for the FP32 inner cycles (3D):
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
// sweep (red from old black, black from new red), so the result is the same
// sweep, bit for bit.  The
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

__device__ inline void cp_async4(float* smem, const float* gmem) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(gmem));
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// FP32 storage: planes arrive by cp.async one step ahead of their use (five
// u slots, three q slots), so the HBM latency of plane k+2 overlaps the
// sweeps of planes k and k-1.
__global__ void __launch_bounds__(NT) k_rb_sweep3_f32(const float* __restrict__ uin,
                                                      float* __restrict__ uout,
                                                      const float* __restrict__ q, int n) {
    __shared__ float su[5][PL];
    __shared__ float sq[3][PL];
    const float c = 1.f / 6.f;
    const int tid = threadIdx.x;
    const int i0 = 1 + TX * blockIdx.x, j0 = 1 + TY * blockIdx.y;
    const int ks = 1 + CHUNK * blockIdx.z;
    const int ke = min(ks + CHUNK, n);
    const int64_t sy = (int64_t)n + 1, sz = sy * sy;
    auto slot = [](int k) { return (k + 10) % 5; };
    auto qslot = [](int k) { return (k + 9) % 3; };
    // asynchronous plane copy (zeros outside the grid written directly)
    auto fetch = [&](const float* src, float* dst, int k) {
        for (int m = tid; m < PL; m += NT) {
            const int i = i0 - 2 + m % PX, j = j0 - 2 + m / PX;
            if (k >= 0 && k <= n && i >= 0 && i <= n && j >= 0 && j <= n)
                cp_async4(&dst[m], &src[k * sz + j * sy + i]);
            else
                dst[m] = 0.f;
        }
    };
    // one colour of plane k over the window region [LO, PX-LO) x [LO, PY-LO)
    // (LO = 1: tile plus ring, LO = 2: tile); compile-time region width
    auto half = [&]<int LO>(int k, int color) {
        if (k < 1 || k > n - 1) return;
        constexpr int W = PX - 2 * LO, HH = PY - 2 * LO;
        float* uc = su[slot(k)];
        const float* um = su[slot(k - 1)];
        const float* up = su[slot(k + 1)];
        const float* qk = sq[qslot(k)];
        for (int t = tid; t < W * HH; t += NT) {
            const int sx = LO + t % W, syy = LO + t / W;
            const int i = i0 - 2 + sx, j = j0 - 2 + syy;
            if (i < 1 || i > n - 1 || j < 1 || j > n - 1 || ((i + j + k) & 1) != color) continue;
            const int m = syy * PX + sx;
            const float s = ((uc[m - 1] + uc[m + 1]) + (uc[m - PX] + um[m])) + (uc[m + PX] + up[m]);
            uc[m] = fmaf(c, s, qk[m]);
        }
    };
    // prologue: planes ks-2 .. ks+1 and q of ks-1, ks
    for (int k = ks - 2; k <= ks + 1; ++k) fetch(uin, su[slot(k)], k);
    fetch(q, sq[qslot(ks - 1)], ks - 1);
    fetch(q, sq[qslot(ks)], ks);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    half.template operator()<2>(ks - 1, 0);
    for (int k = ks; k <= ke; ++k) {
        // plane k+2 and q of k+1 in flight while planes k, k-1 are swept
        fetch(uin, su[slot(k + 2)], k + 2);
        fetch(q, sq[qslot(k + 1)], k + 1);
        cp_async_commit();
        __syncthreads();
        half.template operator()<1>(k, 0);  // red, tile + ring
        __syncthreads();
        if (k - 1 >= ks) {
            half.template operator()<2>(k - 1, 1);  // black, tile
            __syncthreads();
            const float* done = su[slot(k - 1)];
            for (int m = tid; m < TX * TY; m += NT) {
                const int sx = 2 + m % TX, syy = 2 + m / TX;
                const int i = i0 - 2 + sx, j = j0 - 2 + syy;
                if (i <= n - 1 && j <= n - 1)
                    uout[(int64_t)(k - 1) * sz + j * sy + i] = done[syy * PX + sx];
            }
        }
        cp_async_wait<0>();
        __syncthreads();
    }
}

}  // namespace

void rb_sweep3_f32(int n, const float* uin, float* uout, const float* q, cudaStream_t s) {
    dim3 grid((n - 1 + TX - 1) / TX, (n - 1 + TY - 1) / TY, (n - 1 + CHUNK - 1) / CHUNK);
    k_rb_sweep3_f32<<<grid, NT, 0, s>>>(uin, uout, q, n);
}

}  // namespace fused
}  // namespace gmg
