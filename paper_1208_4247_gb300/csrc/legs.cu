// Fused leg kernels (legs.cuh) on the GPU: the plane boxes arrive by TMA
// (cp.async.bulk.tensor, one tensor map per array, this GPU's own memory),
// each batch signalled by an mbarrier; the waits are bounded, and a CTA that
// gives up records a fault word (read by the solve) instead of hanging.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "legs.cuh"
#include "legs_api.h"

namespace gmg {
namespace legs {
namespace {

// Set by a CTA whose wait for a batch of plane loads gave up (about 2 s).
__device__ int g_fault;

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

template <typename T>
struct DevP {
    static constexpr bool kHost = false;
    const CUtensorMap* mu;  // fine iterate (read)
    const CUtensorMap* mq;  // fine right-hand side
    const CUtensorMap* mc;  // coarse iterate (up leg)
    uint64_t* bars;         // D+1 batch barriers
    int box_u_bytes, box_c_bytes;
    int* abort_flag;        // shared: a wait gave up

    __device__ int tid() const { return threadIdx.x; }
    __device__ int nt() const { return blockDim.x; }
    __device__ void sync() const { __syncthreads(); }
    __device__ void* host_scratch(size_t) { return nullptr; }
    __device__ void fence_async() const {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __device__ void tma(T* dst, const CUtensorMap* m, int x, int y, int z, uint64_t* bar) const {
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(saddr(dst)),
            "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(saddr(bar))
            : "memory");
    }
    // a batch: its byte count on barrier `bar` first, then its loads
    int cur_bar = 0;
    __device__ void begin(int bar, int fine_boxes, int coarse_boxes) {
        cur_bar = bar;
        const int bytes = fine_boxes * box_u_bytes + coarse_boxes * box_c_bytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         saddr(bars + bar)),
                     "r"(bytes)
                     : "memory");
    }
    __device__ void load_u(T* dst, int xh, int y, int z) { tma(dst, mu, xh, y, z, bars + cur_bar); }
    __device__ void load_q(T* dst, int xh, int y, int z) { tma(dst, mq, xh, y, z, bars + cur_bar); }
    __device__ void load_c(T* dst, int xh, int y, int z) { tma(dst, mc, xh, y, z, bars + cur_bar); }
    __device__ bool try_wait(int bar, int parity) const {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(saddr(bars + bar)), "r"(parity)
            : "memory");
        return ok != 0;
    }
    // thread 0 waits (bounded, about 2 s), the CTA learns the outcome at the
    // barrier, every thread then observes the completed phase itself
    __device__ bool wait(int bar, int parity) {
        if (threadIdx.x == 0) {
            const long long t0 = clock64();
            bool ok = try_wait(bar, parity);
            while (!ok && clock64() - t0 < 4000000000LL) ok = try_wait(bar, parity);
            *abort_flag = ok ? 0 : 1;
            if (!ok) atomicExch(&g_fault, 1);
        }
        __syncthreads();
        if (*abort_flag) return false;
        // completes at once: thread 0 saw the phase end
        for (int i = 0; i < (1 << 20) && !try_wait(bar, parity); ++i) {
        }
        return true;
    }
    // before leaving after a failed wait: give the batches still in flight
    // (issued for steps t .. min(t + D, zhi)) a bounded time to land
    __device__ void drain(int t, int zhi, int zlo) {
        if (threadIdx.x == 0) {
            for (int L = t; L <= zhi && L <= t + kD; ++L) {
                const int bar = (L - zlo) % (kD + 1);
                const int parity = ((L - zlo) / (kD + 1)) & 1;
                const long long t0 = clock64();
                while (!try_wait(bar, parity) && clock64() - t0 < 4000000000LL) {
                }
            }
        }
        __syncthreads();
    }
};

#ifndef GMG_LEG_MINB
#define GMG_LEG_MINB 1
#endif
template <typename T, int MODE, int S>
__global__ void __launch_bounds__(Geo<T, MODE, S>::NT, GMG_LEG_MINB)
    k_leg(const __grid_constant__ CUtensorMap mu, const __grid_constant__ CUtensorMap mq,
          const __grid_constant__ CUtensorMap mc, LegArgs<T> a) {
    using G = Geo<T, MODE, S>;
    extern __shared__ __align__(1024) unsigned char dsm[];
    T* slots = reinterpret_cast<T*>(dsm);
    uint64_t* bars = reinterpret_cast<uint64_t*>(dsm + (G::SMEM - 256));
    int* abort_flag = reinterpret_cast<int*>(bars + G::D + 1);
    if (threadIdx.x == 0) {
        for (int b = 0; b <= G::D; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bars + b)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    DevP<T> pl;
    pl.mu = &mu;
    pl.mq = &mq;
    pl.mc = &mc;
    pl.bars = bars;
    pl.box_u_bytes = G::BXH * G::BY * (int)sizeof(T);
    pl.box_c_bytes = G::BXHC * G::BYC * (int)sizeof(T);
    pl.abort_flag = abort_flag;
    leg_cta<T, MODE, S>(pl, a, blockIdx.x, blockIdx.y, blockIdx.z, slots);
}

// ------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// A 3D tensor map over a colour-split level array {sy, n+1, n+1} (elements
// of es bytes) with box {bx, by, 1}; rows and planes beyond the grid and
// entries beyond the row read as zero.
bool make_map(CUtensorMap* m, const void* base, const LayS& L, int es, int bx, int by) {
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return false;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)L.sy, (cuuint64_t)L.n + 1, (cuuint64_t)L.n + 1};
    const cuuint64_t strides[2] = {(cuuint64_t)L.sy * es, (cuuint64_t)L.sz * es};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(m, es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                          3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
        return false;
    }
    return true;
}

LayS lays(const Lay& L) { return LayS{L.n, L.he, L.sy, L.sz}; }

// z segments per column: the fewest CTA-rounds x plane steps per CTA, one
// CTA per SM (152 SMs); a CTA over zseg planes of its range runs
// scale * zseg + extra steps (the pipeline fill and the halo planes).
int seg_count(int tiles, int planes, int scale, int extra) {
    int best = 1;
    double best_cost = 1e30;
    for (int nseg = 1; nseg <= 64 && nseg <= planes; ++nseg) {
        const int zseg = (planes + nseg - 1) / nseg;
        const int ctas = tiles * ((planes + zseg - 1) / zseg);
        const double cost = (double)((ctas + 152 * GMG_LEG_MINB - 1) / (152 * GMG_LEG_MINB)) *
                            (scale * zseg + extra);
        if (cost < best_cost * 0.999) {
            best_cost = cost;
            best = nseg;
        }
    }
    if (const char* v = std::getenv("GMG_LEG_SEGS")) {
        const int s = std::atoi(v);
        if (s > 0) best = s;
    }
    return best;
}

template <typename T, int MODE, int S>
cudaError_t launch(const Lay& Fl, const Lay& Cll, const T* u_in, T* u_out, const T* q,
                   const T* ec, T* qc, T* uc, cudaStream_t s) {
    using G = Geo<T, MODE, S>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_leg<T, MODE, S>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const LayS F = lays(Fl), Cl = lays(Cll);
    CUtensorMap mu{}, mq{}, mc{};
    if (!make_map(&mu, u_in, F, sizeof(T), G::BXH, G::BY) ||
        !make_map(&mq, q, F, sizeof(T), G::BXH, G::BY))
        return cudaErrorInvalidValue;
    if (MODE == kUp) {
        if (!make_map(&mc, ec, Cl, sizeof(T), G::BXHC, G::BYC)) return cudaErrorInvalidValue;
    } else {
        mc = mu;
    }
    LegArgs<T> a{};
    a.F = F;
    a.Cl = Cl;
    a.u_in = u_in;
    a.u_out = u_out;
    a.qc = qc;
    a.uc = uc;
    const int n = F.n;
    const int tx = n / G::CX, ty = (n + G::CY - 1) / G::CY;
    const int planes = MODE == kDown ? Cl.n - 1 : n - 1;
    const int nseg = MODE == kDown ? seg_count(tx * ty, planes, 2, 2 * S + 3)
                                   : seg_count(tx * ty, planes, 1, 2 * S);
    a.zseg = (planes + nseg - 1) / nseg;
    dim3 grid(tx, ty, (planes + a.zseg - 1) / a.zseg);
    k_leg<T, MODE, S><<<grid, G::NT, G::SMEM, s>>>(mu, mq, mc, a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(int mode, int S, const Lay& F, const Lay& C, const T* u_in, T* u_out,
                     const T* q, const T* ec, T* qc, T* uc, cudaStream_t s) {
    if (mode == kDown) {
        switch (S) {
            case 2: return launch<T, kDown, 2>(F, C, u_in, u_out, q, ec, qc, uc, s);
            case 3: return launch<T, kDown, 3>(F, C, u_in, u_out, q, ec, qc, uc, s);
            case 4: return launch<T, kDown, 4>(F, C, u_in, u_out, q, ec, qc, uc, s);
        }
    } else {
        switch (S) {
            case 2: return launch<T, kUp, 2>(F, C, u_in, u_out, q, ec, qc, uc, s);
            case 3: return launch<T, kUp, 3>(F, C, u_in, u_out, q, ec, qc, uc, s);
            case 4: return launch<T, kUp, 4>(F, C, u_in, u_out, q, ec, qc, uc, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

template <typename T>
bool applies(int d, int n) {
    constexpr int cx = Geo<T, kDown, 4>::CX;
    static_assert(Geo<T, kDown, 2>::CX == cx && Geo<T, kUp, 4>::CX == cx, "one column width");
    return d == 3 && n >= 2 * cx && n % cx == 0;
}

template <typename T>
cudaError_t down(const Lay& F, const Lay& C, const T* u_in, T* u_out, const T* q, T* qc, T* uc,
                 int S, cudaStream_t s) {
    return dispatch<T>(kDown, S, F, C, u_in, u_out, q, nullptr, qc, uc, s);
}

template <typename T>
cudaError_t up(const Lay& C, const Lay& F, const T* ec, const T* u_in, T* u_out, const T* q,
               int S, cudaStream_t s) {
    return dispatch<T>(kUp, S, F, C, u_in, u_out, q, ec, nullptr, nullptr, s);
}

int fault() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_fault, sizeof(int)) != cudaSuccess) return -1;
    return v;
}

template bool applies<float>(int, int);
template bool applies<df32>(int, int);
template cudaError_t down<float>(const Lay&, const Lay&, const float*, float*, const float*,
                                 float*, float*, int, cudaStream_t);
template cudaError_t down<df32>(const Lay&, const Lay&, const df32*, df32*, const df32*, df32*,
                                df32*, int, cudaStream_t);
template cudaError_t up<float>(const Lay&, const Lay&, const float*, const float*, float*,
                               const float*, int, cudaStream_t);
template cudaError_t up<df32>(const Lay&, const Lay&, const df32*, const df32*, df32*,
                              const df32*, int, cudaStream_t);

}  // namespace legs
}  // namespace gmg
