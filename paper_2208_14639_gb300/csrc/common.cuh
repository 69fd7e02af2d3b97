// Device-side helpers shared by the VV10 kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vv10 {

// Bits of the per-handle device error word (set with atomicOr, read at sync points).
enum : int {
    DEVERR_TIMEOUT = 1,       // a bounded wait gave up
    DEVERR_BAD_ATOM = 2,      // atom_of_point outside [0, n_atom)
    DEVERR_BAD_INPUT = 4,     // non-finite coordinate / weight / gradient
    DEVERR_NONFINITE = 8,     // non-finite output produced
};

// Spin-wait budget in SM clock cycles (~1 s at 2 GHz): a wait that exceeds it sets
// DEVERR_TIMEOUT and returns, so a kernel never hangs the device.
constexpr long long kSpinCycles = 2000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ------------------------------------------------------------------ mbarrier + bulk copy
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity to complete; false (and the TIMEOUT bit set in
// *err) if it did not within kSpinCycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kSpinCycles) {
            atomicOr(err, DEVERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// 1-D bulk asynchronous copy global -> shared (TMA engine), completion signalled as
// transaction bytes on `bar`.  dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ------------------------------------------------------------------ arithmetic
// Reciprocal in FP32: hardware approximation followed by one Newton-Raphson step
// r' = r + r (1 - x r), which roughly squares the relative error of r.
__device__ __forceinline__ float rcp_refined(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    const float e = fmaf(-x, r, 1.0f);
    return fmaf(r, e, r);
}
__device__ __forceinline__ float recip(float x) { return rcp_refined(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Packed per-point records of the pair kernels for arithmetic type T (PointsDev r32a/r32b or
// r64a/r64b): A = {x, y, z, -3/2 w rho}, B = {omega, kappa, rho kappa', rho omega_rho}.
template <class T> struct PairRecs;
template <> struct PairRecs<float> { using A = float4; using B = float4; };
template <> struct PairRecs<double> { using A = double4; using B = double4; };

// ------------------------------------------------------------------ reductions
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed tree for a fixed blockDim); result valid in thread 0.
// `sh` needs blockDim.x/32 elements.
template <class T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
    if (wid == 0) r = warp_sum(r);
    __syncthreads();
    return r;
}

// Error-free transformation of a sum (Knuth's TwoSum): s + e == a + b exactly.
// The molecule whose block range [pre[m], pre[m + 1]) holds launch block k (pre: n_mol + 1
// prefix sums, pre[0] = 0 <= k < pre[n_mol]; molecules with no blocks are skipped), and the
// block's index inside it.
__device__ __forceinline__ int batch_block_mol(const int64_t* __restrict__ pre, int n_mol,
                                               int64_t k, int64_t& local) {
    int lo = 0, hi = n_mol;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= k) lo = mid;
        else hi = mid;
    }
    local = k - pre[lo];
    return lo;
}

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

}  // namespace vv10
