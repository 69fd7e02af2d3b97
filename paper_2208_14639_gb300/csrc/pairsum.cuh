// Device side of the flash-style pair sums, shared by the single-system kernel and the
// batched work-queue kernel (see pairsum.cu for the modes and the arithmetic).
#pragma once

#include "common.cuh"
#include "kernels.hpp"

namespace vv10 {

template <class T> struct Recs;
template <> struct Recs<float> { using A = float4; using B = float4; };
template <> struct Recs<double> { using A = double4; using B = double4; };

__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class T>
struct Row {
    T x, y, z, om, ka;
};

// Accumulate one (i, j) pair into acc[0 .. nq-1] for the given mode.
template <class T, int MODE, class RA, class RB>
__device__ __forceinline__ void pair_accumulate(const Row<T>& r, const RA& a, const RB& b,
                                                T (&acc)[pair_mode_nq(MODE)]) {
    const T dx = r.x - a.x, dy = r.y - a.y, dz = r.z - a.z;
    T r2 = dx * dx;
    r2 = fmadd(dy, dy, r2);
    r2 = fmadd(dz, dz, r2);
    const T g = fmadd(r.om, r2, r.ka);
    const T gp = fmadd(b.x, r2, b.y);
    const T s = g + gp;
    const T ggp = g * gp;
    const T inv = recip(ggp * s);
    const T ph = a.w * inv;  // w_j rho_j Phi_ij  (a.w = -3/2 w_j rho_j)
    if constexpr (MODE == MODE_EUW) {
        const T t = ((g + s) * gp) * inv;  // 1/s + 1/g
        const T pt = ph * t;
        acc[0] += ph;
        acc[1] += pt;
        acc[2] = fmadd(pt, r2, acc[2]);
    } else if constexpr (MODE == MODE_EUWABC) {
        // both of the above from one evaluation of the pair
        const T L = ggp * inv;          // 1/s
        const T Gi = (gp * s) * inv;    // 1/g
        const T t = L + Gi;             // 1/s + 1/g
        const T pt = ph * t;
        acc[0] += ph;
        acc[1] += pt;
        acc[2] = fmadd(pt, r2, acc[2]);
        const T v = ph * fmadd(L, t, Gi * Gi);
        acc[3] += v;
        const T v2 = v * r2;
        acc[4] += v2;
        acc[5] = fmadd(v2, r2, acc[5]);
    } else if constexpr (MODE == MODE_EUWABCG) {
        // the six sums and the gradient sum of MODE_GRAD from one evaluation of the pair
        const T L = ggp * inv;          // 1/s
        const T Gi = (gp * s) * inv;    // 1/g
        const T t = L + Gi;             // 1/s + 1/g
        const T pt = ph * t;
        acc[0] += ph;
        acc[1] += pt;
        acc[2] = fmadd(pt, r2, acc[2]);
        const T v = ph * fmadd(L, t, Gi * Gi);
        acc[3] += v;
        const T v2 = v * r2;
        acc[4] += v2;
        acc[5] = fmadd(v2, r2, acc[5]);
        // D = omega_i/g + omega_j/g' + (omega_i + omega_j)/s
        const T Gj = (g * s) * inv;     // 1/g'
        const T D = fmadd(r.om, Gi, fmadd(b.x, Gj, (r.om + b.x) * L));
        const T f = ph * D;
        acc[6] = fmadd(f, dx, acc[6]);
        acc[7] = fmadd(f, dy, acc[7]);
        acc[8] = fmadd(f, dz, acc[8]);
    } else if constexpr (MODE == MODE_ABC) {
        const T L = ggp * inv;         // 1/s
        const T Gi = (gp * s) * inv;   // 1/g
        const T m = fmadd(L, L + Gi, Gi * Gi);
        const T v = ph * m;
        acc[0] += v;
        const T v2 = v * r2;
        acc[1] += v2;
        acc[2] = fmadd(v2, r2, acc[2]);
    } else {
        // D g g' s = omega_i g' (s + g) + omega_j g (s + g')
        const T num = fmadd(r.om * gp, s + g, (b.x * g) * (s + gp));
        const T f = (ph * inv) * num;
        acc[0] = fmadd(f, dx, acc[0]);
        acc[1] = fmadd(f, dy, acc[1]);
        acc[2] = fmadd(f, dz, acc[2]);
    }
}

// Streams j over [jb, je) (whole kJTile tiles) against the rows i0 + r*NT + tid of this CTA
// and adds the three sums of MODE into dacc (FP32 inside a tile, FP64 across tiles).
// `gtile` counts the tiles this CTA has already passed through its two shared-memory
// buffers; it selects buffer and mbarrier phase and is advanced by the tiles used here.
// Returns false (in every thread) if a bounded wait gave up.
template <class T, int MODE, int RPT, int NT>
__device__ __forceinline__ bool pairsum_range(typename Recs<T>::A (*sa)[kJTile],
                                              typename Recs<T>::B (*sb)[kJTile], uint64_t* bar,
                                              uint32_t& gtile, const typename Recs<T>::A* ra,
                                              const typename Recs<T>::B* rb, int64_t nk,
                                              int64_t i0, int64_t jb, int64_t je,
                                              double (&dacc)[RPT][pair_mode_nq(MODE)], int* err,
                                              bool stalled) {
    constexpr int NQ = pair_mode_nq(MODE);
    using RA = typename Recs<T>::A;
    using RB = typename Recs<T>::B;
    const int tid = threadIdx.x;
    const int ntile = je > jb ? static_cast<int>((je - jb) / kJTile) : 0;
    Row<T> row[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int64_t i = i0 + r * NT + tid;
        if (i < nk) {
            const RA a = ra[i];
            const RB b = rb[i];
            row[r] = Row<T>{a.x, a.y, a.z, b.x, b.y};
        } else {
            row[r] = Row<T>{T(0), T(0), T(0), T(1), T(1)};
        }
    }
    T acc[RPT][NQ];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            acc[r][q] = T(0);
            dacc[r][q] = 0.0;
        }
    constexpr uint32_t kBytesA = sizeof(RA) * kJTile, kBytesB = sizeof(RB) * kJTile;
    int issued = 0;
    if (tid == 0 && !stalled) {
        for (; issued < 2 && issued < ntile; ++issued) {
            const int b = (gtile + issued) & 1;
            const int64_t j0 = jb + static_cast<int64_t>(issued) * kJTile;
            mbar_expect_tx(&bar[b], kBytesA + kBytesB);
            bulk_g2s(sa[b], ra + j0, kBytesA, &bar[b]);
            bulk_g2s(sb[b], rb + j0, kBytesB, &bar[b]);
        }
    }
    int consumed = 0;
    bool all_ok = true;
    for (int t = 0; t < ntile; ++t) {
        const uint32_t g = gtile + t;
        const int buf = g & 1;
        const bool ok = mbar_wait(&bar[buf], (g >> 1) & 1, err);
        const RA* A = sa[buf];
        const RB* B = sb[buf];
#pragma unroll 2
        for (int jj = 0; jj < kJTile; ++jj) {
            const RA a = A[jj];
            const RB b = B[jj];
#pragma unroll
            for (int r = 0; r < RPT; ++r) pair_accumulate<T, MODE>(row[r], a, b, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                dacc[r][q] += static_cast<double>(acc[r][q]);
                acc[r][q] = T(0);
            }
        consumed = t + 1;
        if (__syncthreads_or(!ok)) {  // every thread leaves together
            all_ok = false;
            break;
        }
        if (tid == 0 && !stalled && issued < ntile) {
            const int64_t j0 = jb + static_cast<int64_t>(issued) * kJTile;
            mbar_expect_tx(&bar[buf], kBytesA + kBytesB);
            bulk_g2s(sa[buf], ra + j0, kBytesA, &bar[buf]);
            bulk_g2s(sb[buf], rb + j0, kBytesB, &bar[buf]);
            ++issued;
        }
    }
    // After a timeout, wait (bounded) for copies still in flight before leaving.
    if (tid == 0)
        for (int t = consumed; t < issued; ++t) {
            const uint32_t g = gtile + t;
            mbar_wait(&bar[g & 1], (g >> 1) & 1, err);
        }
    gtile += ntile;
    return all_ok;
}

}  // namespace vv10
