// Weight-derivative sums (Sec. II.B, the three sums that follow the nuclear-Hessian blocks):
// for P weight directions v (the components of w^B, or any other),
//   E_i^v =  sum_j v_j rho_j Phi_ij
//   U_i^v = -sum_j v_j rho_j Phi_ij (1/(g + g') + 1/g)
//   W_i^v = -sum_j v_j rho_j Phi_ij R^2 (1/(g + g') + 1/g),
// i.e. E_i, U_i, W_i of Sec. II.A with v in place of w.  A prep kernel gathers the
// directions into kept order with -3/2 rho_j folded in (y_j = -3/2 rho_j v_j, so that
// y_j / (g g' s) = v_j rho_j Phi_ij); the contraction kernel takes one row per thread and PC
// directions per CTA, j in shared-memory tiles, T arithmetic within a tile and FP64 across
// tiles (per-thread totals in shared memory).  It serves the FP64 path and the mixed path for
// fewer than five directions (weight_tc.cu takes the others).
#include "common.cuh"
#include "kernels.hpp"
#include "pairsum.cuh"

namespace vv10 {

namespace {

constexpr int kWrThreads = 128;
constexpr int kWrJT = 128;  // j per shared-memory tile

__global__ void k_weight_dirs(PointsDev P, int32_t Pn, const double* __restrict__ wt,
                              double* __restrict__ yk) {
    const int p = blockIdx.y;
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= P.nk_pad || p >= Pn) return;
    double v = 0.0;
    if (k < P.nk) v = -1.5 * P.rho[k] * wt[static_cast<int64_t>(p) * P.n + P.orig[k]];
    yk[static_cast<int64_t>(p) * P.nk_pad + k] = v;
}

template <class T, int PC>
struct WrSmem {
    typename PairRecs<T>::A a[kWrJT];
    typename PairRecs<T>::B b[kWrJT];
    T y[kWrJT][PC];
    double tot[3 * PC][kWrThreads];
};

template <class T, int PC>
__global__ void __launch_bounds__(kWrThreads)
k_weight_resp(PointsDev P, const typename PairRecs<T>::A* __restrict__ ra,
              const typename PairRecs<T>::B* __restrict__ rb, const double* __restrict__ yk,
              int32_t Pn, double* __restrict__ outE, double* __restrict__ outU,
              double* __restrict__ outW) {
    using RA = typename PairRecs<T>::A;
    using RB = typename PairRecs<T>::B;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    WrSmem<T, PC>& S = *reinterpret_cast<WrSmem<T, PC>*>(smem_raw);
    const int tid = threadIdx.x;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kWrThreads + tid;
    const int c0 = blockIdx.y * PC;
    const bool valid = i < P.nk;
    T xi = 0, yi = 0, zi = 0, oi = 1, ki = 1;
    if (valid) {
        const RA a = ra[i];
        const RB b = rb[i];
        xi = a.x; yi = a.y; zi = a.z; oi = b.x; ki = b.y;
    }
#pragma unroll
    for (int q = 0; q < 3 * PC; ++q) S.tot[q][tid] = 0.0;
    for (int64_t j0 = 0; j0 < P.nk; j0 += kWrJT) {
        const int cnt = static_cast<int>(P.nk - j0 < kWrJT ? P.nk - j0 : kWrJT);
        __syncthreads();
        for (int t = tid; t < kWrJT; t += kWrThreads)
            if (t < cnt) {
                S.a[t] = ra[j0 + t];
                S.b[t] = rb[j0 + t];
            }
        for (int t = tid; t < kWrJT * PC; t += kWrThreads) {
            const int c = t / kWrJT, jj = t % kWrJT;  // j fastest: coalesced reads
            T v = T(0);
            if (jj < cnt && c0 + c < Pn) v = static_cast<T>(yk[static_cast<int64_t>(c0 + c) * P.nk_pad + j0 + jj]);
            S.y[jj][c] = v;
        }
        __syncthreads();
        T aE[PC], aU[PC], aW[PC];
#pragma unroll
        for (int c = 0; c < PC; ++c) aE[c] = aU[c] = aW[c] = T(0);
        for (int jj = 0; jj < cnt; ++jj) {
            const RA a = S.a[jj];
            const RB b = S.b[jj];
            const T dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
            const T r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
            const T g = fmadd(oi, r2, ki);
            const T gp = fmadd(b.x, r2, b.y);
            const T s = g + gp;
            const T ggp = g * gp;
            const T inv = recip(ggp * s);           // 1/(g g' s); Phi = -3/2 inv
            const T t1 = (ggp + gp * s) * inv;      // 1/s + 1/g
            const T k2 = inv * t1;
            const T k3 = k2 * r2;
#pragma unroll
            for (int c = 0; c < PC; ++c) {
                const T y = S.y[jj][c];
                aE[c] = fmadd(inv, y, aE[c]);
                aU[c] = fmadd(k2, y, aU[c]);
                aW[c] = fmadd(k3, y, aW[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < PC; ++c) {
            S.tot[3 * c][tid] += static_cast<double>(aE[c]);
            S.tot[3 * c + 1][tid] += static_cast<double>(aU[c]);
            S.tot[3 * c + 2][tid] += static_cast<double>(aW[c]);
        }
    }
    if (!valid) return;
    const int64_t oi_idx = P.orig[i];
#pragma unroll
    for (int c = 0; c < PC; ++c) {
        if (c0 + c >= Pn) break;
        const int64_t o = static_cast<int64_t>(c0 + c) * P.n + oi_idx;
        if (outE) outE[o] = S.tot[3 * c][tid];
        if (outU) outU[o] = -S.tot[3 * c + 1][tid];
        if (outW) outW[o] = -S.tot[3 * c + 2][tid];
    }
}

template <class T, int PC>
cudaError_t launch_wr(const PointsDev& p, const typename PairRecs<T>::A* ra,
                      const typename PairRecs<T>::B* rb, const double* yk, int32_t Pn, double* E,
                      double* U, double* W, cudaStream_t st) {
    const int bytes = static_cast<int>(sizeof(WrSmem<T, PC>));
    cudaError_t e = cudaFuncSetAttribute(k_weight_resp<T, PC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    const dim3 g(static_cast<unsigned>((p.nk + kWrThreads - 1) / kWrThreads),
                 static_cast<unsigned>((Pn + PC - 1) / PC));
    k_weight_resp<T, PC><<<g, kWrThreads, bytes, st>>>(p, ra, rb, yk, Pn, E, U, W);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_weight_dirs(const PointsDev& p, int32_t Pn, const double* wt, double* yk,
                               cudaStream_t st) {
    if (p.nk_pad == 0 || Pn <= 0) return cudaSuccess;
    const dim3 g(static_cast<unsigned>((p.nk_pad + 255) / 256), static_cast<unsigned>(Pn));
    k_weight_dirs<<<g, 256, 0, st>>>(p, Pn, wt, yk);
    return cudaGetLastError();
}

cudaError_t launch_weight_response(const PointsDev& p, bool fp64, int32_t Pn, const double* yk,
                                   double* E, double* U, double* W, cudaStream_t st) {
    if (p.nk == 0 || Pn <= 0) return cudaSuccess;
    // (the mixed path takes this kernel only for a few directions: tensor cores otherwise)
    if (fp64) return launch_wr<double, 8>(p, p.r64a, p.r64b, yk, Pn, E, U, W, st);
    return launch_wr<float, 8>(p, p.r32a, p.r32b, yk, Pn, E, U, W, st);
}

}  // namespace vv10
