// The energy alone (Sec. II.A, quadrature form of E^VV10) from the unordered pairs:
//   E = beta sum_i c_i + sum_{i<j} c_i c_j Phi_ij + 1/2 sum_i c_i^2 Phi_ii,   c = w rho,
// since Phi_ij = Phi_ji.  The kept points are cut into blocks of 128; a task is a block pair
// (I, J) with J >= I, one thread per row of I looping over the 128 points of J (in the
// diagonal block only j >= i, the j = i term halved).  A persistent CTA walks tasks
// b, b + grid, ... and keeps one FP64 total; the per-CTA totals are summed in a fixed order,
// so the result does not depend on scheduling.
#include <cmath>

#include "common.cuh"
#include "kernels.hpp"
#include "pairsum.cuh"

namespace vv10 {

namespace {

constexpr int kEhThreads = 128;  // rows per block and points per j block

// Block pair of linear task index t (tasks ordered by I, then J = I .. nb - 1).
__device__ __forceinline__ void eh_task(int64_t t, int64_t nb, int64_t* I, int64_t* J) {
    // tasks before row block I: I nb - I (I - 1) / 2
    const double b = 2.0 * static_cast<double>(nb) + 1.0;
    int64_t i = static_cast<int64_t>((b - sqrt(b * b - 8.0 * static_cast<double>(t))) * 0.5);
    if (i < 0) i = 0;
    if (i > nb - 1) i = nb - 1;
    auto before = [nb](int64_t r) { return r * nb - r * (r - 1) / 2; };
    while (i > 0 && before(i) > t) --i;
    while (i + 1 < nb && before(i + 1) <= t) ++i;
    *I = i;
    *J = i + (t - before(i));
}

template <class T>
__global__ void __launch_bounds__(kEhThreads)
k_energy_half(PointsDev P, const typename PairRecs<T>::A* __restrict__ ra,
              const typename PairRecs<T>::B* __restrict__ rb, int64_t nb, int64_t n_tasks,
              double* __restrict__ cta_total) {
    using RA = typename PairRecs<T>::A;
    using RB = typename PairRecs<T>::B;
    __shared__ RA sa[kEhThreads];
    __shared__ RB sb[kEhThreads];
    __shared__ double sh[kEhThreads / 32];
    const int tid = threadIdx.x;
    double total = 0.0;  // meaningful in thread 0
    for (int64_t t = blockIdx.x; t < n_tasks; t += gridDim.x) {
        int64_t I = 0, J = 0;
        eh_task(t, nb, &I, &J);
        const int64_t i = I * kEhThreads + tid;
        const bool valid = i < P.nk;
        T xi = 0, yi = 0, zi = 0, oi = 1, ki = 1;
        double ci = 0.0;
        if (valid) {
            const RA a = ra[i];
            const RB b = rb[i];
            xi = a.x; yi = a.y; zi = a.z; oi = b.x; ki = b.y;
            ci = P.w[i] * P.rho[i];
        }
        const int64_t j0 = J * kEhThreads;
        const int cnt = static_cast<int>(P.nk - j0 < kEhThreads ? P.nk - j0 : kEhThreads);
        __syncthreads();  // the previous task's tile is no longer read
        if (tid < cnt) {
            sa[tid] = ra[j0 + tid];
            sb[tid] = rb[j0 + tid];
        }
        __syncthreads();
        // c_j Phi_ij of the pair (i, jj) (a.w = -3/2 c_j)
        auto term = [&](int jj) -> T {
            const RA a = sa[jj];
            const RB b = sb[jj];
            const T dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
            const T r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
            const T g = fmadd(oi, r2, ki);
            const T gp = fmadd(b.x, r2, b.y);
            return a.w * recip(g * gp * (g + gp));
        };
        T acc = T(0);
        const bool diag = (I == J);
        if (!diag) {
#pragma unroll 4
            for (int jj = 0; jj < cnt; ++jj) acc += term(jj);
        } else if (tid < cnt) {
            acc = T(0.5) * term(tid);  // j = i
            for (int jj = tid + 1; jj < cnt; ++jj) acc += term(jj);
        }
        double v = valid ? ci * static_cast<double>(acc) : 0.0;
        if (diag && valid) v += P.beta * ci;
        v = block_sum(v, sh);
        if (tid == 0) total += v;
    }
    if (tid == 0) cta_total[blockIdx.x] = total;
}

template <class T>
cudaError_t launch_eh(const PointsDev& p, const typename PairRecs<T>::A* ra,
                      const typename PairRecs<T>::B* rb, int grid, double* cta_total,
                      double* energy, cudaStream_t st) {
    const int64_t nb = (p.nk + kEhThreads - 1) / kEhThreads;
    const int64_t n_tasks = nb * (nb + 1) / 2;
    k_energy_half<T><<<grid, kEhThreads, 0, st>>>(p, ra, rb, nb, n_tasks, cta_total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_sum_blocks(cta_total, grid, energy, st);
}

}  // namespace

// Persistent grid of the energy-only kernel: whole waves of resident CTAs.
int energy_half_grid(bool fp64, int n_sm) {
    int per_sm = 0;
    cudaError_t e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_energy_half<double>, kEhThreads, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_energy_half<float>, kEhThreads, 0);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * (n_sm > 0 ? n_sm : 1);
}

cudaError_t launch_energy_half(const PointsDev& p, bool fp64, int grid, double* cta_total,
                               double* energy, cudaStream_t st) {
    if (p.nk == 0) return cudaMemsetAsync(energy, 0, sizeof(double), st);
    if (fp64) return launch_eh<double>(p, p.r64a, p.r64b, grid, cta_total, energy, st);
    return launch_eh<float>(p, p.r32a, p.r32b, grid, cta_total, energy, st);
}

}  // namespace vv10
