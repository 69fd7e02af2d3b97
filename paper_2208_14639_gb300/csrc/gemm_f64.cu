// FP64 product C = A B^T over a long inner dimension, for the AO-side assembly (Sec. II.A
// Fock-matrix equation, Sec. II.B G^t and F^A): A is M x K and B is N x K, both stored with
// their K index slowest (column k of A at A + k lda, the M values of a column contiguous),
// C is M x N column-major.  M and N are basis-function counts (tens to a few thousand), K the
// number of kept grid points (10^4 .. 10^6).
//
// 64 x 64 tiles of C, 256 threads with 4 x 4 results each, 16 k per shared-memory step (both
// operand tiles loaded with unit stride in m or n), the K range split over gridDim.z CTAs so
// that the grid fills the SMs; each split writes its own partial tile and a second kernel adds
// the splits in a fixed order (results do not depend on timing).  The arithmetic is FP64 FMA
// throughout: GB300's narrow FP64 pipe, not memory, bounds it.
#include "common.cuh"
#include "kernels.hpp"

namespace vv10 {

namespace {

constexpr int kGT = 64;   // tile edge in m and n
constexpr int kGK = 16;   // k per shared-memory step
constexpr int kGThreads = 256;

__global__ void __launch_bounds__(kGThreads)
k_gemm_abt(int M, int N, int64_t K, int64_t k_per_split, const double* __restrict__ A,
           int64_t lda, const double* __restrict__ B, int64_t ldb, double* __restrict__ out,
           int64_t ldo, int64_t split_stride) {
    __shared__ double sa[kGK][kGT];
    __shared__ double sb[kGK][kGT];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * kGT, n0 = blockIdx.y * kGT;
    const int64_t kb = static_cast<int64_t>(blockIdx.z) * k_per_split;
    const int64_t ke = kb + k_per_split < K ? kb + k_per_split : K;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    // loader mapping: 256 threads x 4 elements = one 16 x 64 tile; thread -> (k row, 4 m/n)
    const int lk = tid >> 4, lm = (tid & 15) * 4;
    for (int64_t k0 = kb; k0 < ke; k0 += kGK) {
        const int64_t k = k0 + lk;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int m = m0 + lm + q, n = n0 + lm + q;
            sa[lk][lm + q] = (k < ke && m < M) ? A[k * lda + m] : 0.0;
            sb[lk][lm + q] = (k < ke && n < N) ? B[k * ldb + n] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sa[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sb[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double* o = out + static_cast<int64_t>(blockIdx.z) * split_stride;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int n = n0 + ty + 16 * j;
        if (n >= N) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = m0 + tx + 16 * i;
            if (m < M) o[static_cast<int64_t>(n) * ldo + m] = acc[i][j];
        }
    }
}

// C[m + n ldc] = sum over the splits, in split order.
__global__ void k_gemm_reduce(int M, int N, int n_split, const double* __restrict__ part,
                              double* __restrict__ C, int64_t ldc) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t mn = static_cast<int64_t>(M) * N;
    if (e >= mn) return;
    double s = 0.0;
    for (int z = 0; z < n_split; ++z) s += part[z * mn + e];
    const int64_t n = e / M, m = e % M;
    C[n * ldc + m] = s;
}

}  // namespace

int gemm_abt_splits(int M, int N, int64_t K, int n_sm) {
    const int64_t tiles = static_cast<int64_t>((M + kGT - 1) / kGT) * ((N + kGT - 1) / kGT);
    int64_t s = (4 * static_cast<int64_t>(n_sm) + tiles - 1) / tiles;  // ~4 CTAs per SM
    const int64_t kmax = (K + 8 * kGK - 1) / (8 * kGK);                // >= 8 steps per split
    if (s > kmax) s = kmax;
    if (s > 64) s = 64;
    return static_cast<int>(s < 1 ? 1 : s);
}

cudaError_t launch_gemm_abt(int M, int N, int64_t K, const double* A, int64_t lda, const double* B,
                            int64_t ldb, double* C, int64_t ldc, double* work, int n_split,
                            cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K <= 0) {
        for (int n = 0; n < N; ++n) {
            cudaError_t e = cudaMemsetAsync(C + static_cast<int64_t>(n) * ldc, 0, sizeof(double) * M, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (n_split < 1) n_split = 1;
    int64_t kps = (K + n_split - 1) / n_split;
    kps = ((kps + kGK - 1) / kGK) * kGK;
    n_split = static_cast<int>((K + kps - 1) / kps);
    const dim3 grid(static_cast<unsigned>((M + kGT - 1) / kGT), static_cast<unsigned>((N + kGT - 1) / kGT),
                    static_cast<unsigned>(n_split));
    if (n_split == 1) {
        k_gemm_abt<<<grid, kGThreads, 0, st>>>(M, N, K, kps, A, lda, B, ldb, C, ldc, 0);
        return cudaGetLastError();
    }
    const int64_t mn = static_cast<int64_t>(M) * N;
    k_gemm_abt<<<grid, kGThreads, 0, st>>>(M, N, K, kps, A, lda, B, ldb, work, M, mn);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gemm_reduce<<<static_cast<unsigned>((mn + 255) / 256), 256, 0, st>>>(M, N, n_split, work, C, ldc);
    return cudaGetLastError();
}

}  // namespace vv10
