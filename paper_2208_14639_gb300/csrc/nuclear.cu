// The density and weight terms of the VV10 nuclear gradient (Sec. II.A):
//   E^A_G = sum_i w_i (f^rho_i rho^A_i + 2 f^gamma_i grad rho_i . grad rho^A_i),
//   E^A_w = sum_i w^A_i rho_i (beta + E_i),
// for P directions (rho^p, grad rho^p, w^p), with f^rho, f^gamma formed from the row sums
// E_i, U_i, W_i cached by the last energy call.  Deterministic: per-block partial sums per
// direction, then a fixed-order sum per direction.
#include "common.cuh"
#include "kernels.hpp"

namespace vv10 {

namespace {

constexpr int kNgThreads = 256;

__global__ void __launch_bounds__(kNgThreads)
k_ngrad_partial(PointsDev P, const double* __restrict__ sE, const double* __restrict__ sU,
                const double* __restrict__ sW, const double* __restrict__ rt,
                const double* __restrict__ gt, const double* __restrict__ wt, int64_t per_block,
                double* __restrict__ partial) {
    __shared__ double sh[kNgThreads / 32];
    const int p = blockIdx.y;
    const int64_t k0 = static_cast<int64_t>(blockIdx.x) * per_block;
    const int64_t k1 = k0 + per_block < P.nk ? k0 + per_block : P.nk;
    double acc = 0.0;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += kNgThreads) {
        const int64_t i = P.orig[k];
        const int64_t pi = static_cast<int64_t>(p) * P.n + i;
        const double rho = P.rho[k];
        if (rt) {
            const double fr = P.beta + sE[k] + rho * (P.ka_r[k] * sU[k] + P.om_r[k] * sW[k]);
            const double fg = rho * P.om_g[k] * sW[k];
            const double* g = gt + 3 * pi;
            acc += P.w[k] * (fr * rt[pi] + 2.0 * fg * (P.gx[k] * g[0] + P.gy[k] * g[1] + P.gz[k] * g[2]));
        }
        if (wt) acc += wt[pi] * rho * (P.beta + sE[k]);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[static_cast<int64_t>(p) * gridDim.x + blockIdx.x] = acc;
}

__global__ void k_ngrad_sum(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    const int p = blockIdx.x;
    double s = 0.0, c = 0.0;  // compensated, in block order
    for (int b = 0; b < nblk; ++b) {
        const double x = partial[static_cast<int64_t>(p) * nblk + b];
        const double t = s + x;
        c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    out[p] = s + c;
}

}  // namespace

int ngrad_blocks(int64_t nk) {
    const int64_t b = (nk + 8 * kNgThreads - 1) / (8 * kNgThreads);
    return static_cast<int>(b < 1 ? 1 : (b > 512 ? 512 : b));
}

cudaError_t launch_nuclear_gradient(const PointsDev& p, const double* sE, const double* sU,
                                    const double* sW, int32_t Pn, const double* rt,
                                    const double* gt, const double* wt, double* partial,
                                    double* out, cudaStream_t st) {
    if (Pn <= 0) return cudaSuccess;
    if (p.nk == 0) return cudaMemsetAsync(out, 0, sizeof(double) * Pn, st);
    const int nblk = ngrad_blocks(p.nk);
    const int64_t per_block = (p.nk + nblk - 1) / nblk;
    k_ngrad_partial<<<dim3(nblk, Pn), kNgThreads, 0, st>>>(p, sE, sU, sW, rt, gt, wt, per_block, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ngrad_sum<<<Pn, 32, 0, st>>>(partial, nblk, out);
    return cudaGetLastError();
}

}  // namespace vv10
