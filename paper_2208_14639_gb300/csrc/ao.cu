// AO-side assembly of the VV10 Fock matrix (Sec. II.A) and of the contracted orbital Hessian
// (Sec. II.B):
//   M_mu_nu = sum_i w_i [s_i phi_mu phi_nu + 2 v_i . (phi_nu grad phi_mu + phi_mu grad phi_nu)]
// with (s, v) = (f^rho, f^gamma grad rho) for F and (f^{rho,t}, f^{gamma,t} grad rho +
// f^gamma grad rho^t) for G^t.  With Z_i,mu = w_i (s_i phi_i,mu / 2 + 2 v_i . grad phi_i,mu),
// M = Phi^T Z + Z^T Phi: a plain FP64 GEMM over the kept points (cuBLAS; the channels of a
// chunk side by side as the columns of one product), then the symmetrisation.
#include <cublas_v2.h>

#include "common.cuh"
#include "kernels.hpp"

namespace vv10 {

namespace {

__global__ void k_ao_gather(PointsDev P, int32_t nbf, const double* __restrict__ phi,
                            double* __restrict__ phik) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= P.nk * nbf) return;
    const int64_t k = e / nbf;
    const int mu = static_cast<int>(e % nbf);
    phik[e] = phi[P.orig[k] * nbf + mu];
}

// Z[k][c - c0][mu] (rows of nc x nbf) for the channels c0 .. c0 + nc - 1, nc = gridDim.y.
// s: channel c's scalar at caller point i = s[c n + i]; the vector part is fg[c n + i]
// grad rho_k (+ vg[i] gt[(c n + i) 3 + d] when gt is given).
__global__ void k_ao_z(PointsDev P, int32_t nbf, const double* __restrict__ phi,
                       const double* __restrict__ dphi, const double* __restrict__ s,
                       const double* __restrict__ fg, const double* __restrict__ vg,
                       const double* __restrict__ gt, int32_t c0, double* __restrict__ Z) {
    const int c = c0 + static_cast<int>(blockIdx.y);
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= P.nk * nbf) return;
    const int64_t k = e / nbf;
    const int mu = static_cast<int>(e % nbf);
    const int64_t i = P.orig[k];
    const int64_t ci = static_cast<int64_t>(c) * P.n + i;
    const double w = P.w[k];
    double vx = fg[ci] * P.gx[k], vy = fg[ci] * P.gy[k], vz = fg[ci] * P.gz[k];
    if (gt) {
        const double f = vg[i];
        vx += f * gt[3 * ci];
        vy += f * gt[3 * ci + 1];
        vz += f * gt[3 * ci + 2];
    }
    const int64_t a = i * nbf + mu;
    const double* d = dphi + 3 * a;
    Z[(k * gridDim.y + blockIdx.y) * nbf + mu] =
        w * (0.5 * s[ci] * phi[a] + 2.0 * (vx * d[0] + vy * d[1] + vz * d[2]));
}

// out[c] = M_c + M_c^T (M_c column-major nbf x nbf)
__global__ void k_ao_sym(int32_t nbf, const double* __restrict__ M, double* __restrict__ out) {
    const int c = blockIdx.y;
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nn = static_cast<int64_t>(nbf) * nbf;
    if (e >= nn) return;
    const int mu = static_cast<int>(e / nbf), nu = static_cast<int>(e % nbf);
    const double* m = M + c * nn;
    out[c * nn + e] = m[mu + static_cast<int64_t>(nu) * nbf] + m[nu + static_cast<int64_t>(mu) * nbf];
}

}  // namespace

int64_t ao_channels_per_chunk(int64_t nk, int32_t nbf, int32_t n_ch, size_t max_bytes) {
    const size_t per = sizeof(double) * static_cast<size_t>(nk > 0 ? nk : 1) * static_cast<size_t>(nbf);
    int64_t c = static_cast<int64_t>(max_bytes / per);
    if (c < 1) c = 1;
    return c < n_ch ? c : n_ch;
}

cudaError_t launch_ao_assemble(const PointsDev& p, void* blas, int32_t nbf, const double* phi,
                               const double* dphi, int32_t n_ch, const double* s,
                               const double* fg, const double* vg, const double* gt,
                               int64_t chunk, double* phik, double* Z, double* M, double* out,
                               cudaStream_t st, int* blas_status) {
    *blas_status = 0;
    const int64_t nn = static_cast<int64_t>(nbf) * nbf;
    if (p.nk == 0) return cudaMemsetAsync(out, 0, sizeof(double) * nn * n_ch, st);
    const int64_t ne = p.nk * nbf;
    const unsigned gx = static_cast<unsigned>((ne + 255) / 256);
    k_ao_gather<<<gx, 256, 0, st>>>(p, nbf, phi, phik);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cublasHandle_t h = static_cast<cublasHandle_t>(blas);
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) {
        *blas_status = 1;
        return cudaSuccess;
    }
    const double one = 1.0, zero = 0.0;
    for (int32_t c0 = 0; c0 < n_ch; c0 += static_cast<int32_t>(chunk)) {
        const int32_t nc = static_cast<int32_t>(n_ch - c0 < chunk ? n_ch - c0 : chunk);
        k_ao_z<<<dim3(gx, static_cast<unsigned>(nc)), 256, 0, st>>>(p, nbf, phi, dphi, s, fg, vg, gt, c0, Z);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        // one GEMM for the chunk: M (column-major nbf x nc nbf) = A B^T with A = phik viewed
        // as nbf x nk and B = Z viewed as (nc nbf) x nk (both column-major); column c nbf + nu
        // of M is column nu of M_c
        const cublasStatus_t bs = cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_T, nbf, nc * nbf,
                                              static_cast<int>(p.nk), &one, phik, nbf, Z, nc * nbf,
                                              &zero, M, nbf);
        if (bs != CUBLAS_STATUS_SUCCESS) {
            *blas_status = static_cast<int>(bs);
            return cudaSuccess;
        }
        k_ao_sym<<<dim3(static_cast<unsigned>((nn + 255) / 256), static_cast<unsigned>(nc)), 256, 0, st>>>(
            nbf, M, out + c0 * nn);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int ao_blas_create(void** blas) {
    cublasHandle_t h = nullptr;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return 1;
    // the default (no atomics) keeps results bitwise reproducible
    *blas = h;
    return 0;
}

void ao_blas_destroy(void* blas) {
    if (blas) cublasDestroy(static_cast<cublasHandle_t>(blas));
}

}  // namespace vv10
