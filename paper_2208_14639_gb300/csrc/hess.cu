// K3: nonlocal response contracted with P trial densities (Sec. II.B, Eq. frhot).
//
// With L = 1/s, G_i = 1/g, G_j = 1/g', M = 2/s^2 + 2/(g g'), rho_i a_i = p_i + q_i R^2
// (p = rho kappa', q = rho omega_rho), sigma = rho omega_gamma, the pair parts of
// f^{rho rho}, f^{rho gamma}, f^{gamma rho}, f^{gamma gamma} printed in Sec. II.B factor as
//   f^{rho rho}_ij     = T1 = Phi [1 - rho_i a_i (L+G_i) - rho_j a_j (L+G_j) + rho_i a_i rho_j a_j M]
//   f^{rho gamma}_ij   = sigma_j T2,  T2 = R^2 Phi [rho_i a_i M - (L + G_j)]
//   f^{gamma rho}_ij   = sigma_i T3,  T3 = R^2 Phi [rho_j a_j M - (L + G_i)]
//   f^{gamma gamma}_ij = sigma_i sigma_j T4,  T4 = R^4 Phi M
// so with u_jt = w_j rho^t_j and y_jt = 2 w_j sigma_j gamma^t_j
//   f^{rho,t}_i   = sum_j (T1 u_jt + T2 y_jt)            + diagonal terms
//   f^{gamma,t}_i = sigma_i sum_j (T3 u_jt + T4 y_jt)    + diagonal terms,
// a product of a generated N x 2N kernel matrix with a 2N x P trial matrix.  The
// diagonal terms are the delta_ij / w_i parts of the four printed coefficients.
#include "common.cuh"
#include "kernels.hpp"
#include "tc.cuh"

namespace vv10 {

__host__ __device__ static inline int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

__global__ void __launch_bounds__(256)
k_trial_prep(PointsDev P, int32_t Pn, const double* __restrict__ rho_t,
             const double* __restrict__ grad_rho_t, double* __restrict__ u,
             double* __restrict__ y, double* __restrict__ rt_k, double* __restrict__ gt_k) {
    const int t = blockIdx.y;
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= P.nk_pad) return;
    const int64_t o = static_cast<int64_t>(t) * P.nk_pad + p;
    if (p >= P.nk) {
        u[o] = 0.0;
        y[o] = 0.0;
        return;
    }
    const int64_t i = P.orig[p];
    const int64_t src = static_cast<int64_t>(t) * P.n + i;
    const double rt = rho_t[src];
    const double* g = grad_rho_t + 3 * src;
    const double gt = P.gx[p] * g[0] + P.gy[p] * g[1] + P.gz[p] * g[2];  // gamma^t
    const double w = P.w[p];
    u[o] = w * rt;
    y[o] = 2.0 * w * (P.rho[p] * P.om_g[p]) * gt;
    rt_k[static_cast<int64_t>(t) * P.nk + p] = rt;
    gt_k[static_cast<int64_t>(t) * P.nk + p] = gt;
}

// Batched: trial values and their split-TF32 cut in one pass (the same values as
// k_trial_prep followed by the tensor-core path's trial split).  Rows t >= n_t are zero.
__global__ void __launch_bounds__(256)
k_trial_tc_batch(const EpiMol* __restrict__ mols, const int64_t* __restrict__ pre, int n_mol,
                 const double* __restrict__ rho_t, const double* __restrict__ grad_rho_t) {
    int64_t blk;
    const EpiMol& M = mols[batch_block_mol(pre, n_mol, blockIdx.x, blk)];
    const int64_t nb = M.P.nk_pad / 256;
    const int t = static_cast<int>(blk / nb);
    const int64_t p = (blk - t * nb) * 256 + threadIdx.x;
    float a = 0.f, c = 0.f;
    if (t < M.n_t && p < M.P.nk) {
        double u, y, rt, gt;
        trial_values(M.P, rho_t + M.toff, grad_rho_t + 3 * M.toff, t, p, u, y, rt, gt);
        M.rt[static_cast<int64_t>(t) * M.P.nk + p] = rt;
        M.gt[static_cast<int64_t>(t) * M.P.nk + p] = gt;
        a = static_cast<float>(-1.5 * u);  // the kernel tiles omit the -3/2 of Phi and the sign of T2
        c = static_cast<float>(1.5 * y);
    }
    const float ah = __uint_as_float(tc::to_tf32(a)), ch = __uint_as_float(tc::to_tf32(c));
    const int64_t o = static_cast<int64_t>(t) * M.P.nk_pad + p;
    float* sp = static_cast<float*>(M.split);
    sp[o] = ah;
    sp[M.split_step + o] = a - ah;
    sp[2 * M.split_step + o] = ch;
    sp[3 * M.split_step + o] = c - ch;
}

cudaError_t launch_trial_tc_batch(const EpiMol* mols, const int64_t* pre, int n_mol, int64_t n_blocks,
                                  const double* rho_t, const double* grad_rho_t, cudaStream_t st) {
    if (n_blocks <= 0) return cudaSuccess;
    k_trial_tc_batch<<<static_cast<unsigned>(n_blocks), 256, 0, st>>>(mols, pre, n_mol, rho_t,
                                                                      grad_rho_t);
    return cudaGetLastError();
}

cudaError_t launch_trial_prep(const PointsDev& p, int32_t P, const double* rho_t,
                              const double* grad_rho_t, double* u, double* y, double* rt_k,
                              double* gt_k, cudaStream_t st) {
    if (p.nk_pad == 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>(cdiv64(p.nk_pad, 256)), static_cast<unsigned>(P));
    k_trial_prep<<<grid, 256, 0, st>>>(p, P, rho_t, grad_rho_t, u, y, rt_k, gt_k);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 SIMT contraction
constexpr int kHessThreads = 128;
constexpr int kHessJT = 32;

// The four generated kernel values of one pair (FP64).
struct Tiles64 {
    double t1, t2, t3, t4;
};
__device__ __forceinline__ Tiles64 tiles64(double xi, double yi, double zi, double oi, double ki,
                                           double pi_, double qi, const double4& a,
                                           const double4& b) {
    const double dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double g = oi * r2 + ki;
    const double gp = b.x * r2 + b.y;
    const double s = g + gp;
    const double inv = 1.0 / (g * gp * s);
    const double phi = -1.5 * inv;
    const double L = g * gp * inv, Gi = gp * s * inv, Gj = g * s * inv;
    const double M = 2.0 * (L * L + Gi * Gj);
    const double Ai = pi_ + qi * r2, Aj = b.z + b.w * r2;
    const double LGi = L + Gi, LGj = L + Gj;
    Tiles64 T;
    T.t1 = phi * (1.0 - Ai * LGi - Aj * LGj + Ai * Aj * M);
    const double rp = r2 * phi;
    T.t2 = rp * (Ai * M - LGj);
    T.t3 = rp * (Aj * M - LGi);
    T.t4 = rp * r2 * M;
    return T;
}

template <int PC>
__global__ void __launch_bounds__(kHessThreads)
k_hess_f64(PointsDev P, int32_t Pn, const double* __restrict__ u, const double* __restrict__ y,
           int64_t j_per_split, double* __restrict__ acc) {
    __shared__ __align__(16) double4 sA[kHessJT];
    __shared__ __align__(16) double4 sB[kHessJT];
    __shared__ double su[PC][kHessJT];
    __shared__ double sy[PC][kHessJT];
    const int tid = threadIdx.x;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kHessThreads + tid;
    const int t0 = blockIdx.y * PC;
    const int split = blockIdx.z, n_split = gridDim.z;
    const int64_t jb = static_cast<int64_t>(split) * j_per_split;
    const int64_t je = min(P.nk_pad, jb + j_per_split);

    double xi = 0, yi = 0, zi = 0, oi = 1, ki = 1, pi_ = 0, qi = 0;
    if (i < P.nk) {
        const double4 a = P.r64a[i], b = P.r64b[i];
        xi = a.x; yi = a.y; zi = a.z; oi = b.x; ki = b.y; pi_ = b.z; qi = b.w;
    }
    double ar[PC], ag[PC];
#pragma unroll
    for (int k = 0; k < PC; ++k) { ar[k] = 0.0; ag[k] = 0.0; }

    for (int64_t j0 = jb; j0 < je; j0 += kHessJT) {
        __syncthreads();
        if (tid < kHessJT) sA[tid] = P.r64a[j0 + tid];
        else if (tid < 2 * kHessJT) sB[tid - kHessJT] = P.r64b[j0 + tid - kHessJT];
        for (int e = tid; e < PC * kHessJT; e += kHessThreads) {
            const int tt = e / kHessJT, jj = e % kHessJT;
            const int t = t0 + tt;
            const int64_t o = static_cast<int64_t>(t) * P.nk_pad + j0 + jj;
            su[tt][jj] = (t < Pn) ? u[o] : 0.0;
            sy[tt][jj] = (t < Pn) ? y[o] : 0.0;
        }
        __syncthreads();
#pragma unroll 1
        for (int jj = 0; jj < kHessJT; ++jj) {
            const Tiles64 T = tiles64(xi, yi, zi, oi, ki, pi_, qi, sA[jj], sB[jj]);
#pragma unroll
            for (int k = 0; k < PC; ++k) {
                const double uu = su[k][jj], yy = sy[k][jj];
                ar[k] = fma(T.t1, uu, fma(T.t2, yy, ar[k]));
                ag[k] = fma(T.t3, uu, fma(T.t4, yy, ag[k]));
            }
        }
    }
    if (i < P.nk) {
#pragma unroll
        for (int k = 0; k < PC; ++k) {
            const int t = t0 + k;
            if (t < Pn) {
                acc[((static_cast<int64_t>(0) * n_split + split) * Pn + t) * P.nk_pad + i] = ar[k];
                acc[((static_cast<int64_t>(1) * n_split + split) * Pn + t) * P.nk_pad + i] = ag[k];
            }
        }
    }
}

static inline void hess_split_geometry(int64_t nk_pad, int req, int64_t& jps, int& ns) {
    const int64_t ntile = nk_pad / kJTile;
    if (req < 1) req = 1;
    if (req > ntile) req = static_cast<int>(ntile > 0 ? ntile : 1);
    const int64_t tps = cdiv64(ntile, req);
    jps = tps * kJTile;
    ns = static_cast<int>(ntile > 0 ? cdiv64(ntile, tps) : 1);
}

int hess_f64_default_split(const PointsDev& p, int32_t P, int pc, int n_sm) {
    const int64_t ctas = cdiv64(p.nk, kHessThreads) * cdiv64(P, pc);
    const int64_t target = static_cast<int64_t>(n_sm) * 6;
    int req = static_cast<int>(cdiv64(target, ctas > 0 ? ctas : 1));
    int64_t jps;
    int ns;
    hess_split_geometry(p.nk_pad, req, jps, ns);
    return ns;
}

cudaError_t launch_hess_f64(const PointsDev& p, int32_t P, const double* u, const double* y,
                            const HessLaunch& cfg, double* acc, int* err, cudaStream_t st) {
    (void)err;
    if (p.nk == 0) return cudaSuccess;
    int64_t jps;
    int ns;
    hess_split_geometry(p.nk_pad, cfg.n_split, jps, ns);
    const int pc = cfg.trials_per_cta <= 8 ? 8 : (cfg.trials_per_cta <= 16 ? 16 : 32);
    dim3 grid(static_cast<unsigned>(cdiv64(p.nk, kHessThreads)),
              static_cast<unsigned>(cdiv64(P, pc)), static_cast<unsigned>(ns));
    if (pc == 8) k_hess_f64<8><<<grid, kHessThreads, 0, st>>>(p, P, u, y, jps, acc);
    else if (pc == 16) k_hess_f64<16><<<grid, kHessThreads, 0, st>>>(p, P, u, y, jps, acc);
    else k_hess_f64<32><<<grid, kHessThreads, 0, st>>>(p, P, u, y, jps, acc);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ epilogue
__device__ __forceinline__ void hess_epilogue_point(
    const PointsDev& P, int32_t Pn, const double* __restrict__ acc, int n_split, int64_t acc_ld,
    const double* __restrict__ U, const double* __restrict__ W, const double* __restrict__ A,
    const double* __restrict__ B, const double* __restrict__ C, const double* __restrict__ rt_k,
    const double* __restrict__ gt_k, double* __restrict__ f_rho_t, double* __restrict__ f_gamma_t,
    int* err, int t, int64_t p) {
    if (p >= P.nk) return;
    double ar = 0.0, ag = 0.0;
    for (int k = 0; k < n_split; ++k) {
        ar += acc[((static_cast<int64_t>(0) * n_split + k) * Pn + t) * acc_ld + p];
        ag += acc[((static_cast<int64_t>(1) * n_split + k) * Pn + t) * acc_ld + p];
    }
    const double r = P.rho[p];
    const double om_r = P.om_r[p], om_g = P.om_g[p], ka_r = P.ka_r[p];
    const double u = U[p], w = W[p], a = A[p], b = B[p], c = C[p];
    // delta_ij / w_i parts of f^{rho rho}, f^{rho gamma} = f^{gamma rho}, f^{gamma gamma}
    const double d_rr = 2.0 * om_r * w + 2.0 * ka_r * u +
                        r * (P.om_rr[p] * w + P.ka_rr[p] * u + ka_r * ka_r * a +
                             om_r * om_r * c + 2.0 * om_r * ka_r * b);
    const double d_rg = om_g * w + r * P.om_rg[p] * w + r * om_g * ka_r * b + r * om_g * om_r * c;
    const double d_gg = r * (P.om_gg[p] * w + om_g * om_g * c);
    const double rt = rt_k[static_cast<int64_t>(t) * P.nk + p];
    const double gt = gt_k[static_cast<int64_t>(t) * P.nk + p];
    const double fr = ar + d_rr * rt + 2.0 * d_rg * gt;
    const double fg = r * om_g * ag + d_rg * rt + 2.0 * d_gg * gt;
    const int64_t o = static_cast<int64_t>(t) * P.n + P.orig[p];
    f_rho_t[o] = fr;
    f_gamma_t[o] = fg;
    if (!isfinite(fr) || !isfinite(fg)) atomicOr(err, DEVERR_NONFINITE);
}

__global__ void __launch_bounds__(256)
k_hess_epilogue(PointsDev P, int32_t Pn, const double* __restrict__ acc, int n_split,
                int64_t acc_ld, const double* __restrict__ U, const double* __restrict__ W,
                const double* __restrict__ A, const double* __restrict__ B,
                const double* __restrict__ C, const double* __restrict__ rt_k,
                const double* __restrict__ gt_k, double* __restrict__ f_rho_t,
                double* __restrict__ f_gamma_t, int* err) {
    hess_epilogue_point(P, Pn, acc, n_split, acc_ld, U, W, A, B, C, rt_k, gt_k, f_rho_t, f_gamma_t,
                        err, blockIdx.y, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
}

// Block k of molecule m: trial t = k / nb, kept points 256 (k mod nb) .., nb = ceil(nk / 256);
// one split (the tensor-core partials), row sums E..C at sums + k cap.
__global__ void __launch_bounds__(256)
k_hess_epilogue_batch(const EpiMol* __restrict__ mols, const int64_t* __restrict__ pre, int n_mol,
                      double* __restrict__ f_rho_t, double* __restrict__ f_gamma_t, int* err) {
    int64_t blk;
    const EpiMol& M = mols[batch_block_mol(pre, n_mol, blockIdx.x, blk)];
    const int64_t nb = cdiv64(M.P.nk, 256);
    const int t = static_cast<int>(blk / nb);
    const int64_t p = (blk - t * nb) * 256 + threadIdx.x;
    const double* s = M.sums;
    hess_epilogue_point(M.P, M.n_t, M.acc, 1, M.P.nk_pad, s + M.cap, s + 2 * M.cap, s + 3 * M.cap,
                        s + 4 * M.cap, s + 5 * M.cap, M.rt, M.gt, f_rho_t + M.toff,
                        f_gamma_t + M.toff, err, t, p);
}

cudaError_t launch_hess_epilogue_batch(const EpiMol* mols, const int64_t* pre, int n_mol, int64_t n_blocks,
                                       double* f_rho_t, double* f_gamma_t, int* err,
                                       cudaStream_t st) {
    if (n_blocks <= 0) return cudaSuccess;
    k_hess_epilogue_batch<<<static_cast<unsigned>(n_blocks), 256, 0, st>>>(mols, pre, n_mol, f_rho_t,
                                                                           f_gamma_t, err);
    return cudaGetLastError();
}

cudaError_t launch_hess_epilogue(const PointsDev& p, int32_t P, const double* acc, int n_split,
                                 int64_t acc_ld, const double* U, const double* W,
                                 const double* A, const double* B, const double* C,
                                 const double* rt_k, const double* gt_k, double* f_rho_t,
                                 double* f_gamma_t, int* err, cudaStream_t st) {
    if (p.nk == 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>(cdiv64(p.nk, 256)), static_cast<unsigned>(P));
    k_hess_epilogue<<<grid, 256, 0, st>>>(p, P, acc, n_split, acc_ld, U, W, A, B, C, rt_k, gt_k,
                                          f_rho_t, f_gamma_t, err);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Hessian-vector product
// Second derivatives of E along trial directions (Sec. II.B, Eq. frhot with dE/d rho_i =
// w_i f^rho_i and dE/d grad rho_i = 2 w_i f^gamma_i grad rho_i, Sec. II.A):
//   hv_rho[t][i]     = w_i f^{rho,t}_i
//   hv_grad[t][i][c] = 2 w_i (f^{gamma,t}_i d_c rho_i + f^gamma_i d_c rho^t_i),
// f^gamma_i = rho_i omega_gamma,i W_i; kept points only (the caller zeroes the rest).
__global__ void __launch_bounds__(256)
k_hvp_assemble(PointsDev P, int32_t Pn, const double* __restrict__ W,
               const double* __restrict__ f_rho_t, const double* __restrict__ f_gamma_t,
               const double* __restrict__ grad_rho_t, double* __restrict__ hv_rho,
               double* __restrict__ hv_grad) {
    const int t = blockIdx.y;
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= P.nk) return;
    const int64_t i = P.orig[p];
    const int64_t o = static_cast<int64_t>(t) * P.n + i;
    const double w = P.w[p];
    const double fg = P.rho[p] * P.om_g[p] * W[p];
    const double ft = f_gamma_t[o];
    hv_rho[o] = w * f_rho_t[o];
    const double* gt = grad_rho_t + 3 * o;
    hv_grad[3 * o + 0] = 2.0 * w * (ft * P.gx[p] + fg * gt[0]);
    hv_grad[3 * o + 1] = 2.0 * w * (ft * P.gy[p] + fg * gt[1]);
    hv_grad[3 * o + 2] = 2.0 * w * (ft * P.gz[p] + fg * gt[2]);
}

cudaError_t launch_hvp_assemble(const PointsDev& p, int32_t P, const double* W, const double* f_rho_t,
                                const double* f_gamma_t, const double* grad_rho_t, double* hv_rho,
                                double* hv_grad, cudaStream_t st) {
    if (p.nk == 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>(cdiv64(p.nk, 256)), static_cast<unsigned>(P));
    k_hvp_assemble<<<grid, 256, 0, st>>>(p, P, W, f_rho_t, f_gamma_t, grad_rho_t, hv_rho, hv_grad);
    return cudaGetLastError();
}

}  // namespace vv10
