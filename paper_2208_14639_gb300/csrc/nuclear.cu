// The density and weight terms of the VV10 nuclear gradient (Sec. II.A), and the assembly of
// the nine-term nuclear Hessian (Sec. II.B, Eq. E_hess) from the pair sums.
//
// Gradient terms:
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

constexpr int kNhThreads = 256;

// The integrand of the nine-term nuclear Hessian (Sec. II.B, Eq. E_hess) for the direction
// pair (a, b) = (blockIdx.y / P, blockIdx.y % P), summed over a block's range of kept points:
//   E_GG  : w [f^rho rho^{ab} + f^gamma gamma^{ab} + rho^a f^{rho,b} + gamma^a f^{gamma,b}]
//   E_ww  : w^{ab} rho (beta + E) + w^a rho E^{bw}
//   E_wgr : w^a rho E^{b,gr} + (a <-> b)
//   E_Gw  : w^b (f^rho rho^a + f^gamma gamma^a) + w rho^a [E^{bw} + rho (kappa' U^{bw} +
//           omega_rho W^{bw})] + w gamma^a rho omega_gamma W^{bw} + (a <-> b)
//   E_Ggr : w rho^a [E^{b,gr} + rho (kappa' U^{b,gr} + omega_rho W^{b,gr})]
//           + w gamma^a rho omega_gamma W^{b,gr} + (a <-> b)
// with gamma^a = 2 grad rho . grad rho^a and gamma^{ab} = 2 (grad rho^a . grad rho^b +
// grad rho . grad rho^{ab}) (full derivatives of gamma), f^{rho,b}, f^{gamma,b} the Hessian
// contraction with the trial (rho^b, grad rho^b), E the row sums E_i.
__global__ void __launch_bounds__(kNhThreads)
k_nhess_partial(PointsDev P, NucHessIn in, int64_t per_block, double* __restrict__ partial) {
    __shared__ double sh[kNhThreads / 32];
    const int np = in.P;
    const int a = blockIdx.y / np, b = blockIdx.y % np;
    const int64_t n = P.n;
    const int64_t k0 = static_cast<int64_t>(blockIdx.x) * per_block;
    const int64_t k1 = k0 + per_block < P.nk ? k0 + per_block : P.nk;
    const int64_t ab = static_cast<int64_t>(a) * np + b;
    double acc = 0.0;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += kNhThreads) {
        const int64_t i = P.orig[k];
        const double w = P.w[k], rho = P.rho[k];
        const double g0 = P.gx[k], g1 = P.gy[k], g2 = P.gz[k];
        const double kr = P.ka_r[k], omr = P.om_r[k], omg = P.om_g[k];
        const double vr = in.vrho[i], vg = in.vgamma[i];
        const int64_t ia = a * n + i, ib = b * n + i;
        const double* ga = in.grad_rho_a + 3 * ia;
        const double* gb = in.grad_rho_a + 3 * ib;
        const double* gab = in.grad_rho_ab + 3 * (ab * n + i);
        const double ra = in.rho_a[ia], rb = in.rho_a[ib];
        const double gam_a = 2.0 * (g0 * ga[0] + g1 * ga[1] + g2 * ga[2]);
        const double gam_b = 2.0 * (g0 * gb[0] + g1 * gb[1] + g2 * gb[2]);
        const double gam_ab = 2.0 * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2] +
                                     g0 * gab[0] + g1 * gab[1] + g2 * gab[2]);
        const double wa = in.w_a[ia], wb = in.w_a[ib];
        // atom-resolved sums E/U/W^{a,gr}: [3][n][n_atom][3] = [3][n][P]
        const double* egr = in.EUW_gr;
        const int64_t np64 = np;
        const double Ea_gr = egr[i * np64 + a], Ua_gr = egr[(n + i) * np64 + a], Wa_gr = egr[(2 * n + i) * np64 + a];
        const double Eb_gr = egr[i * np64 + b], Ub_gr = egr[(n + i) * np64 + b], Wb_gr = egr[(2 * n + i) * np64 + b];
        double t = w * (vr * in.rho_ab[ab * n + i] + vg * gam_ab + ra * in.f_rho_a[ib] + gam_a * in.f_gamma_a[ib]);
        t += in.w_ab[ab * n + i] * rho * (P.beta + in.sumE[k]) + wa * rho * in.E_w[ib];
        t += rho * (wa * Eb_gr + wb * Ea_gr);
        t += wb * (vr * ra + vg * gam_a) + wa * (vr * rb + vg * gam_b);
        t += w * ra * (in.E_w[ib] + rho * (kr * in.U_w[ib] + omr * in.W_w[ib])) + w * gam_a * rho * omg * in.W_w[ib];
        t += w * rb * (in.E_w[ia] + rho * (kr * in.U_w[ia] + omr * in.W_w[ia])) + w * gam_b * rho * omg * in.W_w[ia];
        t += w * ra * (Eb_gr + rho * (kr * Ub_gr + omr * Wb_gr)) + w * gam_a * rho * omg * Wb_gr;
        t += w * rb * (Ea_gr + rho * (kr * Ua_gr + omr * Wa_gr)) + w * gam_b * rho * omg * Wa_gr;
        acc += t;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x] = acc;
}

// H[a][b] = the block partials in order (compensated) + E^{AB}_{gr,gr}[A][B][c][d] for
// a = 3 A + c, b = 3 B + d.
__global__ void k_nhess_sum(const double* __restrict__ partial, int nblk, int32_t n_atom,
                            const double* __restrict__ Hgg, double* __restrict__ H) {
    const int np = 3 * n_atom;
    const int ab = blockIdx.x * blockDim.x + threadIdx.x;
    if (ab >= np * np) return;
    const int a = ab / np, b = ab % np;
    double s = 0.0, c = 0.0;
    for (int k = 0; k < nblk; ++k) {
        const double x = partial[static_cast<int64_t>(ab) * nblk + k];
        const double t = s + x;
        c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    const int A = a / 3, ca = a % 3, B = b / 3, cb = b % 3;
    H[ab] = s + c + Hgg[((static_cast<int64_t>(A) * n_atom + B) * 3 + ca) * 3 + cb];
}

}  // namespace

int nhess_blocks(int64_t nk) {
    const int64_t b = (nk + 8 * kNhThreads - 1) / (8 * kNhThreads);
    return static_cast<int>(b < 1 ? 1 : (b > 64 ? 64 : b));
}

cudaError_t launch_nuclear_hessian(const PointsDev& p, const NucHessIn& in, const double* Hgg,
                                   double* partial, double* H, cudaStream_t st) {
    const int np = in.P;
    if (np <= 0) return cudaSuccess;
    const int nblk = nhess_blocks(p.nk);
    if (p.nk > 0) {
        const int64_t per_block = (p.nk + nblk - 1) / nblk;
        k_nhess_partial<<<dim3(nblk, np * np), kNhThreads, 0, st>>>(p, in, per_block, partial);
    } else {
        cudaError_t e = cudaMemsetAsync(partial, 0, sizeof(double) * nblk * np * np, st);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_nhess_sum<<<(np * np + 127) / 128, 128, 0, st>>>(partial, nblk, p.n_atom, Hgg, H);
    return cudaGetLastError();
}

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
