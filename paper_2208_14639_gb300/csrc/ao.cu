// AO-side assembly of the VV10 Fock matrix (Sec. II.A) and of the contracted orbital Hessian
// (Sec. II.B):
//   M_mu_nu = sum_i w_i [s_i phi_mu phi_nu + 2 v_i . (phi_nu grad phi_mu + phi_mu grad phi_nu)]
// with (s, v) = (f^rho, f^gamma grad rho) for F and (f^{rho,t}, f^{gamma,t} grad rho +
// f^gamma grad rho^t) for G^t.  With Z_i,mu = w_i (s_i phi_i,mu / 2 + 2 v_i . grad phi_i,mu),
// M = Phi^T Z + Z^T Phi: a plain FP64 GEMM over the kept points (this library's own split-K
// kernel, gemm_f64.cu; the channels of a chunk side by side as the columns of one product),
// then the symmetrisation.
//
// The nuclear derivative of the Fock matrix (Sec. II.B, F^a = F^a_G + F^a_gr + F^a_w, a = 3 A + c)
// regroups the same terms in two parts.  (1) The terms whose basis products are not
// differentiated have the form above with, per kept point and direction,
//   s^a = w [f^{rho,a} + E^{aw} + E^{a,gr} + rho (kappa' (U^{aw} + U^{a,gr})
//            + omega_rho (W^{aw} + W^{a,gr}))] + w^a f^rho
//   v^a = {w [f^{gamma,a} + rho omega_gamma (W^{aw} + W^{a,gr})] + w^a f^gamma} grad rho
//         + w f^gamma grad rho^a.
// (2) The derivative of the basis functions, phi^a_mu(i) = sigma d_c phi_mu(i) with sigma =
// [A owns point i] - [A is the centre of mu]: with alpha_i = w f^rho, b_i = 2 w f^gamma grad rho,
//   X_mu_nu = sum_i sigma [d_c phi_mu (alpha phi_nu + b . grad phi_nu) + (b . grad d_c phi_mu) phi_nu]
//           = K^c(A)_mu_nu - [mu on A] K^c(all)_mu_nu,
//   K^c(S) = sum_{i in S} [d_c phi_mu, b . grad d_c phi_mu] . [alpha phi_nu + b . grad phi_nu, phi_nu]
// and F^a += X + X^T.  K^c over the points of one atom is one GEMM over that atom's contiguous
// range of kept points (the kept order groups the points by atom), the two factors of each
// point side by side as two consecutive columns.
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

// Part (1) of the nuclear derivative: Z[k][a - a0][mu] = s^a phi / 2 + 2 v^a . grad phi for the
// directions a0 .. a0 + gridDim.y - 1 (direction arrays: [a n + i], EUW_gr [(q n + i) P + a]).
__global__ void k_fa_z(PointsDev P, FockDerivIn in, int32_t a0, double* __restrict__ Z) {
    const int nbf = in.nbf;
    const int a = a0 + static_cast<int>(blockIdx.y);
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= P.nk * nbf) return;
    const int64_t k = e / nbf;
    const int mu = static_cast<int>(e % nbf);
    const int64_t i = P.orig[k];
    const int64_t ia = static_cast<int64_t>(a) * P.n + i;
    const int64_t np = static_cast<int64_t>(3) * P.n_atom;
    const double w = P.w[k], rho = P.rho[k];
    const double egr = in.EUW_gr[i * np + a];
    const double ugr = in.EUW_gr[(P.n + i) * np + a];
    const double wgr = in.EUW_gr[(2 * P.n + i) * np + a];
    const double uu = in.U_w[ia] + ugr, ww = in.W_w[ia] + wgr;
    const double fr = in.vrho[i], fg = in.vgamma[i], wa = in.w_a[ia];
    const double s = w * (in.f_rho_a[ia] + in.E_w[ia] + egr + rho * (P.ka_r[k] * uu + P.om_r[k] * ww)) +
                     wa * fr;
    const double tg = w * (in.f_gamma_a[ia] + rho * P.om_g[k] * ww) + wa * fg;
    const double* ga = in.grad_rho_a + 3 * ia;
    const double vx = tg * P.gx[k] + w * fg * ga[0];
    const double vy = tg * P.gy[k] + w * fg * ga[1];
    const double vz = tg * P.gz[k] + w * fg * ga[2];
    const int64_t q = i * nbf + mu;
    const double* d = in.dphi + 3 * q;
    Z[(k * gridDim.y + blockIdx.y) * nbf + mu] =
        0.5 * s * in.phi[q] + 2.0 * (vx * d[0] + vy * d[1] + vz * d[2]);
}

// Right factor of K^c (column-major nbf x 2 nk): column 2k = alpha phi + b . grad phi, column
// 2k + 1 = phi, at kept point k.
__global__ void k_fa_right(PointsDev P, FockDerivIn in, double* __restrict__ R) {
    const int nbf = in.nbf;
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= P.nk * nbf) return;
    const int64_t k = e / nbf;
    const int mu = static_cast<int>(e % nbf);
    const int64_t i = P.orig[k];
    const double w = P.w[k];
    const double al = w * in.vrho[i], bf = 2.0 * w * in.vgamma[i];
    const int64_t q = i * nbf + mu;
    const double* d = in.dphi + 3 * q;
    const double ph = in.phi[q];
    R[2 * k * nbf + mu] = al * ph + bf * (P.gx[k] * d[0] + P.gy[k] * d[1] + P.gz[k] * d[2]);
    R[(2 * k + 1) * nbf + mu] = ph;
}

// Left factor of K^c: column 2k = d_c phi, column 2k + 1 = b . grad d_c phi.
__global__ void k_fa_left(PointsDev P, FockDerivIn in, int c, double* __restrict__ L) {
    const int nbf = in.nbf;
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= P.nk * nbf) return;
    const int64_t k = e / nbf;
    const int mu = static_cast<int>(e % nbf);
    const int64_t i = P.orig[k];
    const double bf = 2.0 * P.w[k] * in.vgamma[i];
    const int64_t q = i * nbf + mu;
    const double* h = in.hphi + 9 * q + 3 * c;
    L[2 * k * nbf + mu] = in.dphi[3 * q + c];
    L[(2 * k + 1) * nbf + mu] = bf * (P.gx[k] * h[0] + P.gy[k] * h[1] + P.gz[k] * h[2]);
}

// out += X + X^T with X = K^c(A) - [mu on A] K^c(all) (column-major; KA null: no kept point on A)
__global__ void k_fa_basis(int32_t nbf, int32_t A, const int32_t* __restrict__ bf_atom,
                           const double* __restrict__ Kall, const double* __restrict__ KA,
                           double* __restrict__ out) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= static_cast<int64_t>(nbf) * nbf) return;
    const int mu = static_cast<int>(e / nbf), nu = static_cast<int>(e % nbf);
    const int64_t mn = mu + static_cast<int64_t>(nu) * nbf, nm = nu + static_cast<int64_t>(mu) * nbf;
    double x = 0.0;
    if (KA) x = KA[mn] + KA[nm];
    if (bf_atom[mu] == A) x -= Kall[mn];
    if (bf_atom[nu] == A) x -= Kall[nm];
    out[e] += x;
}

}  // namespace

// Split-K scratch of the largest product an assembly makes: nbf x (chunk nbf) results per
// split, at most ~4 CTAs per SM of 64 x 64 tiles, and never fewer than 64 splits of the
// nbf x nbf products of the basis-function derivatives.
size_t ao_gemm_work_elems(int32_t nbf, int64_t chunk, int n_sm) {
    const size_t nn = static_cast<size_t>(nbf) * nbf;
    const size_t big = nn * static_cast<size_t>(chunk) * static_cast<size_t>(gemm_abt_splits(nbf, static_cast<int>(chunk * nbf), int64_t(1) << 40, n_sm));
    const size_t small = nn * 64;
    return big > small ? big : small;
}

int64_t ao_channels_per_chunk(int64_t nk, int32_t nbf, int32_t n_ch, size_t max_bytes) {
    const size_t per = sizeof(double) * static_cast<size_t>(nk > 0 ? nk : 1) * static_cast<size_t>(nbf);
    int64_t c = static_cast<int64_t>(max_bytes / per);
    if (c < 1) c = 1;
    return c < n_ch ? c : n_ch;
}

namespace {

// Split count of one product, limited by the split-K scratch (work_elems doubles).
int ao_splits(int M, int N, int64_t K, int n_sm, size_t work_elems) {
    int s = gemm_abt_splits(M, N, K, n_sm);
    const size_t per = static_cast<size_t>(M) * static_cast<size_t>(N);
    const int cap = static_cast<int>(work_elems / (per > 0 ? per : 1));
    return s < cap ? s : (cap > 0 ? cap : 1);
}

// The channel chunks of M = Phi^T Z + Z^T Phi: make_z(c0, nc) launches the kernel that writes Z
// for channels c0 .. c0 + nc - 1; phik holds the gathered basis values.
template <class MakeZ>
cudaError_t assemble_chunks(const PointsDev& p, const AoGemm& g, int32_t nbf, int32_t n_ch,
                            int64_t chunk, const double* phik, double* Z, double* M, double* out,
                            cudaStream_t st, MakeZ make_z) {
    const int64_t nn = static_cast<int64_t>(nbf) * nbf;
    for (int32_t c0 = 0; c0 < n_ch; c0 += static_cast<int32_t>(chunk)) {
        const int32_t nc = static_cast<int32_t>(n_ch - c0 < chunk ? n_ch - c0 : chunk);
        make_z(c0, nc);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        // one product for the chunk: M (column-major nbf x nc nbf) = A B^T with A = phik
        // viewed as nbf x nk and B = Z viewed as (nc nbf) x nk (k slowest in both); column
        // c nbf + nu of M is column nu of M_c
        const int N = nc * nbf;
        e = launch_gemm_abt(nbf, N, p.nk, phik, nbf, Z, N, M, nbf, g.work,
                            ao_splits(nbf, N, p.nk, g.n_sm, g.work_elems), st);
        if (e != cudaSuccess) return e;
        k_ao_sym<<<dim3(static_cast<unsigned>((nn + 255) / 256), static_cast<unsigned>(nc)), 256, 0, st>>>(
            nbf, M, out + c0 * nn);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_ao_assemble(const PointsDev& p, const AoGemm& g, int32_t nbf, const double* phi,
                               const double* dphi, int32_t n_ch, const double* s,
                               const double* fg, const double* vg, const double* gt,
                               int64_t chunk, double* phik, double* Z, double* M, double* out,
                               cudaStream_t st) {
    const int64_t nn = static_cast<int64_t>(nbf) * nbf;
    if (p.nk == 0) return cudaMemsetAsync(out, 0, sizeof(double) * nn * n_ch, st);
    const int64_t ne = p.nk * nbf;
    const unsigned gx = static_cast<unsigned>((ne + 255) / 256);
    k_ao_gather<<<gx, 256, 0, st>>>(p, nbf, phi, phik);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return assemble_chunks(p, g, nbf, n_ch, chunk, phik, Z, M, out, st,
                           [&](int32_t c0, int32_t nc) {
                               k_ao_z<<<dim3(gx, static_cast<unsigned>(nc)), 256, 0, st>>>(
                                   p, nbf, phi, dphi, s, fg, vg, gt, c0, Z);
                           });
}

cudaError_t launch_fock_derivative(const PointsDev& p, const AoGemm& g, const FockDerivIn& in,
                                   const int64_t* seg, int64_t chunk, double* phik, double* Z,
                                   double* M, double* LR, double* K2, double* out, cudaStream_t st) {
    const int32_t nbf = in.nbf;
    const int32_t n_dir = 3 * p.n_atom;
    const int64_t nn = static_cast<int64_t>(nbf) * nbf;
    if (p.nk == 0) return cudaMemsetAsync(out, 0, sizeof(double) * nn * n_dir, st);
    const int64_t ne = p.nk * nbf;
    const unsigned gx = static_cast<unsigned>((ne + 255) / 256);
    const unsigned gn = static_cast<unsigned>((nn + 255) / 256);
    k_ao_gather<<<gx, 256, 0, st>>>(p, nbf, in.phi, phik);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // (1) the terms without derivatives of the basis functions (writes every out[a])
    e = assemble_chunks(p, g, nbf, n_dir, chunk, phik, Z, M, out, st,
                        [&](int32_t a0, int32_t nc) {
                            k_fa_z<<<dim3(gx, static_cast<unsigned>(nc)), 256, 0, st>>>(p, in, a0, Z);
                        });
    if (e != cudaSuccess) return e;
    // (2) the derivatives of the basis functions
    double* R = LR;
    double* L = LR + 2 * ne;
    double* Kall = K2;
    double* KA = K2 + nn;
    k_fa_right<<<gx, 256, 0, st>>>(p, in, R);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int c = 0; c < 3; ++c) {
        k_fa_left<<<gx, 256, 0, st>>>(p, in, c, L);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_gemm_abt(nbf, nbf, 2 * p.nk, L, nbf, R, nbf, Kall, nbf, g.work,
                            ao_splits(nbf, nbf, 2 * p.nk, g.n_sm, g.work_elems), st);
        if (e != cudaSuccess) return e;
        for (int32_t A = 0; A < p.n_atom; ++A) {
            const int64_t s0 = seg[A], na = seg[A + 1] - seg[A];
            if (na > 0) {
                e = launch_gemm_abt(nbf, nbf, 2 * na, L + 2 * s0 * nbf, nbf, R + 2 * s0 * nbf, nbf,
                                    KA, nbf, g.work, ao_splits(nbf, nbf, 2 * na, g.n_sm, g.work_elems), st);
                if (e != cudaSuccess) return e;
            }
            k_fa_basis<<<gn, 256, 0, st>>>(nbf, A, in.bf_atom, Kall, na > 0 ? KA : nullptr,
                                          out + (3 * static_cast<int64_t>(A) + c) * nn);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace vv10
