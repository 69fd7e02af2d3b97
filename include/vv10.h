/*
 * vv10.h -- C ABI of a single-GPU (sm_103a) library for the VV10 nonlocal-correlation
 * double grid sum and its analytic derivatives (Liang, Feng, Liu, Head-Gordon,
 * "Analytic second derivatives of VV10-containing functionals", arXiv 2208.14639).
 *
 * Notation follows the paper (Sec. II): for a grid point i, rho_i, grad rho_i,
 * gamma_i = |grad rho_i|^2, weight w_i, position r_i; for a pair, R^2 = |r_i - r_j|^2,
 * g = omega_i R^2 + kappa_i, g' = omega_j R^2 + kappa_j, Phi_ij = -3/(2 g g' (g + g')).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Array arguments are caller-owned DEVICE pointers (e.g. torch CUDA tensors' data_ptr),
 *    C-contiguous, FP64 unless noted; the library never frees or keeps them after the
 *    call returns (it copies what it needs into handle-owned device memory).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    All work is enqueued on it; a call returns once its work is enqueued, except where
 *    it says it synchronises.
 *  - Outputs are written in the caller's original point indexing; points dropped by the
 *    density cutoff (rho_i < rho_cut) get zeros.
 *  - All inner sums over j include j = i (Phi_ii = -3/(4 kappa_i^3)); with that reading
 *    the delta_ij/w_i terms of Sec. II.B are exactly the Hessian of the quadrature energy.
 *  - Errors are reported by return code only; the library never aborts or prints.  A
 *    device-side condition detected asynchronously (a bounded wait that gave up, an
 *    invalid atom index, a non-finite output) is reported by the next call that
 *    synchronises (vv10_energy_potential, vv10_prepare_points, vv10_sync).
 *  - A handle is not thread-safe; use one handle per host thread / stream.
 */
#ifndef VV10_H
#define VV10_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VV10_OK = 0,
    VV10_ERR_INVALID_ARG = 1,  /* bad pointer, size, parameter, or call order            */
    VV10_ERR_CUDA = 2,         /* a CUDA runtime/driver call failed (see vv10_last_error) */
    VV10_ERR_OOM = 3,          /* device allocation failed                                */
    VV10_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up                      */
    VV10_ERR_NONFINITE = 5,    /* a NaN/Inf was produced in an output                     */
    VV10_ERR_UNSUPPORTED = 6   /* valid request outside the library's limits             */
} vv10_status;

typedef enum {
    VV10_FP64 = 0,          /* all pair arithmetic and sums in FP64                          */
    VV10_MIXED_TF32X3 = 1,  /* FP32 pair tiles; Hessian contraction on tensor cores as split
                               TF32 (hi*hi + hi*lo + lo*hi), FP32 accumulate; FP64 point
                               precompute and FP64 cross-tile / final reductions            */
    VV10_MIXED_BF16X3 = 2,  /* as above with split BF16 operands for the contraction; not
                               built for the contraction (UNSUPPORTED there): a two-piece
                               bf16 split keeps ~16 bits, above the 1e-6 tolerance, and a
                               three-piece split costs as many MMAs as split TF32.  Split
                               TF32 or split FP16 stands in for it.                          */
    VV10_MIXED_F16X3 = 3,   /* FP32 pair tiles; Hessian contraction on tensor cores as split
                               FP16 (hi*hi + hi*lo + lo*hi, K = 16 per MMA: half the MMA
                               instructions of split TF32) with FP32 accumulate; every
                               operand scaled by an exact power of two into FP16's range
                               (per trial column; per row and 32-j stage for the kernel
                               tiles); elsewhere as VV10_MIXED_TF32X3                       */
    VV10_FP64_TC = 4        /* as VV10_FP64, except the pair part of the Hessian contraction:
                               kernel tiles generated in FP64 and the trials are cut into five
                               8-bit integer slices each (FP16-exact), whose 15 leading
                               products the tensor cores sum exactly in FP32 (about 40 bits
                               of each tile and trial kept); results agree with VV10_FP64 to
                               ~1e-11 relative in norm, each element to ~1e-10 of its size
                               (the double-FP32 tiles carry ~46 bits).  Single systems only:
                               the batched contraction returns VV10_ERR_UNSUPPORTED.       */
} vv10_precision;

/* VV10 parameters b and C (Sec. II.A) and the density cutoff below which a point is
 * dropped from every sum (the paper does not state one; 1e-10 is used throughout). */
typedef struct {
    double b;
    double C;
    double rho_cut;
} vv10_params;

typedef struct vv10_ctx* vv10_handle;

/* Limits of the library. */
#define VV10_MAX_ATOMS 4096
#define VV10_MAX_TRIALS 4096
#define VV10_MAX_BASIS 4096

/* Create a handle bound to CUDA device `device`.  Allocates no large buffers yet.
 * Errors: INVALID_ARG (h NULL, bad device), CUDA. */
vv10_status vv10_create(vv10_handle* h, int device);

/* Release the handle and every device buffer it owns (synchronises the device's work
 * on those buffers first).  NULL is accepted. */
vv10_status vv10_destroy(vv10_handle h);

/* Static English description of a status code. */
const char* vv10_status_string(vv10_status s);

/* Description of the last error seen on this handle ("" if none). */
const char* vv10_last_error(vv10_handle h);

/* Per-point precompute (Sec. II.A definitions of gamma, omega, kappa and beta, and the
 * derivatives of omega and kappa used by f^rho, f^gamma (Sec. II.A) and by f^{rho rho},
 * f^{gamma rho}, f^{rho gamma}, f^{gamma gamma} (Sec. II.B)), in FP64.
 *   n              number of grid points (>= 1)
 *   xyz            n x 3 point coordinates r_i (bohr)
 *   w              n quadrature weights w_i
 *   rho            n densities rho_i
 *   grad_rho       n x 3 density gradients
 *   atom_of_point  n int32 atom index of each point ("i in A" of Eqs. grad_gr, EiBgr),
 *                  values in [0, n_atom); may be NULL (then n_atom must be 0 and the
 *                  atom outputs of vv10_coord_grad are unavailable)
 *   n_atom         number of atoms, 0 <= n_atom <= VV10_MAX_ATOMS
 *   prm            b > 0, C >= 0, rho_cut > 0
 *   n_kept         host out: number of points with rho >= rho_cut
 * Replaces any previously prepared point set (and invalidates cached sums).  Synchronises
 * `stream` once (to return n_kept).  Errors: INVALID_ARG (null pointer, n < 1, bad
 * params, atom index out of range, non-finite input), UNSUPPORTED (n_atom too large),
 * OOM, CUDA. */
vv10_status vv10_prepare_points(vv10_handle h, int64_t n, const double* xyz, const double* w,
                                const double* rho, const double* grad_rho,
                                const int32_t* atom_of_point, int32_t n_atom, vv10_params prm,
                                int64_t* n_kept, void* stream);

/* Energy and potential (Sec. II.A):
 *   E^VV10 = sum_i w_i rho_i (beta + E_i / 2),       E_i = sum_j w_j rho_j Phi_ij
 *   f^rho_i = beta + E_i + rho_i (kappa'_i U_i + omega_rho,i W_i),
 *   f^gamma_i = rho_i omega_gamma,i W_i,
 * with U_i, W_i the pair sums defined there.  f^rho and f^gamma are per unit weight:
 * dE/d rho_i = w_i f^rho_i and dE/d(grad rho_i) = 2 w_i f^gamma_i grad rho_i.
 *   prec      VV10_FP64 (VV10_FP64_TC computes the same here), or a mixed mode (FP32
 *             pair arithmetic, FP64 sums)
 *   energy    HOST pointer, receives E (may be NULL: then the call does not synchronise)
 *   vrho      n device out, f^rho (may be NULL)
 *   vgamma    n device out, f^gamma (may be NULL)
 * Caches E_i, U_i, W_i in the handle for vv10_hessian_contract / vv10_weight_grad.
 * Errors: INVALID_ARG (no prepared points), OOM, CUDA, TIMEOUT, NONFINITE. */
vv10_status vv10_energy_potential(vv10_handle h, vv10_precision prec, double* energy,
                                  double* vrho, double* vgamma, void* stream);

/* The energy alone (Sec. II.A, the quadrature form of E^VV10), from the unordered pairs:
 *   E = beta sum_i c_i + sum_{i<j} c_i c_j Phi_ij + 1/2 sum_i c_i^2 Phi_ii,   c_i = w_i rho_i,
 * the same E as vv10_energy_potential with half the pair evaluations (Phi_ij = Phi_ji).
 *   prec     VV10_FP64 (VV10_FP64_TC computes the same here), or a mixed mode (FP32
 *            pair arithmetic, FP64 sums)
 *   energy   HOST pointer, receives E (required; the call synchronises `stream`)
 * Leaves the row sums cached by vv10_energy_potential as they were.  The sum is formed in a
 * fixed order: repeated calls give identical results.  Errors: INVALID_ARG, OOM, CUDA. */
vv10_status vv10_energy(vv10_handle h, vv10_precision prec, double* energy, void* stream);

/* Nonlocal response contracted with P trial densities (Sec. II.B, Eq. frhot):
 *   f^{rho,t}_i   = sum_j w_j (f^{rho rho}_ij rho^t_j + 2 f^{rho gamma}_ij gamma^t_j)
 *   f^{gamma,t}_i = sum_j w_j (f^{gamma rho}_ij rho^t_j + 2 f^{gamma gamma}_ij gamma^t_j)
 * with gamma^t_j = grad rho_j . grad rho^t_j (formed here), including the delta_ij/w_i
 * terms built from U_i, W_i, A_i, B_i, C_i.  These are the directional derivatives of
 * f^rho, f^gamma along (rho^t, grad rho^t).
 *   P            number of trials, 1 <= P <= VV10_MAX_TRIALS
 *   rho_t        P x n trial densities (row t contiguous over points)
 *   grad_rho_t   P x n x 3 trial density gradients
 *   f_rho_t      P x n device out
 *   f_gamma_t    P x n device out
 * vv10_energy_potential must have been called on the current point set first (it
 * provides U_i, W_i; an FP64 contraction after a mixed-precision energy call forms them
 * again in FP64); otherwise INVALID_ARG.  Errors: INVALID_ARG, UNSUPPORTED, OOM,
 * CUDA, TIMEOUT. */
vv10_status vv10_hessian_contract(vv10_handle h, vv10_precision prec, int32_t P,
                                  const double* rho_t, const double* grad_rho_t,
                                  double* f_rho_t, double* f_gamma_t, void* stream);

/* Second derivatives of E along P directions (rho^t, grad rho^t) at once: with dE/d rho_i =
 * w_i f^rho_i and dE/d grad rho_i = 2 w_i f^gamma_i grad rho_i (Sec. II.A), their directional
 * derivatives from the contraction above (Sec. II.B, Eq. frhot):
 *   hv_rho[t][i]     = w_i f^{rho,t}_i
 *   hv_grad[t][i][c] = 2 w_i (f^{gamma,t}_i d_c rho_i + f^gamma_i d_c rho^t_i)
 * (a Hessian-vector product of E in the variables (rho, grad rho); zero at dropped points).
 *   P, rho_t, grad_rho_t   as for vv10_hessian_contract
 *   hv_rho     P x n device out;  hv_grad  P x n x 3 device out
 * Uses handle scratch of 2 P n doubles.  Errors: as vv10_hessian_contract. */
vv10_status vv10_hessian_vector_product(vv10_handle h, vv10_precision prec, int32_t P,
                                        const double* rho_t, const double* grad_rho_t,
                                        double* hv_rho, double* hv_grad, void* stream);

/* Grid-position derivative terms (Sec. II.A Eq. grad_gr, first form; Sec. II.B Eq. EiBgr):
 *   grad_points  n x 3 out (may be NULL): dE/dr_i with rho, grad rho and w held fixed,
 *                = -2 w_i rho_i sum_j w_j rho_j Phi_ij D_ij (r_i - r_j),
 *                D_ij = omega_i/g + omega_j/g' + (omega_i + omega_j)/(g + g')
 *   grad_atoms   n_atom x 3 out (may be NULL): E^A_gr = sum_{i in A} dE/dr_i
 *   EUW_Bgr      3 x n x n_atom x 3 out (may be NULL): E_i^{Bgr}, U_i^{Bgr}, W_i^{Bgr};
 *                for i not in B the sums over j in B of Eq. EiBgr and the two that
 *                follow it, for i in B minus the sum over the other atoms
 * Atom outputs need atom_of_point at prepare time (else INVALID_ARG).  Needs no earlier
 * call other than vv10_prepare_points.  Errors: INVALID_ARG, OOM, CUDA, TIMEOUT. */
vv10_status vv10_coord_grad(vv10_handle h, vv10_precision prec, double* grad_points,
                            double* grad_atoms, double* EUW_Bgr, void* stream);

/* Grid-grid block of the nuclear Hessian (Sec. II.B, the E^{AB}_{gr,gr} line of the nuclear
 * second derivative and the D_i^B equation that follows it): for a kept point i and an atom
 * B that does not own it,
 *   D_i^B = -2 sum_{j in B} w_j rho_j Phi_ij [ 2 (D_ij^2 + (omega_i/g)^2 + (omega_j/g')^2
 *           + ((omega_i + omega_j)/(g + g'))^2) (r_j - r_i)(r_j - r_i)^T - D_ij I_3 ],
 * D_ij as for vv10_coord_grad, and
 *   E^{AB}_{gr,gr} = sum_{i in A} w_i rho_i D_i^B (A != B),
 *   E^{AA}_{gr,gr} = -sum_{B != A} E^{AB}_{gr,gr} (translational invariance).
 * This is the second derivative of E with respect to the positions of the grid points
 * (each moving with its atom) with rho, grad rho and w held fixed.
 *   E_grgr     n_atom x n_atom x 3 x 3 device out (may be NULL): block (A, B) row-major
 *   D_points   n x n_atom x 3 x 3 device out (may be NULL): D_i^B in the caller's point
 *              order; zero for B = atom(i) and for points below rho_cut
 *   prec       VV10_FP64 (VV10_FP64_TC computes the same here), or a mixed mode (FP32
 *              pair arithmetic, FP64 sums)
 * Needs atom_of_point at prepare time (else INVALID_ARG) and no earlier call other than
 * vv10_prepare_points.  Holds about 48 n_atom (n / 128 + n_atom) bytes of scratch.  The
 * blocks are summed in a fixed order: repeated calls give identical results.
 * Errors: INVALID_ARG, OOM, CUDA. */
vv10_status vv10_coord_hessian(vv10_handle h, vv10_precision prec, double* E_grgr,
                               double* D_points, void* stream);

/* Weight-derivative sums (Sec. II.B, the sums E_i^{Bw}, U_i^{Bw}, W_i^{Bw} that enter the
 * E^{AB}_{w,w} and E^{AB}_{G,w} blocks of the nuclear Hessian): for P weight directions v
 * (for the nuclear Hessian the 3 N_atom components of w^B = d w / d R_B),
 *   E_i^v =  sum_j v_j rho_j Phi_ij
 *   U_i^v = -sum_j v_j rho_j Phi_ij (1/(g + g') + 1/g)
 *   W_i^v = -sum_j v_j rho_j Phi_ij R^2 (1/(g + g') + 1/g)
 * (the E_i, U_i, W_i of Sec. II.A with v in place of w; j = i included).
 *   P          number of directions, 1 <= P <= VV10_MAX_TRIALS
 *   w_t        P x n device in, direction p of point i at w_t[p n + i] (caller order)
 *   E_t, U_t, W_t   P x n device out, same layout (each may be NULL); zero for points
 *              below rho_cut
 *   prec       VV10_FP64 (VV10_FP64_TC computes the same here), or a mixed mode (FP32
 *              pair arithmetic, FP64 sums)
 * Needs no earlier call other than vv10_prepare_points.  Holds 8 P n_kept bytes of scratch.
 * Errors: INVALID_ARG, UNSUPPORTED (P too large), OOM, CUDA. */
vv10_status vv10_weight_response(vv10_handle h, vv10_precision prec, int32_t P,
                                 const double* w_t, double* E_t, double* U_t, double* W_t,
                                 void* stream);

/* AO-side assembly (Sec. II.A, the VV10 contribution to the Fock matrix; Sec. II.B, the
 * contracted orbital Hessian), from the per-point results of the calls above:
 *   F_mu_nu   = sum_i w_i [f^rho_i phi_mu phi_nu
 *                          + 2 f^gamma_i grad rho_i . (phi_nu grad phi_mu + phi_mu grad phi_nu)]
 *   G^t_mu_nu = sum_i w_i [f^{rho,t}_i phi_mu phi_nu
 *                          + 2 (f^{gamma,t}_i grad rho_i + f^gamma_i grad rho^t_i)
 *                            . (phi_nu grad phi_mu + phi_mu grad phi_nu)]
 * over the points kept at vv10_prepare_points (w and grad rho as prepared), in FP64 (a cuBLAS
 * DGEMM over the points, the trials side by side).  For rho = sum P_mu_nu phi_mu phi_nu, F_mu_nu = dE/dP_mu_nu
 * and G^t = dF along P^t.
 *   nbf          number of basis functions, 1 <= nbf <= VV10_MAX_BASIS
 *   phi          n x nbf device in, phi_mu at point i at phi[i nbf + mu] (caller order)
 *   grad_phi     n x nbf x 3 device in
 *   vrho, vgamma n device in: f^rho, f^gamma from vv10_energy_potential / vv10_evaluate
 *   F            nbf x nbf device out (symmetric)
 *   P            trials, f_rho_t, f_gamma_t (P x n) from vv10_hessian_contract, grad_rho_t
 *                (P x n x 3) its input
 *   G            P x nbf x nbf device out (each symmetric)
 * Scratch: nbf n_kept doubles, and about 1 GB at most for the per-trial operands (trials are
 * taken in chunks).  Errors: INVALID_ARG, UNSUPPORTED (nbf or P too large), OOM, CUDA. */
vv10_status vv10_fock_matrix(vv10_handle h, int32_t nbf, const double* phi, const double* grad_phi,
                             const double* vrho, const double* vgamma, double* F, void* stream);
vv10_status vv10_orbital_hessian(vv10_handle h, int32_t nbf, const double* phi,
                                 const double* grad_phi, int32_t P, const double* f_rho_t,
                                 const double* f_gamma_t, const double* grad_rho_t,
                                 const double* vgamma, double* G, void* stream);

/* The density and weight terms of the VV10 nuclear gradient (Sec. II.A, E^A_G and E^A_w) along
 * P directions p:
 *   out[p] = sum_i w_i (f^rho_i rho^p_i + 2 f^gamma_i grad rho_i . grad rho^p_i)
 *          + sum_i w^p_i rho_i (beta + E_i)
 * with f^rho, f^gamma, E_i from the row sums cached by the last vv10_energy_potential (or
 * vv10_evaluate) call, which must precede (else INVALID_ARG).  For p = (A, c), rho^p and
 * grad rho^p the derivatives of the density at grid points that move with their atoms and
 * w^p the derivatives of the weights, out[3 A + c] plus E^A_gr (vv10_coord_grad's grad_atoms)
 * is the VV10 nuclear gradient.
 *   rho_t, grad_rho_t   P x n and P x n x 3 device in (caller order; both or neither)
 *   w_t                 P x n device in (may be NULL; at least one of the two terms)
 *   out                 P device out
 * Sums over the kept points in a fixed order.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
vv10_status vv10_nuclear_gradient(vv10_handle h, int32_t P, const double* rho_t,
                                  const double* grad_rho_t, const double* w_t, double* out,
                                  void* stream);

/* The nuclear derivative of the VV10 Fock matrix (Sec. II.B, F^A = F^A_G + F^A_gr + F^A_w) along
 * the 3 n_atom directions a = 3 A + c, for grid points and basis functions that move with their
 * atoms, from the per-point results of the calls above (all in caller order, n points):
 *   F^a_mu_nu = sum_i w^a_i [f^rho phi_mu phi_nu + 2 f^gamma grad rho . B_mu_nu]
 *             + sum_i w_i [s^a_i phi_mu phi_nu + 2 t^a_i grad rho . B_mu_nu
 *                          + 2 f^gamma grad rho^a . B_mu_nu]
 *             + sum_i w_i [f^rho d_a(phi_mu phi_nu) + 2 f^gamma grad rho . d_a B_mu_nu]
 * with B_mu_nu = grad(phi_mu phi_nu), s^a = f^{rho,a} + E^{aw} + E^{a,gr} + rho (kappa' (U^{aw} +
 * U^{a,gr}) + omega_rho (W^{aw} + W^{a,gr})), t^a = f^{gamma,a} + rho omega_gamma (W^{aw} +
 * W^{a,gr}) and d_a phi_mu(i) = ([A owns point i] - [A is the centre of mu]) d phi_mu / d x_c.
 * Sums over the points kept at vv10_prepare_points, in FP64 (cuBLAS DGEMMs over the points).
 * Needs atom_of_point at prepare time (n_atom >= 1, else INVALID_ARG).
 *   nbf, phi, grad_phi   as for vv10_fock_matrix
 *   hess_phi             n x nbf x 3 x 3 device in: second derivatives of phi_mu at point i
 *   bf_atom              nbf int32 device in: the atom each basis function is centred on (a
 *                        value outside [0, n_atom) marks a function that moves with no atom)
 *   vrho, vgamma         n device in: f^rho, f^gamma (vv10_energy_potential)
 *   f_rho_a, f_gamma_a   3 n_atom x n device in: vv10_hessian_contract with the trials
 *                        (rho^a, grad rho^a), the density derivatives at the moving points
 *   grad_rho_a           3 n_atom x n x 3 device in: that trial's grad rho^a
 *   w_a                  3 n_atom x n device in: the weight derivatives w^a
 *   E_w, U_w, W_w        3 n_atom x n device in: vv10_weight_response along w^a
 *   EUW_gr               3 x n x n_atom x 3 device in: vv10_coord_grad's atom-resolved sums
 *   FA                   3 n_atom x nbf x nbf device out (each symmetric)
 * Scratch: 5 n_kept nbf + 2 nbf^2 doubles, plus per-direction operands and products of about 1 GB
 * at most (the directions are taken in chunks).  Reads the
 * n_atom + 1 atom segment starts back to the host (the call synchronises the stream and cannot
 * be captured in a CUDA graph).  Errors: INVALID_ARG, UNSUPPORTED (nbf too large), OOM, CUDA. */
vv10_status vv10_fock_derivative(vv10_handle h, int32_t nbf, const double* phi,
                                 const double* grad_phi, const double* hess_phi,
                                 const int32_t* bf_atom, const double* vrho, const double* vgamma,
                                 const double* f_rho_a, const double* f_gamma_a,
                                 const double* grad_rho_a, const double* w_a, const double* E_w,
                                 const double* U_w, const double* W_w, const double* EUW_gr,
                                 double* FA, void* stream);

/* The VV10 nuclear Hessian, all nine terms of Sec. II.B Eq. E_hess, a = 3 A + c:
 *   E^{ab} = E_GG + E_ww + E_grgr + E_Gw + E_Gw^T + E_Ggr + E_Ggr^T + E_wgr + E_wgr^T
 * with, over the kept points,
 *   E_GG  = sum w [f^rho rho^{ab} + f^gamma gamma^{ab} + rho^a f^{rho,b} + gamma^a f^{gamma,b}]
 *   E_ww  = sum w^{ab} rho (beta + E) + sum w^a rho E^{bw},   E_wgr = sum w^a rho E^{b,gr}
 *   E_Gw  = sum w^b (f^rho rho^a + f^gamma gamma^a) + sum w rho^a [E^{bw} + rho (kappa' U^{bw}
 *           + omega_rho W^{bw})] + sum w gamma^a rho omega_gamma W^{bw}
 *   E_Ggr = the same two sums with E/U/W^{b,gr} in place of E/U/W^{bw}
 *   E_grgr = E^{AB}_{gr,gr} (vv10_coord_hessian)
 * gamma^a = 2 grad rho . grad rho^a and gamma^{ab} = 2 (grad rho^a . grad rho^b + grad rho .
 * grad rho^{ab}) are full derivatives.  Every pair sum comes from this library in precision
 * `prec` (the energy call, the Hessian contraction with the trials (rho^a, grad rho^a), the
 * weight-derivative sums along w^a, the atom-resolved sums and the grid-grid blocks), the
 * local derivatives kappa', omega_rho, omega_gamma from the prepared points; the assembly
 * runs in FP64 with per-block partials summed in a fixed order.
 *   rho_a, grad_rho_a     P x n, P x n x 3: the density's nuclear derivatives at the grid
 *                         points moving with their atoms (P = 3 n_atom, caller order)
 *   rho_ab, grad_rho_ab   P x P x n, P x P x n x 3: their second derivatives
 *   w_a, w_ab             P x n, P x P x n: the quadrature weights' derivatives
 *   H                     P x P device out
 * Needs atom_of_point at prepare time.  Replaces the row sums cached by the last energy call
 * with those of `prec`.  Errors: INVALID_ARG, UNSUPPORTED (3 n_atom > VV10_MAX_TRIALS), OOM,
 * CUDA, TIMEOUT. */
vv10_status vv10_nuclear_hessian(vv10_handle h, vv10_precision prec, const double* rho_a,
                                 const double* grad_rho_a, const double* rho_ab,
                                 const double* grad_rho_ab, const double* w_a, const double* w_ab,
                                 double* H, void* stream);

/* dE/dw_i = rho_i (beta + E_i) (the integrand of E^A_w, Sec. II.A) from the E_i cached
 * by the last vv10_energy_potential call.  dEdw: n device out. */
vv10_status vv10_weight_grad(vv10_handle h, double* dEdw, void* stream);

/* Energy and potential for callers that cannot allocate device memory (the paper has no
 * counterpart).  Some callers may not call cudaMalloc at all: a host whose runtime took
 * (nearly) all device memory up front for its own allocator, or a plug-in that is only
 * ever handed buffers and has no allocator to call.  This entry point gives them the same
 * E, f^rho and f^gamma as vv10_energy_potential (same pair-sum kernel) without a handle and
 * without allocating: its scratch is one static device array of about 11 MB that every GPU
 * which loads this library holds until the process exits, which caps n at
 * VV10_NOALLOC_MAX_POINTS.
 *   n                  number of points, 1 <= n <= VV10_NOALLOC_MAX_POINTS
 *   xyz, w, rho, grad_rho   as for vv10_prepare_points (device pointers, FP64)
 *   prm, prec          as for vv10_prepare_points / vv10_energy_potential
 *   energy             DEVICE pointer to one double (out)
 *   vrho, vgamma       n device out, f^rho and f^gamma (may be NULL)
 * It runs on the calling thread's current device and does not synchronise.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current): make that first call before any stream capture.  Every call shares
 * the one array and leaves its contents behind (each call clears what it needs cleared);
 * calls that overlap on the GPU (other streams, other host threads) race on it and must
 * be serialised by the caller.  Points below rho_cut take part in no sum and get zero
 * outputs, as elsewhere.
 * Errors: INVALID_ARG (n < 1, bad pointer or parameter), UNSUPPORTED (n above the
 * maximum), CUDA.  Device-side failures are not returned (the call does not wait for the
 * GPU): a non-finite input value or a bounded wait that gave up makes the call write NaN
 * to *energy and to every vrho / vgamma value, so that no partial result passes as one. */
#define VV10_NOALLOC_MAX_POINTS 32768
vv10_status vv10_energy_potential_noalloc(int64_t n, const double* xyz, const double* w,
                                          const double* rho, const double* grad_rho,
                                          vv10_params prm, vv10_precision prec, double* energy,
                                          double* vrho, double* vgamma, void* stream);

/* ---------------------------------------------------------------- batched molecules
 * Many independent molecules in one call (the paper has no counterpart: it evaluates one
 * system at a time; every quantity below is, per molecule, exactly the one defined for a
 * single system in Sec. II.A and Sec. II.B, and molecules never interact).  The pair sums
 * of all molecules run as one persistent launch over a table of (molecule, row tile,
 * j-split) tasks; the tensor-core contraction as one launch per padded trial width.
 * Molecule m owns the points offsets[m] .. offsets[m+1]-1 of the concatenated arrays.
 *
 * vv10_batch_prepare: like vv10_prepare_points, for n_mol >= 1 molecules.
 *   offsets       HOST int64[n_mol + 1], offsets[0] = 0, strictly increasing (each
 *                 molecule has at least one point); offsets[n_mol] = n_total
 *   xyz, w, rho, grad_rho   device FP64, n_total rows, layouts as for vv10_prepare_points
 *   atom_of_point device int32[n_total] with per-molecule atom indices, or NULL
 *   n_atom        HOST int32[n_mol] (each in [1, VV10_MAX_ATOMS]) or NULL (with
 *                 atom_of_point NULL)
 *   n_kept        HOST int64[n_mol] out: points kept per molecule (rho >= rho_cut)
 * The prepared blocks are owned by the handle and replace any earlier batch; the
 * single-system state of the handle is not touched.  Synchronises `stream` once.
 * Errors: INVALID_ARG, OOM, CUDA, NONFINITE.
 *
 * vv10_batch_energy_potential: E per molecule (energies: DEVICE double[n_mol] out, written
 * on `stream`, not synchronised) and f^rho, f^gamma (device n_total out, caller indexing,
 * may be NULL).  prec as for vv10_energy_potential.  Errors: INVALID_ARG, OOM, CUDA;
 * device-side conditions are reported by the next vv10_sync.
 *
 * vv10_batch_hessian_contract: f^{rho,t}, f^{gamma,t} (Eq. frhot) for P[m] trial densities
 * of molecule m (P: HOST int32[n_mol], each in [1, VV10_MAX_TRIALS]).  rho_t, grad_rho_t,
 * f_rho_t, f_gamma_t are the concatenation over molecules of each molecule's [P[m]][n_m]
 * (and [P[m]][n_m][3]) row-major blocks, molecule 0 first.  prec: VV10_FP64,
 * VV10_MIXED_TF32X3 or VV10_MIXED_F16X3 (VV10_MIXED_BF16X3 and VV10_FP64_TC:
 * UNSUPPORTED).  Needs a preceding
 * vv10_batch_energy_potential.  Not synchronised.  Errors: INVALID_ARG, UNSUPPORTED, OOM,
 * CUDA.
 *
 * vv10_batch_run: vv10_batch_energy_potential followed by vv10_batch_hessian_contract.
 * The first call for a given (prec, P, pointer set) runs eagerly and then records the
 * same launches into a CUDA graph owned by the handle; later calls with the same
 * arguments replay that graph on `stream` (one graph launch, no host work per kernel).
 * The graph reads the argument pointers given at recording time: their contents may
 * change between calls, their addresses may not (other addresses record a new graph).
 * It stays valid until the next vv10_batch_prepare, vv10_set_tiles or vv10_destroy.  Do
 * not call it while `stream` is being captured by the caller.  Errors: as above. */
vv10_status vv10_batch_prepare(vv10_handle h, int32_t n_mol, const int64_t* offsets,
                               const double* xyz, const double* w, const double* rho,
                               const double* grad_rho, const int32_t* atom_of_point,
                               const int32_t* n_atom, vv10_params prm, int64_t* n_kept,
                               void* stream);
vv10_status vv10_batch_energy_potential(vv10_handle h, vv10_precision prec, double* energies,
                                        double* vrho, double* vgamma, void* stream);
vv10_status vv10_batch_hessian_contract(vv10_handle h, vv10_precision prec, const int32_t* P,
                                        const double* rho_t, const double* grad_rho_t,
                                        double* f_rho_t, double* f_gamma_t, void* stream);
vv10_status vv10_batch_run(vv10_handle h, vv10_precision prec, const int32_t* P,
                           const double* rho_t, const double* grad_rho_t, double* energies,
                           double* vrho, double* vgamma, double* f_rho_t, double* f_gamma_t,
                           void* stream);

/* Synchronise `stream` and report any deferred device-side error on this handle. */
vv10_status vv10_sync(vv10_handle h, void* stream);

/* Tile shapes (the paper has no counterpart).  `what` selects a kernel:
 *   0..5  single-system pair sums, mode + 3 * fp64 (mode 0 = energy/potential sums, 1 = the
 *         A/B/C sums of the Hessian diagonal, 2 = coordinate gradient): rows_per_thread in
 *         {1, 2, 4} (FP64: {1, 2}), n_split = number of j-splits (0 = from the SM count);
 *   6, 7  batched pair sums, 6 + fp64: rows_per_thread as above, n_split = j tiles (of 256
 *         points) per split (0 = 32);
 *   8     tensor-core contraction: rows_per_thread = the widest trial group, in [32, 192];
 *         n_split = the split-FP16 contraction's j chunk in MB of trial tiles, in [4, 96]
 *         (0 = 24): the persistent CTAs walk the chunks in order so that a chunk's tiles
 *         stay in L2.  Groups of at most 64 trials produce both outputs from one tile
 *         generation; wider groups issue fewer MMAs per trial.
 * vv10_set_tiles fixes a shape (rows_per_thread = 0: back to automatic, i.e. the autotuner's
 * choice when tuning is enabled, else the default); the autotuner never replaces a fixed
 * shape.  vv10_get_tiles reads the shape in effect (for 8: the width fixed, else the one the
 * last mixed vv10_hessian_contract used; 0 before any).  Errors: INVALID_ARG. */
vv10_status vv10_set_tiles(vv10_handle h, int what, int rows_per_thread, int n_split);
vv10_status vv10_get_tiles(vv10_handle h, int what, int* rows_per_thread, int* n_split);

/* Everything of one evaluation in one call (the quantities of vv10_energy_potential,
 * vv10_hessian_contract and vv10_coord_grad, Sec. II.A and Sec. II.B; the call itself has no
 * counterpart in the paper).  When EUW_Bgr is requested, one pass over the pairs forms the
 * E/U/W and A/B/C row sums, the atom-resolved terms and the point gradient together (the
 * separate calls need two passes); when only grad_points / grad_atoms are, one pass forms
 * the six row sums and the point gradient; otherwise it is the energy call (with the A/B/C
 * sums formed in its pass when trials are given) and the contraction.
 *   P            number of trials, 0 <= P <= VV10_MAX_TRIALS (0: no Hessian contraction;
 *                rho_t, grad_rho_t, f_rho_t, f_gamma_t then unused and may be NULL)
 *   energy       HOST double out (may be NULL; when given the call synchronises `stream`)
 *   other arrays as for the three calls; vrho, vgamma, grad_points, grad_atoms, EUW_Bgr
 *                may be NULL (grad_atoms, EUW_Bgr need atom_of_point at prepare time)
 * Leaves the handle as the three calls would (the cached sums serve later calls).
 * Errors: as for the three calls. */
vv10_status vv10_evaluate(vv10_handle h, vv10_precision prec, int32_t P, const double* rho_t,
                          const double* grad_rho_t, double* energy, double* vrho, double* vgamma,
                          double* f_rho_t, double* f_gamma_t, double* grad_points,
                          double* grad_atoms, double* EUW_Bgr, void* stream);

/* Handle options (the paper has no counterpart).
 *   VV10_OPT_FUSE_HESSIAN_SUMS  vv10_energy_potential (and vv10_batch_energy_potential) also
 *       form the A_i, B_i, C_i sums of the Hessian diagonal (Sec. II.B) in the same pass over
 *       the pairs, so that a following vv10_hessian_contract (vv10_batch_hessian_contract)
 *       needs no pass of its own.  Worth it when the Hessian follows; costs about half a pass
 *       extra when it does not.  vv10_batch_run always does this.
 * Errors: INVALID_ARG (unknown flag). */
#define VV10_OPT_FUSE_HESSIAN_SUMS 1
vv10_status vv10_set_options(vv10_handle h, int flags);

/* Autotuner (the paper has no counterpart).  Times every candidate shape of a kernel (see
 * vv10_set_tiles) on the handle's prepared data, on `stream`, and applies the fastest:
 *   VV10_TUNE_PAIRSUMS     the three pair-sum modes of the prepared single system (for prec:
 *                          rows per thread x {default, half, twice} the j-splits);
 *   VV10_TUNE_BATCH        the batched pair sums of the prepared batch (for prec: rows per
 *                          thread x {16, 32, 64} j tiles per split);
 *   VV10_TUNE_CONTRACTION  the widest trial group of the mixed contraction (64, 96, 128,
 *                          192; only for P > 64), timed on the real trials.
 * Choices are cached for the process, keyed by kernel, mode, precision, N bucket
 * (ceil(log2 N_kept); for a batch that of its largest molecule and of its total), trial
 * count (contraction) and SM count, so a later handle with a same-keyed workload reuses them
 * without timing.  vv10_autotune(h, prec, what, stream) tunes VV10_TUNE_PAIRSUMS and / or
 * VV10_TUNE_BATCH now (synchronises the stream; INVALID_ARG while the stream is captured).
 * vv10_set_autotune(h, flags) makes the handle tune on first use of each key instead: the
 * pair sums on the first call that runs them, the batched pair sums on the first
 * vv10_batch_energy_potential / vv10_batch_run, the contraction width on the first mixed
 * vv10_hessian_contract for a trial count (the batched contraction uses the cached width
 * of each molecule's key, else 192).  Nothing is timed while a stream is being captured.
 * Tuning runs are not counted by vv10_profile_read.  Errors: INVALID_ARG, OOM, CUDA. */
#define VV10_TUNE_PAIRSUMS 1
#define VV10_TUNE_BATCH 2
#define VV10_TUNE_CONTRACTION 4
vv10_status vv10_autotune(vv10_handle h, vv10_precision prec, int what, void* stream);
vv10_status vv10_set_autotune(vv10_handle h, int flags);

/* Launch accounting and per-phase GPU timing (the paper has no counterpart).
 * vv10_profile_enable(h, 1): from now on every kernel launch of this handle is bracketed
 * by CUDA events recorded on the call's stream; launches are always counted.
 * vv10_profile_read synchronises the device, writes for phases 0..n-1 (n <= VV10_N_PHASES)
 * the accumulated milliseconds (ms, may be NULL; 0 when timing was off) and launch counts
 * (launches, may be NULL), then resets both.  Phase names: vv10_profile_phase_name. */
#define VV10_N_PHASES 16
vv10_status vv10_profile_enable(vv10_handle h, int on);
vv10_status vv10_profile_read(vv10_handle h, int n, double* ms, int64_t* launches);
const char* vv10_profile_phase_name(int phase);

/* Failure-injection hooks for tests (the paper has no counterpart).
 *   VV10_DEBUG_FAIL_ALLOC  value k > 0: the k-th device allocation from now fails (OOM)
 *   VV10_DEBUG_STALL_COPY  value 1: in the next pair-sum launch one CTA never issues its
 *                          tile copies, so its bounded wait gives up after about one
 *                          second and the call that synchronises returns TIMEOUT.
 * Errors: INVALID_ARG. */
#define VV10_DEBUG_FAIL_ALLOC 1
#define VV10_DEBUG_STALL_COPY 2
vv10_status vv10_debug_inject(vv10_handle h, int what, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* VV10_H */
