// Host-side launch interface between the VV10 translation units (not part of the ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vv10 {

constexpr int kJTile = 256;  // j records are padded to a multiple of this

// Prepared point block (device memory owned by the handle), kept points only, sorted
// by atom (stable), so that each atom's points form one contiguous segment.
struct PointsDev {
    int64_t n = 0;       // caller's points
    int64_t nk = 0;      // kept points
    int64_t nk_pad = 0;  // nk rounded up to kJTile (padding records have c = 0)
    int32_t n_atom = 0;
    double beta = 0.0;
    const int64_t* orig = nullptr;  // nk: kept -> caller index
    const int64_t* seg = nullptr;   // n_atom + 1 segment starts (kept indexing)
    const int32_t* atom = nullptr;  // nk atom of each kept point (0 if none given)
    // FP64 per kept point
    const double *w, *rho, *gx, *gy, *gz;
    const double *om, *ka, *om_r, *om_g, *ka_r, *om_rr, *om_rg, *om_gg, *ka_rr;
    // packed pair records, nk_pad each
    const double4* r64a;  // x, y, z, -1.5 w rho
    const double4* r64b;  // omega, kappa, rho kappa', rho omega_rho
    const float4* r32a;   // x-cx, y-cy, z-cz, -1.5 w rho   (recentred, FP32)
    const float4* r32b;   // omega, kappa, rho kappa', rho omega_rho
    // Pair-packed FP32 records for two consecutive j (2m, 2m+1), 4 float4 per pair:
    //   {-x0,-x1,-y0,-y1}, {-z0,-z1,om0,om1}, {ka0,ka1,-p0,-p1}, {-q0,-q1,c0,c1}
    // (recentred coordinates; p = rho kappa', q = rho omega_rho, c = -1.5 w rho), nk_pad/2 pairs.
    const float4* r32p;
};

// One molecule of a batch, as the batched per-point kernels read it (a device table, one
// entry per molecule).  A launch over many molecules takes the prefix sums `pre` (n_mol + 1
// entries) of the blocks each molecule's own grid has: block k of the launch plays block
// k - pre[m] of molecule m, pre[m] <= k < pre[m + 1].
struct EpiMol {
    PointsDev P;
    const double* part = nullptr;  // pair-sum partials [q][n_split][nk_pad]
    double* sums = nullptr;        // E, U, W, A, B, C at sums + k cap
    double* eblk = nullptr;        // energy block partials (nblk)
    double* rt = nullptr;          // rho^t, gamma^t at kept points [n_t][nk]
    double* gt = nullptr;
    void* split = nullptr;         // split TF32: four FP32 arrays uh, ul, yh, yl, split_step
                                   // floats apart; split FP16: hi, lo tiles split_step halves apart
    void* f16small = nullptr;      // split FP16: column maxima, factors and y balance
    double* acc = nullptr;         // contraction partials [2][n_t][nk_pad]
    int64_t cap = 0;               // row-sum stride
    int64_t off = 0;               // first caller point
    int64_t toff = 0;              // first trial value in the caller's concatenated arrays
    int64_t split_step = 0;
    int32_t n_split = 1, nblk = 0;  // pair-sum splits; energy blocks
    int32_t n_t = 0, rows = 0;      // trials; rows of each trial split
};
#ifdef __CUDACC__
// Trial values of row t at kept point p: u = w rho^t and y = 2 w sigma gamma^t (zero at padding
// points), and rho^t, gamma^t for the epilogue.
__device__ __forceinline__ void trial_values(const PointsDev& P, const double* __restrict__ rho_t,
                                             const double* __restrict__ grad_rho_t, int t, int64_t p,
                                             double& u, double& y, double& rt, double& gt) {
    const int64_t i = P.orig[p];
    const int64_t src = static_cast<int64_t>(t) * P.n + i;
    rt = rho_t[src];
    const double* g = grad_rho_t + 3 * src;
    gt = P.gx[p] * g[0] + P.gy[p] * g[1] + P.gz[p] * g[2];  // gamma^t
    const double w = P.w[p];
    u = w * rt;
    y = 2.0 * w * (P.rho[p] * P.om_g[p]) * gt;
}

#endif

// SoA field order inside the FP64 per-point arena (each field nk_pad long).
enum SoaField : int {
    F_W = 0, F_RHO, F_GX, F_GY, F_GZ, F_OM, F_KA, F_OMR, F_OMG, F_KAR, F_OMRR, F_OMRG, F_OMGG,
    F_KARR, F_COUNT
};

// ---------------------------------------------------------------- prepare (prepare.cu)
struct PrepareScratch {
    int32_t* hist;      // n_keys * nblk
    int64_t* offs;      // n_keys * nblk
    double* bbox_part;  // nblk * 6
    double* center;     // 3
    int64_t* nk_dev;    // 1
};
int prepare_nblk(int64_t n);
// One molecule of a batched prepare (device table).  Phase 1 (count + scan) reads the caller
// arrays and writes hist / offs / bbox_part / center / nk_dev; phase 2 (scatter + points, once
// nk is known) writes the molecule's point block.
struct PrepMol {
    int64_t n = 0;
    const double *xyz = nullptr, *w = nullptr, *rho = nullptr, *grad = nullptr;
    const int32_t* atom = nullptr;
    int32_t n_atom = 0, n_keys = 0, nblk = 0, pad = 0;
    int32_t* hist = nullptr;
    int64_t* offs = nullptr;      // n_keys nblk offsets, then the segment starts
    double* bbox_part = nullptr;
    double* center = nullptr;
    int64_t* nk_dev = nullptr;
    int64_t nk = 0, nk_pad = 0;
    int64_t *orig = nullptr, *seg = nullptr;
    int32_t* atom_k = nullptr;
    double* soa = nullptr;
    double4 *r64a = nullptr, *r64b = nullptr;
    float4 *r32a = nullptr, *r32b = nullptr, *r32p = nullptr;
};
// Batched prepare: the count blocks (pre: prefix sums of nblk) and one scan CTA per
// molecule; then the scatter blocks (pre_blk) and the point blocks (pre_pts: prefix sums of
// nk_pad / 256).  max_keys: the largest n_keys.
cudaError_t launch_prepare_count_batch(const PrepMol* mols, const int64_t* pre, int n_mol,
                                       int64_t n_blocks, int max_keys, double rho_cut, int* err,
                                       cudaStream_t st);
cudaError_t launch_prepare_scatter_batch(const PrepMol* mols, const int64_t* pre_blk,
                                         const int64_t* pre_pts, int n_mol, int64_t n_blocks,
                                         int64_t n_point_blocks, int max_keys, double rho_cut,
                                         double b, double C, cudaStream_t st);
cudaError_t launch_prepare_count(int64_t n, const double* xyz, const double* w, const double* rho,
                                 const double* grad, const int32_t* atom, int32_t n_atom,
                                 double rho_cut, const PrepareScratch& s, int* err,
                                 cudaStream_t st);
cudaError_t launch_prepare_scatter(int64_t n, const double* xyz, const double* w,
                                   const double* rho, const double* grad, const int32_t* atom,
                                   int32_t n_atom, double rho_cut, double b, double C,
                                   const PrepareScratch& s, int64_t nk, int64_t nk_pad,
                                   int64_t* orig, int64_t* seg, int32_t* atom_k, double* soa,
                                   double4* r64a, double4* r64b, float4* r32a, float4* r32b,
                                   float4* r32p, cudaStream_t st);

// Precisions the library knows (vv10_precision values); every mixed one runs the pair sums
// in FP32 and differs only in the Hessian contraction's tensor-core operands.
constexpr bool precision_known(int prec) { return prec >= 0 && prec <= 4; }
// FP64 pair arithmetic and sums (VV10_FP64 and VV10_FP64_TC, which differ in the
// Hessian contraction only).
constexpr bool precision_fp64(int prec) { return prec == 0 || prec == 4; }

// ---------------------------------------------------------------- pair sums (pairsum.cu)
enum PairMode : int { MODE_EUW = 0, MODE_ABC = 1, MODE_GRAD = 2, MODE_EUWABC = 3, MODE_EUWABCG = 4 };
constexpr int kPairModes = 5;
// Quantities a mode accumulates per row (the leading dimension of its partial buffer).
constexpr int pair_mode_nq(int mode) { return mode == MODE_EUWABCG ? 9 : (mode == MODE_EUWABC ? 6 : 3); }

struct PairLaunch {
    int rows_per_thread = 2;  // FP32: 1, 2, 4; FP64: 1, 2
    int n_split = 1;          // j-splits (partials reduced by the epilogue)
    int stall = 0;            // test hook: CTA (0,0) issues no copies, so its waits time out
};
// part: [nq][n_split][nk_pad] FP64 partial sums (quantity-major, nq = pair_mode_nq(mode)),
// n_split = pairsum_split_count(nk_pad, cfg.n_split), the number of splits the launch uses.
int pairsum_split_count(int64_t nk_pad, int requested_split);
cudaError_t launch_pairsum(const PointsDev& p, int mode, bool fp64, const PairLaunch& cfg,
                           double* part, int* err, cudaStream_t st);
int pairsum_default_split(const PointsDev& p, int mode, bool fp64, int rows_per_thread, int n_sm);

// Batched pair sums (batch.cu): one persistent launch over a task table with an atomic
// work counter.  PairMol describes one molecule's records and partial buffer
// part[nq][n_split][nk_pad]; PairTask one (molecule, row tile, j-split) unit.
struct PairMol {
    const void* ra32;
    const void* rb32;
    const void* ra64;
    const void* rb64;
    int64_t nk, nk_pad, j_per_split;
    int32_t n_split, pad;
    double* part;
};
struct PairTask {
    int32_t mol, row_tile, split, pad;
};
cudaError_t launch_pairsum_batch(const PairMol* mols, const PairTask* tasks, int n_tasks,
                                 int* counter, int mode, bool fp64, int rows_per_thread, int n_sm,
                                 int* err, cudaStream_t st);
int pairsum_rows_per_cta(bool fp64, int rows_per_thread);

// Energy / potential epilogue: reduces the partials, writes E,U,W (kept indexing),
// f^rho, f^gamma (caller indexing) and per-block energy partials.
int ep_epilogue_blocks(int64_t nk);
cudaError_t launch_ep_epilogue(const PointsDev& p, const double* part, int n_split, double* E,
                               double* U, double* W, double* vrho, double* vgamma,
                               double* eblk, int* err, cudaStream_t st);
cudaError_t launch_sum_blocks(const double* eblk, int nblk, double* out, cudaStream_t st);
cudaError_t launch_abc_epilogue(const PointsDev& p, const double* part, int n_split, double* A,
                                double* B, double* C, cudaStream_t st);
// Batched forms over a molecule table `mols` (device) and block prefix sums `pre` (device,
// n_mol + 1 entries, pre[n_mol] blocks in all): the energy/potential epilogue (blocks of 256 kept points; vrho/vgamma at the
// molecule's caller offset, may be NULL), the A/B/C epilogue (partials from quantity 3 of
// each molecule's buffer), the energy block sums (one block per molecule, into energies[m]).
cudaError_t launch_ep_epilogue_batch(const EpiMol* mols, const int64_t* pre, int n_mol, int64_t n_blocks,
                                     double* vrho, double* vgamma, int* err, cudaStream_t st);
cudaError_t launch_abc_epilogue_batch(const EpiMol* mols, const int64_t* pre, int n_mol, int64_t n_blocks,
                                      cudaStream_t st);
cudaError_t launch_sum_blocks_batch(const EpiMol* mols, int n_mol, double* energies,
                                    cudaStream_t st);
cudaError_t launch_weight_grad(const PointsDev& p, const double* E, double* dEdw,
                               cudaStream_t st);

// ---------------------------------------------------------------- Hessian (hess.cu)
// Trial inputs at kept points: u = w rho^t, y = 2 w sigma gamma^t (sigma = rho omega_gamma)
// as FP64 [P][nk_pad] (j contiguous), and rho^t, gamma^t (FP64 [P][nk]) for the diagonal.
cudaError_t launch_trial_prep(const PointsDev& p, int32_t P, const double* rho_t,
                              const double* grad_rho_t, double* u, double* y, double* rt_k,
                              double* gt_k, cudaStream_t st);
// Split u, y (FP64 [P][nk_pad]) into TF32 hi and FP32 lo parts, FP32 [Prows][nk_pad];
// rows t >= P are zero.
cudaError_t launch_trial_split(const double* u, const double* y, int32_t P, int32_t Prows,
                               int64_t nk_pad, bool bf16, float* uh, float* ul, float* yh,
                               float* yl, cudaStream_t st);
// Batched split-FP16 trial preparation (hess_f16.cu): rho^t, gamma^t and every trial's column
// maxima (blocks of nk_pad / 256 x n_t per molecule, pre_max; the f16 areas' maxima zeroed by
// the caller), the factors (one CTA per molecule), the FP16 hi / lo tiles (blocks of
// nk_pad / 256 x rows, pre_split).
cudaError_t launch_f16_trial_batch(const EpiMol* mols, const int64_t* pre_max,
                                   const int64_t* pre_split, int n_mol, int64_t n_max_blocks,
                                   int64_t n_split_blocks, const double* rho_t,
                                   const double* grad_rho_t, cudaStream_t st);
// Batched trial preparation fused with the split-TF32 cut (the results of launch_trial_prep
// followed by launch_trial_split, without the FP64 u, y in between): block k of molecule m
// covers points 256 (k mod nb) .. of row t = k / nb of its splits, nb = nk_pad / 256.
cudaError_t launch_trial_tc_batch(const EpiMol* mols, const int64_t* pre, int n_mol, int64_t n_blocks,
                                  const double* rho_t, const double* grad_rho_t, cudaStream_t st);

// Tensor-core (split-TF32) contraction of trials [t0, t0 + Pn), Pn <= 192, into the FP64
// partial output acc [2][acc_P][nk_pad] (zeroed by the caller).  uh/ul/yh/yl: FP32
// [rows][nk_pad] hi/lo parts of u and y; `flush` = stages between FP64 flushes.
int hess_tc_ppad(int32_t P);
cudaError_t launch_hess_tc(const PointsDev& p, int32_t Pn, int32_t t0, int64_t acc_P,
                           const float* uh, const float* ul, const float* yh, const float* yl,
                           int64_t rows, int n_sm, int flush, double* acc, int* err,
                           cudaStream_t st);

// Tensor-core split-FP16 contraction (hess_f16.cu).  chunk_bytes: trial-tile bytes of one j
// chunk (0: the default, hess_f16_default_chunk_bytes(), 24 MB).  launch_f16_trial_split turns u, y
// (FP64 [P][nk_pad]) into scaled FP16 hi / lo tiles [rows][2 nk_pad] (per stage of 16 j: 16 u
// then 16 y), the global y balance factor (params[0] = 1/c_y, params[1] = c_y) and per-trial
// factors (scale[t] = s_t, col_isc[t] = 1/s_t; colmax: 2 P scratch words).  launch_hess_f16
// contracts the trials [t0, t0 + Pn), Pn <= 192, into acc [2][acc_P][nk_pad] (zeroed by the
// caller), already multiplied by 1/s_t.
cudaError_t launch_f16_trial_split(const double* u, const double* y, int32_t P, int32_t rows,
                                   int64_t nk_pad, unsigned int* colmax, float* params,
                                   float* scale, double* col_isc, void* bh, void* bl,
                                   cudaStream_t st);
int hess_f16_kinds_per_tile(int ppad);
size_t hess_f16_default_chunk_bytes();
// Batched split-FP16 contraction over a task table (one launch per padded width): tasks
// (molecule, 128-row tile, kind) largest molecules first, taken from an atomic counter.
size_t hess_f16_mol_bytes();
size_t hess_f16_task_bytes();
bool hess_f16_make_maps(void* out2 /* 2 CUtensorMap */, const void* bh, const void* bl,
                        int64_t nk_pad, int64_t rows, int ppad);
void hess_f16_fill_mol(void* dst, const float4* r32a, const float4* r32b, const float4* r32p,
                       const void* maps_dev, double* acc, const double* col_isc,
                       const float* params, int64_t nk, int64_t nk_pad, int64_t acc_P, int32_t Pn,
                       int32_t t0);
void hess_f16_fill_task(void* dst, int32_t mol, int32_t row_tile, int32_t kind);
cudaError_t launch_hess_f16_batch(const void* mols, const void* tasks, int64_t n_tasks, int ppad,
                                  int* counter, int n_sm, int flush, int* err, cudaStream_t st);
cudaError_t launch_hess_f16(const PointsDev& p, int32_t Pn, int32_t t0, int64_t acc_P,
                            const void* bh, const void* bl, int64_t rows, const double* col_isc,
                            const float* params, int n_sm, int flush, size_t chunk_bytes,
                            double* acc, int* err, cudaStream_t st);

// Tensor-core contraction with FP64 accuracy (hess_o64.cu).  launch_o64_prep writes the
// kept points' column records (`rec`, 64 B per point, nk_pad of them), cuts u, y (FP64
// [P][nk_pad]) into hess_o64_slices() FP16 integer slice arrays [rows][2 nk_pad]
// (`slice_stride` halves apart; per 16-j block 16 u' then 16 c_y y', scaled per trial and
// block) with params[0] = 1/c_y, params[1] = c_y (colmax: 2 scratch words), and the factors'
// inverses civ [group][nk_pad / 16][32] for trial groups of pg <= hess_o64_max_group()
// (hess_o64_civ_floats floats).  launch_hess_o64 contracts the trials [t0, t0 + Pn), Pn <= pg,
// with `civ` pointing at their group's block, into acc [2][acc_P][nk_pad] (zeroed by the
// caller).
int hess_o64_max_group();
int hess_o64_slices();
int64_t hess_o64_civ_floats(int32_t P, int32_t pg, int64_t nk_pad);
cudaError_t launch_o64_prep(const PointsDev& p, const double* u, const double* y, int32_t P,
                            int32_t rows, int32_t pg, void* rec, unsigned long long* colmax,
                            double* params, void* slices, int64_t slice_stride, float* civ,
                            cudaStream_t st);
cudaError_t launch_hess_o64(const PointsDev& p, int32_t Pn, int32_t t0, int64_t acc_P,
                            const void* rec, const void* slices, int64_t slice_stride,
                            int64_t rows, const float* civ, const double* params, int n_sm,
                            int flush, double* acc, int* err, cudaStream_t st);

// Batched tensor-core contraction (molecule and task tables in device memory; see
// hess_tc.cu for the record layouts the fill helpers write).
int hess_tc_kinds_per_tile(int ppad);
bool hess_tc_make_maps(void* out4 /* 4 CUtensorMap */, const float* uh, const float* ul,
                       const float* yh, const float* yl, int64_t nk_pad, int64_t rows, int ppad);
cudaError_t launch_hess_tc_batch(const void* mols, const void* tasks, int64_t n_tasks, int ppad,
                                 int n_sm, int flush, int* err, cudaStream_t st);
size_t hess_tc_mol_bytes();
size_t hess_tc_task_bytes();
void hess_tc_fill_mol(void* dst, const float4* r32a, const float4* r32b, const float4* r32p,
                      const void* maps_dev, double* acc, int64_t nk, int64_t nk_pad, int64_t acc_P,
                      int32_t Pn, int32_t t0);
void hess_tc_fill_task(void* dst, int32_t mol, int32_t row_tile, int32_t kind);

struct HessLaunch {
    int trials_per_cta = 16;  // FP64 SIMT: 8, 16, 32
    int n_split = 1;
};
int hess_f64_default_split(const PointsDev& p, int32_t P, int pc, int n_sm);
int hess_f64_trials_per_cta(int32_t P);
// acc: [2][n_split][P][nk_pad] partial sums of the pair part (rho row, gamma row).
cudaError_t launch_hess_f64(const PointsDev& p, int32_t P, const double* u, const double* y,
                            const HessLaunch& cfg, double* acc, int* err, cudaStream_t st);
cudaError_t launch_hess_epilogue(const PointsDev& p, int32_t P, const double* acc, int n_split,
                                 int64_t acc_ld, const double* U, const double* W,
                                 const double* A, const double* B, const double* C,
                                 const double* rt_k, const double* gt_k, double* f_rho_t,
                                 double* f_gamma_t, int* err, cudaStream_t st);
// Hessian-vector product from the contraction (caller order): hv_rho = w f^{rho,t},
// hv_grad = 2 w (f^{gamma,t} grad rho + f^gamma grad rho^t) at kept points.
cudaError_t launch_hvp_assemble(const PointsDev& p, int32_t P, const double* W, const double* f_rho_t,
                                const double* f_gamma_t, const double* grad_rho_t, double* hv_rho,
                                double* hv_grad, cudaStream_t st);
// Batched Hessian epilogue: block k of molecule m covers kept points 256 (k mod nb) .. of
// trial t = k / nb, nb = ceil(nk / 256); outputs at the molecule's trial offset.
cudaError_t launch_hess_epilogue_batch(const EpiMol* mols, const int64_t* pre, int n_mol, int64_t n_blocks,
                                       double* f_rho_t, double* f_gamma_t, int* err,
                                       cudaStream_t st);

// ---------------------------------------------------------------- coordinates (coord.cu)
cudaError_t launch_grad_epilogue(const PointsDev& p, const double* part, int n_split,
                                 double* gk /* nk x 3 kept */, double* grad_points,
                                 cudaStream_t st);
cudaError_t launch_atom_sums(const PointsDev& p, const double* gk, double* grad_atoms,
                             cudaStream_t st);
// out: E/U/W^Bgr; gk (nk x 3, kept order) and grad_points (n x 3, caller order), when not
// null, receive the point gradient dE/dr_i from the same pass; sums, when not null,
// receives the MODE_EUWABC row sums as part[6][1][nk_pad] (one split) from the same pass.
cudaError_t launch_atom_resolved(const PointsDev& p, bool fp64, double* out, double* gk,
                                 double* grad_points, double* sums, int* err, cudaStream_t st);

// Grid-grid block of the nuclear Hessian (Sec. II.B): E (n_atom x n_atom x 3 x 3) receives
// the blocks E^{AB}_{gr,gr}, Dout (n x n_atom x 3 x 3, zeroed beforehand), when not null,
// the D_i^B of the kept rows; without Dout only the atom pairs A < B are evaluated.
// Scratch: off (n_atom + 1 int64), part (coord_hessian_chunk_bound(nk, n_atom) x n_atom x 6
// doubles).  An empty grid gives zero blocks.
int64_t coord_hessian_chunk_bound(int64_t nk, int32_t n_atom);
cudaError_t launch_coord_hessian(const PointsDev& p, bool fp64, int64_t* off, double* part,
                                 double* E, double* Dout, cudaStream_t st);

// Weight-derivative sums (Sec. II.B): yk (Pn x nk_pad) = -3/2 rho_k v_k of the caller's
// directions wt (Pn x n) in kept order; E, U, W (Pn x n, caller order, may be null) receive
// E_i^v, U_i^v, W_i^v for the kept rows (other rows untouched).
cudaError_t launch_weight_dirs(const PointsDev& p, int32_t Pn, const double* wt, double* yk,
                               cudaStream_t st);
cudaError_t launch_weight_response(const PointsDev& p, bool fp64, int32_t Pn, const double* yk,
                                   double* E, double* U, double* W, cudaStream_t st);
// The same sums on tensor cores (mixed precision): directions in groups of at most 64
// (weight_tc_groups), yk split into TF32 hi / FP32 lo arrays of `rows` >= groups x Ppad
// rows (launch_weight_split); E, U, W must be zero on entry (the kernel adds into them).
void weight_tc_groups(int32_t P, int* n_groups, int* ppad);
cudaError_t launch_weight_split(const double* yk, int32_t Pn, int32_t rows, int64_t nk_pad,
                                float* yh, float* yl, cudaStream_t st);
cudaError_t launch_weight_tc(const PointsDev& p, int32_t Pn, const float* yh, const float* yl,
                             int32_t rows, double* E, double* U, double* W, int n_sm, int* err,
                             cudaStream_t st);
// 2-D tensor map over a [rows][nk_pad] FP32 array, box 16 j x ppad rows, 64-byte swizzle.
bool tc_make_map_f32(void* out /* CUtensorMap */, const float* base, int64_t nk_pad, int64_t rows,
                     int ppad);

// Energy alone from the unordered pairs (Sec. II.A): one persistent launch of `grid` CTAs
// (energy_half_grid) writing cta_total[grid], then their fixed-order sum into *energy
// (device).
int energy_half_grid(bool fp64, int n_sm);
cudaError_t launch_energy_half(const PointsDev& p, bool fp64, int grid, double* cta_total,
                               double* energy, cudaStream_t st);

// FP64 C = A B^T (gemm_f64.cu): A M x K, B N x K with k slowest (column k at A + k lda), C
// M x N column-major; the K range split n_split ways (gemm_abt_splits), partials in work
// (n_split x M x N doubles) summed in a fixed order.
int gemm_abt_splits(int M, int N, int64_t K, int n_sm);
cudaError_t launch_gemm_abt(int M, int N, int64_t K, const double* A, int64_t lda, const double* B,
                            int64_t ldb, double* C, int64_t ldc, double* work, int n_split,
                            cudaStream_t st);

// AO-side assembly (Sec. II.A Fock matrix, Sec. II.B contracted orbital Hessian): out[c] =
// M_c + M_c^T, M_c = Phi^T Z_c over the kept points, channels in chunks of `chunk`
// (ao_channels_per_chunk).  Scratch: phik (nk x nbf), Z (chunk x nk x nbf), M (chunk x nbf x
// nbf) and the product's split-K partials (AoGemm: ao_gemm_work_elems doubles).
struct AoGemm {
    double* work;
    size_t work_elems;
    int n_sm;
};
size_t ao_gemm_work_elems(int32_t nbf, int64_t chunk, int n_sm);
int64_t ao_channels_per_chunk(int64_t nk, int32_t nbf, int32_t n_ch, size_t max_bytes);
cudaError_t launch_ao_assemble(const PointsDev& p, const AoGemm& g, int32_t nbf, const double* phi,
                               const double* dphi, int32_t n_ch, const double* s,
                               const double* fg, const double* vg, const double* gt,
                               int64_t chunk, double* phik, double* Z, double* M, double* out,
                               cudaStream_t st);
// Nuclear derivative of the Fock matrix (Sec. II.B) for the 3 n_atom directions a = 3 A + c:
// caller-order inputs (direction arrays [a n + i], grad_rho_a [(a n + i) 3 + d], EUW_gr
// [(q n + i) 3 n_atom + a]); seg = the host copy of the n_atom + 1 kept-point segment starts;
// LR: 4 nk nbf doubles, K2: 2 nbf^2 doubles.
struct FockDerivIn {
    int32_t nbf;
    const double *phi, *dphi, *hphi;  // n x nbf, n x nbf x 3, n x nbf x 3 x 3
    const int32_t* bf_atom;           // nbf
    const double *vrho, *vgamma;      // n
    const double *f_rho_a, *f_gamma_a, *grad_rho_a, *w_a, *E_w, *U_w, *W_w, *EUW_gr;
};
cudaError_t launch_fock_derivative(const PointsDev& p, const AoGemm& g, const FockDerivIn& in,
                                   const int64_t* seg, int64_t chunk, double* phik, double* Z,
                                   double* M, double* LR, double* K2, double* out, cudaStream_t st);

// E^A_G + E^A_w (Sec. II.A) for Pn directions from the cached row sums sE, sU, sW (kept
// order); rt, gt (Pn x n, Pn x n x 3) and wt (Pn x n) in caller order, either pair may be
// null.  partial: Pn x ngrad_blocks(nk) scratch; out: Pn (device).
int ngrad_blocks(int64_t nk);
cudaError_t launch_nuclear_gradient(const PointsDev& p, const double* sE, const double* sU,
                                    const double* sW, int32_t Pn, const double* rt,
                                    const double* gt, const double* wt, double* partial,
                                    double* out, cudaStream_t st);

// Inputs of the nine-term nuclear Hessian assembly (Sec. II.B, Eq. E_hess), P = 3 n_atom
// directions a = 3 A + c, every array in caller point order unless stated:
struct NucHessIn {
    int32_t P;
    const double* rho_a;        // [P][n]     rho^a at the points moving with their atoms
    const double* grad_rho_a;   // [P][n][3]
    const double* rho_ab;       // [P][P][n]  second derivatives
    const double* grad_rho_ab;  // [P][P][n][3]
    const double* w_a;          // [P][n]     weight derivatives
    const double* w_ab;         // [P][P][n]
    const double* f_rho_a;      // [P][n]     Hessian contraction with (rho^a, grad rho^a)
    const double* f_gamma_a;    // [P][n]
    const double* E_w;          // [P][n]     weight-derivative sums along w^a
    const double* U_w;
    const double* W_w;
    const double* EUW_gr;       // [3][n][n_atom][3] atom-resolved sums
    const double* vrho;         // [n] f^rho, f^gamma
    const double* vgamma;
    const double* sumE;         // [nk] row sums E_i (kept order)
};
// H (P x P, device) = the point sums of the integrand + Hgg (E^{AB}_{gr,gr}, n_atom x n_atom x
// 3 x 3); partial: P^2 x nhess_blocks(nk) scratch.
int nhess_blocks(int64_t nk);
cudaError_t launch_nuclear_hessian(const PointsDev& p, const NucHessIn& in, const double* Hgg,
                                   double* partial, double* H, cudaStream_t st);

}  // namespace vv10
