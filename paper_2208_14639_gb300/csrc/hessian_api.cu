// Orchestration of vv10_hessian_contract (Sec. II.B, Eq. frhot): A/B/C row sums for the
// delta_ij/w_i terms, trial preparation, the pair-part contraction and the epilogue.
#include "kernels.hpp"
#include "vv10_internal.hpp"

using namespace vv10;

#define H_CUDA(expr, where)                                  \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);  \
    } while (0)
#define H_TRY(expr)                   \
    do {                              \
        vv10_status s_ = (expr);      \
        if (s_ != VV10_OK) return s_; \
    } while (0)

// Trials per CTA of the FP64 SIMT contraction: minimise chunks * (pair-generation cost +
// 4 FMAs per trial), the FP64 operation count per pair.
int vv10::hess_f64_trials_per_cta(int32_t P) {
    int best = 8;
    long best_cost = -1;
    for (int pc : {8, 16, 32}) {
        const long chunks = (P + pc - 1) / pc;
        const long cost = chunks * (45 + 4L * pc);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = pc;
        }
    }
    return best;
}

vv10_status vv10_ctx::hessian(vv10_precision prec, int32_t Pn, const double* rho_t,
                              const double* grad_rho_t, double* f_rho_t, double* f_gamma_t,
                              cudaStream_t st) {
    const bool fp64 = precision_fp64(prec);
    const size_t out_bytes = sizeof(double) * static_cast<size_t>(Pn) * P.n;
    H_CUDA(cudaMemsetAsync(f_rho_t, 0, out_bytes, st), "memset f_rho_t");
    H_CUDA(cudaMemsetAsync(f_gamma_t, 0, out_bytes, st), "memset f_gamma_t");
    if (P.nk == 0) return VV10_OK;
    if (prec == VV10_MIXED_BF16X3) {
        set_error("the BF16x3 Hessian contraction is not available in this library");
        return VV10_ERR_UNSUPPORTED;
    }

    // U_i, W_i of the diagonal terms in FP64 too when the energy call was mixed
    if (fp64 && !euw_fp64) {
        int ns = 1;
        H_TRY(run_pairsum(MODE_EUW, true, st, &ns));
        PhaseScope ph(this, PH_EP_EPILOGUE, st, 1);
        H_CUDA(launch_ep_epilogue(P, static_cast<double*>(part.p), ns, static_cast<double*>(sumE.p),
                                  static_cast<double*>(sumU.p), static_cast<double*>(sumW.p), nullptr,
                                  nullptr, static_cast<double*>(eblk.p), static_cast<int*>(dev_err.p), st),
               "E/U/W epilogue");
        euw_fp64 = true;
    }
    // A_i, B_i, C_i (pair sums of the diagonal terms), in the requested precision
    const size_t nkb = sizeof(double) * static_cast<size_t>(soa_ld);
    if (!have_abc || (fp64 && !abc_fp64)) {
        H_TRY(ensure(sumA, nkb, "A_i"));
        H_TRY(ensure(sumB, nkb, "B_i"));
        H_TRY(ensure(sumC, nkb, "C_i"));
        int ns = 1;
        H_TRY(run_pairsum(MODE_ABC, fp64, st, &ns));
        PhaseScope ph(this, PH_PAIR_ABC, st, 1);
        H_CUDA(launch_abc_epilogue(P, static_cast<double*>(part.p), ns,
                                   static_cast<double*>(sumA.p), static_cast<double*>(sumB.p),
                                   static_cast<double*>(sumC.p), st),
               "A/B/C epilogue");
        have_abc = true;
        abc_fp64 = fp64;
    }

    // trial inputs at kept points
    const size_t tpad = sizeof(double) * static_cast<size_t>(Pn) * P.nk_pad;
    const size_t tk = sizeof(double) * static_cast<size_t>(Pn) * (P.nk > 0 ? P.nk : 1);
    H_TRY(ensure(tu, tpad, "trial u"));
    H_TRY(ensure(ty, tpad, "trial y"));
    H_TRY(ensure(trt, tk, "trial rho at kept points"));
    H_TRY(ensure(tgt, tk, "trial gamma at kept points"));
    {
    PhaseScope ph(this, PH_TRIAL_PREP, st, 1);
    H_CUDA(launch_trial_prep(P, Pn, rho_t, grad_rho_t, static_cast<double*>(tu.p),
                             static_cast<double*>(ty.p), static_cast<double*>(trt.p),
                             static_cast<double*>(tgt.p), st),
           "trial prep");
    }

    if (!fp64) {
        // tensor-core path: trials in groups of at most `cap` (<= 192, the MMA N of one launch)
        int cap = tc_cap_for(Pn, P.nk);
        if (prec == VV10_MIXED_F16X3) {
            H_TRY(f16_contract(Pn, cap, st));
        } else {
            if (autotune & VV10_TUNE_CONTRACTION) H_TRY(tune_tc_cap(Pn, st, &cap));
            H_TRY(tc_contract(Pn, cap, st));
        }
        tc_cap_last = cap;
        PhaseScope ph2(this, PH_HESS_EPILOGUE, st, 1);
        H_CUDA(launch_hess_epilogue(P, Pn, static_cast<double*>(hacc.p), 1, P.nk_pad,
                                    static_cast<double*>(sumU.p), static_cast<double*>(sumW.p),
                                    static_cast<double*>(sumA.p), static_cast<double*>(sumB.p),
                                    static_cast<double*>(sumC.p), static_cast<double*>(trt.p),
                                    static_cast<double*>(tgt.p), f_rho_t, f_gamma_t,
                                    static_cast<int*>(dev_err.p), st),
               "Hessian epilogue");
        return VV10_OK;
    }

    if (prec == VV10_FP64_TC) {  // FP64 accuracy on the tensor cores (integer slices)
        H_TRY(o64_contract(Pn, st));
        PhaseScope ph2(this, PH_HESS_EPILOGUE, st, 1);
        H_CUDA(launch_hess_epilogue(P, Pn, static_cast<double*>(hacc.p), 1, P.nk_pad,
                                    static_cast<double*>(sumU.p), static_cast<double*>(sumW.p),
                                    static_cast<double*>(sumA.p), static_cast<double*>(sumB.p),
                                    static_cast<double*>(sumC.p), static_cast<double*>(trt.p),
                                    static_cast<double*>(tgt.p), f_rho_t, f_gamma_t,
                                    static_cast<int*>(dev_err.p), st),
               "Hessian epilogue");
        return VV10_OK;
    }
    HessLaunch cfg;
    cfg.trials_per_cta = hess_f64_trials_per_cta(Pn);
    cfg.n_split = hess_f64_default_split(P, Pn, cfg.trials_per_cta, n_sm);
    H_TRY(ensure(hacc, sizeof(double) * 2 * static_cast<size_t>(cfg.n_split) * Pn * P.nk_pad,
                 "contraction partials"));
    {
        PhaseScope ph(this, PH_CONTRACT_F64, st, 1);
        H_CUDA(launch_hess_f64(P, Pn, static_cast<double*>(tu.p), static_cast<double*>(ty.p), cfg,
                               static_cast<double*>(hacc.p), static_cast<int*>(dev_err.p), st),
               "FP64 contraction");
    }
    PhaseScope ph2(this, PH_HESS_EPILOGUE, st, 1);
    H_CUDA(launch_hess_epilogue(P, Pn, static_cast<double*>(hacc.p), cfg.n_split, P.nk_pad,
                                static_cast<double*>(sumU.p), static_cast<double*>(sumW.p),
                                static_cast<double*>(sumA.p), static_cast<double*>(sumB.p),
                                static_cast<double*>(sumC.p), static_cast<double*>(trt.p),
                                static_cast<double*>(tgt.p), f_rho_t, f_gamma_t,
                                static_cast<int*>(dev_err.p), st),
           "Hessian epilogue");
    return VV10_OK;
}

// Split u, y (already in tu, ty) and contract all Pn trials on the tensor cores in groups of
// at most `cap` trials into hacc [2][Pn][nk_pad].
vv10_status vv10_ctx::tc_contract(int32_t Pn, int cap, cudaStream_t st) {
    const int ng = (Pn + cap - 1) / cap;
    const int pg = (Pn + ng - 1) / ng;
    const int ppad = hess_tc_ppad(pg);
    const int64_t rows = static_cast<int64_t>(ng - 1) * pg + ppad;
    const size_t sb = sizeof(float) * static_cast<size_t>(rows) * P.nk_pad;
    H_TRY(ensure(tc_uh, sb, "trial u hi"));
    H_TRY(ensure(tc_ul, sb, "trial u lo"));
    H_TRY(ensure(tc_yh, sb, "trial y hi"));
    H_TRY(ensure(tc_yl, sb, "trial y lo"));
    {
        PhaseScope ph(this, PH_TRIAL_PREP, st, 1);
        H_CUDA(launch_trial_split(static_cast<double*>(tu.p), static_cast<double*>(ty.p), Pn,
                                  static_cast<int32_t>(rows), P.nk_pad, false,
                                  static_cast<float*>(tc_uh.p), static_cast<float*>(tc_ul.p),
                                  static_cast<float*>(tc_yh.p), static_cast<float*>(tc_yl.p), st),
               "trial split");
    }
    const size_t ab = sizeof(double) * 2 * static_cast<size_t>(Pn) * P.nk_pad;
    H_TRY(ensure(hacc, ab, "contraction partials"));
    H_CUDA(cudaMemsetAsync(hacc.p, 0, ab, st), "zero contraction partials");
    PhaseScope ph(this, PH_CONTRACT_TC, st, ng);
    for (int g = 0; g < ng; ++g) {
        const int t0 = g * pg;
        const int pn = (Pn - t0 < pg) ? Pn - t0 : pg;
        H_CUDA(launch_hess_tc(P, pn, t0, Pn, static_cast<float*>(tc_uh.p),
                              static_cast<float*>(tc_ul.p), static_cast<float*>(tc_yh.p),
                              static_cast<float*>(tc_yl.p), rows, n_sm, tc_flush,
                              static_cast<double*>(hacc.p), static_cast<int*>(dev_err.p), st),
               "tensor-core contraction");
    }
    return VV10_OK;
}

// Split u, y (in tu, ty) into scaled FP16 hi / lo tiles and contract all Pn trials on the
// tensor cores (kind::f16) in groups of at most `cap` trials into hacc [2][Pn][nk_pad].
vv10_status vv10_ctx::f16_contract(int32_t Pn, int cap, cudaStream_t st) {
    const int ng = (Pn + cap - 1) / cap;
    const int pg = (Pn + ng - 1) / ng;
    const int ppad = hess_tc_ppad(pg);
    const int64_t rows = static_cast<int64_t>(ng - 1) * pg + ppad;
    const size_t sb = 2 * sizeof(uint16_t) * static_cast<size_t>(rows) * P.nk_pad;
    H_TRY(ensure(tc16_bh, sb, "FP16 trial tiles (hi)"));
    H_TRY(ensure(tc16_bl, sb, "FP16 trial tiles (lo)"));
    // colmax [2 Pn] words | params [4] floats | scale [Pn] floats | col_isc [Pn] doubles
    const size_t o_par = ((2 * sizeof(unsigned int) * Pn + 15) / 16) * 16;
    const size_t o_sc = o_par + 16;
    const size_t o_isc = ((o_sc + sizeof(float) * Pn + 15) / 16) * 16;
    H_TRY(ensure(tc16_small, o_isc + sizeof(double) * Pn, "FP16 trial factors"));
    char* sm = static_cast<char*>(tc16_small.p);
    float* params = reinterpret_cast<float*>(sm + o_par);
    const double* col_isc = reinterpret_cast<const double*>(sm + o_isc);
    {
        PhaseScope ph(this, PH_TRIAL_PREP, st, 3);
        H_CUDA(launch_f16_trial_split(static_cast<double*>(tu.p), static_cast<double*>(ty.p), Pn,
                                      static_cast<int32_t>(rows), P.nk_pad,
                                      reinterpret_cast<unsigned int*>(sm), params,
                                      reinterpret_cast<float*>(sm + o_sc),
                                      reinterpret_cast<double*>(sm + o_isc), tc16_bh.p, tc16_bl.p, st),
               "FP16 trial split");
    }
    const size_t ab = sizeof(double) * 2 * static_cast<size_t>(Pn) * P.nk_pad;
    H_TRY(ensure(hacc, ab, "contraction partials"));
    H_CUDA(cudaMemsetAsync(hacc.p, 0, ab, st), "zero contraction partials");
    PhaseScope ph(this, PH_CONTRACT_TC, st, ng);
    for (int g = 0; g < ng; ++g) {
        const int t0 = g * pg;
        const int pn = (Pn - t0 < pg) ? Pn - t0 : pg;
        H_CUDA(launch_hess_f16(P, pn, t0, Pn, tc16_bh.p, tc16_bl.p, rows, col_isc, params, n_sm,
                               tc_flush, static_cast<size_t>(tc_chunk_mb) << 20,
                               static_cast<double*>(hacc.p), static_cast<int*>(dev_err.p), st),
               "FP16 tensor-core contraction");
    }
    return VV10_OK;
}

// Cut u, y (in tu, ty) into FP16 integer slices and contract all Pn trials with FP64
// accuracy on the tensor cores, in groups of at most 32 trials, into hacc [2][Pn][nk_pad].
vv10_status vv10_ctx::o64_contract(int32_t Pn, cudaStream_t st) {
    const int cap = hess_o64_max_group();
    const int ng = (Pn + cap - 1) / cap;
    const int pg = (Pn + ng - 1) / ng;
    const int64_t rows = static_cast<int64_t>(ng - 1) * pg + cap;
    const int64_t stride = 2 * static_cast<int64_t>(rows) * P.nk_pad;  // halves per slice array
    H_TRY(ensure(o64_sl, hess_o64_slices() * sizeof(uint16_t) * static_cast<size_t>(stride),
                 "FP64 trial slices"));
    H_TRY(ensure(o64_rec, 64 * static_cast<size_t>(P.nk_pad), "FP32-pair point records"));
    // colmax [2] words | params [2] doubles | civ [ng][nk_pad / 16][32] floats
    const int64_t civ_n = hess_o64_civ_floats(Pn, pg, P.nk_pad);
    H_TRY(ensure(o64_small, 32 + sizeof(float) * static_cast<size_t>(civ_n), "FP64 trial factors"));
    char* sm = static_cast<char*>(o64_small.p);
    double* params = reinterpret_cast<double*>(sm + 16);
    float* civ = reinterpret_cast<float*>(sm + 32);
    {
        PhaseScope ph(this, PH_TRIAL_PREP, st, 5);
        H_CUDA(launch_o64_prep(P, static_cast<double*>(tu.p), static_cast<double*>(ty.p), Pn,
                               static_cast<int32_t>(rows), pg, o64_rec.p,
                               reinterpret_cast<unsigned long long*>(sm), params, o64_sl.p, stride,
                               civ, st),
               "FP64 trial slices");
    }
    const size_t ab = sizeof(double) * 2 * static_cast<size_t>(Pn) * P.nk_pad;
    H_TRY(ensure(hacc, ab, "contraction partials"));
    H_CUDA(cudaMemsetAsync(hacc.p, 0, ab, st), "zero contraction partials");
    const int64_t civ_group = civ_n / ng;
    PhaseScope ph(this, PH_CONTRACT_TC, st, ng);
    for (int g = 0; g < ng; ++g) {
        const int t0 = g * pg;
        const int pn = (Pn - t0 < pg) ? Pn - t0 : pg;
        H_CUDA(launch_hess_o64(P, pn, t0, Pn, o64_rec.p, o64_sl.p, stride, rows, civ + g * civ_group,
                               params, n_sm, tc_flush, static_cast<double*>(hacc.p),
                               static_cast<int*>(dev_err.p), st),
               "FP64 tensor-core contraction");
    }
    return VV10_OK;
}
