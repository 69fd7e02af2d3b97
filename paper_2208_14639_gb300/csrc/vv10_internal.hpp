// Definition of the opaque handle behind vv10_handle (host side, not part of the ABI).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

#include "kernels.hpp"
#include "vv10.h"

namespace vv10 {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct TileChoice {
    int rows_per_thread = 2;
    int n_split = 0;  // 0 = derive from the SM count
};

struct TileOverride {
    bool active = false;
    bool manual = false;  // set by vv10_set_tiles (the autotuner never replaces it)
    int mode = 0;
    bool fp64 = false;
    int rows_per_thread = 0;
    int n_split = 0;      // single system: j-splits (0 = from the SM count); batch: j tiles per split
    int bucket = -1;      // tuned entries: the N bucket they were chosen for
};

// Process-wide cache of tuned choices (autotune.cu).
enum TuneKind : int { TUNE_PAIRSUM = 0, TUNE_BATCH = 1, TUNE_TC_CAP = 2 };
int n_bucket(int64_t n);
bool tune_cache_get(int kind, int mode, int fp64, int nbucket, int pbucket, int n_sm, int* v0,
                    int* v1);
void tune_cache_put(int kind, int mode, int fp64, int nbucket, int pbucket, int n_sm, int v0,
                    int v1);
bool stream_capturing(cudaStream_t st);

enum Phase : int {
    PH_PREPARE = 0, PH_PAIR_EUW, PH_EP_EPILOGUE, PH_PAIR_ABC, PH_TRIAL_PREP, PH_CONTRACT_F64,
    PH_CONTRACT_TC, PH_HESS_EPILOGUE, PH_PAIR_GRAD, PH_GRAD_EPILOGUE, PH_ATOM_RESOLVED,
    PH_COORD_HESSIAN, PH_WEIGHT_RESPONSE, PH_ENERGY_HALF, PH_AO_ASSEMBLY,
    PH_NUCLEAR_GRADIENT, PH_COUNT
};

struct ProfRec {
    int phase;
    cudaEvent_t a, b;
};

// One molecule of a batch (byte offsets into the batch's device arenas).
struct BatchMol {
    int64_t off = 0, n = 0, nk = 0, nk_pad = 0, cap = 0;
    int32_t n_atom = 0;
    PointsDev P;
    size_t sums = 0;             // E, U, W, A, B, C (6 x cap doubles)
    int n_split = 1;             // pair-sum j-splits of the current task table
    int64_t j_per_split = 0;
    size_t part = 0;             // pair-sum partials [3][n_split][nk_pad]
    size_t eblk = 0;             // energy block partials
    int nblk = 0;
    int32_t n_t = 0;             // trials of the current Hessian layout
    int64_t toff = 0;            // first trial value in the caller's concatenated arrays
    int ng = 1, pg = 0, ppad = 0;  // tensor-core groups of <= 192 trials, padded group width
    int64_t rows = 0;            // rows of each trial split ((ng - 1) pg + ppad)
    size_t rt = 0, gt = 0;       // rho^t, gamma^t at kept points (n_t x nk doubles each)
    size_t split = 0;            // four FP32 [rows][nk_pad] trial splits (split TF32), or the
                                 // FP16 hi / lo tiles [rows][2 nk_pad] (split FP16)
    size_t f16small = 0;         // split FP16: column maxima, factors, y balance
    size_t acc = 0;              // FP64 [2][n_t][nk_pad] contraction partials
};

struct TcClass {
    int ppad = 0;
    int64_t n_tasks = 0;
    size_t mols = 0, tasks = 0;  // byte offsets in tc_tab
};

struct BatchState {
    std::vector<BatchMol> mol;
    std::vector<int> order;      // molecules, largest first
    int64_t n_total = 0;
    bool prepared = false, have_euw = false, have_abc = false, abc_fp64 = false;
    DevBuf scratch, small, arena, sums, part, eblk, pair_tab, counter;
    void* h_small = nullptr;
    size_t h_small_bytes = 0;
    int pair_tab_fp64 = -1, pair_tab_rpt = 0, pair_tab_split_tiles = 0, n_pair_tasks = 0;
    size_t pair_mols = 0, pair_tasks = 0;
    // Hessian layout (valid for hess_P)
    std::vector<int32_t> hess_P;
    DevBuf rtgt, splits, acc, maps, tc_tab;
    std::vector<TcClass> tc_classes;
    DevBuf f16small, f16tab, f16counter;  // split-FP16 layout (shares rtgt, splits, acc, maps)
    // batched per-point kernels: molecule table and block prefix sums (energy / A,B,C
    // epilogues; trial values + split TF32; Hessian epilogue); hess parts valid with tc_classes
    DevBuf epi, prep_tab;
    size_t epi_pre_ep = 0, epi_pre_tr = 0, epi_pre_mx = 0, epi_pre_hs = 0;
    int64_t epi_n_ep = 0, epi_n_tr = 0, epi_n_mx = 0, epi_n_hs = 0;
    std::vector<TcClass> f16_classes;
    // graph of a whole batched pass, and what it was captured for
    cudaGraphExec_t graph = nullptr;
    std::vector<const void*> graph_key;
    int graph_prec = -1;
    std::vector<int32_t> graph_P;
    int64_t graph_launches[PH_COUNT] = {0};  // kernel launches (by phase) in one replay
};

}  // namespace vv10

struct vv10_ctx {
    int device = 0;
    int n_sm = 0;
    int cc_major = 0, cc_minor = 0;
    char last_error[512] = {0};
    void* h_pinned = nullptr;  // small pinned host scratch for scalar read-backs

    // device error word (DEVERR_* bits)
    vv10::DevBuf dev_err;

    // prepare scratch
    vv10::DevBuf prep_hist, prep_offs, prep_bbox, prep_small;
    // prepared point block
    vv10::DevBuf orig, seg, atom_k, soa, r64a, r64b, r32a, r32b, r32p;
    vv10::PointsDev P;
    int64_t soa_ld = 0;
    vv10_params prm{6.0, 0.01, 1e-10};
    bool prepared = false;

    // cached row sums (kept indexing)
    vv10::DevBuf sumE, sumU, sumW, sumA, sumB, sumC;
    bool have_euw = false, euw_fp64 = false;
    bool have_abc = false, abc_fp64 = false;

    // pair-sum partials and energy reduction scratch
    vv10::DevBuf part, eblk, scal;

    // Hessian scratch
    vv10::DevBuf tu, ty, trt, tgt, hacc;
    vv10::DevBuf tc_uh, tc_ul, tc_yh, tc_yl;
    vv10::DevBuf tc16_bh, tc16_bl;  // split-FP16 trial tiles [rows][2 nk_pad]
    vv10::DevBuf tc16_small;        // their column maxima, factors and y balance
    vv10::DevBuf o64_sl;            // FP64-accurate contraction: FP16 trial slice arrays
    vv10::DevBuf o64_small;         // their factors and y balance
    vv10::DevBuf o64_rec;           // and the points' FP32-pair column records
    vv10::DevBuf hvp_fr, hvp_fg;    // Hessian-vector product: the contraction's outputs

    // coordinate scratch
    vv10::DevBuf gk;
    vv10::DevBuf chpart;  // per-CTA partials of the grid-grid Hessian blocks
    vv10::DevBuf wdir;    // weight directions in kept order (weight-derivative sums)
    vv10::DevBuf wsplit;  // their TF32 hi / FP32 lo split (tensor-core path)
    vv10::DevBuf ehalf;   // per-CTA totals of the energy-only kernel
    vv10::DevBuf aophik, aoz, aom;  // AO assembly: gathered phi, Z, GEMM results
    vv10::DevBuf aogw;              // AO assembly: split-K partials of its FP64 products
    vv10::DevBuf aofa;              // nuclear derivative of F: basis-derivative factors, K^c
    vv10::DevBuf ngpart;            // per-block partials of the nuclear-gradient terms
    vv10::DevBuf nhess;             // nuclear Hessian: its pair sums and block partials

    // tile overrides (index = mode + kPairModes * fp64, modes MODE_EUW..MODE_EUWABCG), set by
    // vv10_set_tiles / the autotuner
    vv10::TileOverride overrides[2 * vv10::kPairModes];
    int options = 0;  // VV10_OPT_* flags
    vv10::TileOverride batch_over[2];  // batched pair sums (index = fp64)
    int tc_cap_manual = 0;             // widest trial group of the contraction (0 = automatic)
    int tc_cap_last = 0;               // the width used by the last mixed Hessian call
    int autotune = 0;                  // VV10_TUNE_* flags: tune on first use

    // stages between FP64 flushes of the tensor-core contraction's register accumulators
    int tc_flush = 512;
    int tc_chunk_mb = 0;            // j-chunk of the split-FP16 contraction (MB of trial tiles; 0 = 24)

    // launch accounting / profiling
    bool prof_on = false;
    int64_t launches[vv10::PH_COUNT] = {0};
    std::vector<vv10::ProfRec> prof;
    std::vector<cudaEvent_t> event_pool;
    cudaEvent_t take_event();
    void phase_begin(int phase, cudaStream_t st, vv10::ProfRec* rec);
    void phase_end(vv10::ProfRec* rec, cudaStream_t st, int n_launch);

    // batched molecules (vv10_batch_*)
    vv10::BatchState batch;
    vv10_status batch_pair_tables(bool fp64, int rpt, int split_tiles);
    void batch_tiles(bool fp64, int* rpt, int* split_tiles) const;
    vv10_status batch_ep(vv10_precision prec, double* energies, double* vrho, double* vgamma,
                         bool with_abc, cudaStream_t st);
    vv10_status batch_hess(vv10_precision prec, const int32_t* P, const double* rho_t,
                           const double* grad_rho_t, double* f_rho_t, double* f_gamma_t,
                           cudaStream_t st);
    vv10_status batch_hess_f16(bool same_P, const int32_t* P, const double* rho_t,
                               const double* grad_rho_t, double* f_rho_t, double* f_gamma_t,
                               cudaStream_t st);
    void batch_release();
    void batch_drop_graph();

    // test hooks
    int debug_fail_alloc = 0;
    int debug_stall = 0;

    void set_error(const char* fmt, ...);
    vv10_status cuda_fail(cudaError_t e, const char* where);
    vv10_status ensure(vv10::DevBuf& b, size_t bytes, const char* what);
    void release_all();
    vv10_status bind();
    vv10_status check_device_errors(cudaStream_t st);
    vv10_status require_prepared();
    vv10::PointsDev points() const;
    vv10::TileChoice tiles_for(int mode, bool fp64) const;
    vv10_status run_pairsum(int mode, bool fp64, cudaStream_t st, int* n_split_out);
    // autotuner (autotune.cu)
    vv10_status tune_pairsum(int mode, bool fp64, cudaStream_t st, bool force);
    vv10_status tune_batch(bool fp64, cudaStream_t st, bool force);
    int tc_cap_for(int32_t P, int64_t nk) const;
    vv10_status tc_contract(int32_t P, int cap, cudaStream_t st);
    vv10_status f16_contract(int32_t P, int cap, cudaStream_t st);
    vv10_status o64_contract(int32_t P, cudaStream_t st);
    vv10_status batch_epi_tables();
    vv10_status tune_tc_cap(int32_t P, cudaStream_t st, int* cap);
    vv10_status hessian(vv10_precision prec, int32_t P, const double* rho_t,
                        const double* grad_rho_t, double* f_rho_t, double* f_gamma_t,
                        cudaStream_t st);
};

namespace vv10 {
// Brackets the kernel launches of one phase: counts them and, when profiling is on,
// records CUDA events around them on the call's stream.
struct PhaseScope {
    vv10_ctx* h;
    cudaStream_t st;
    ProfRec rec;
    int n;
    PhaseScope(vv10_ctx* h_, int phase, cudaStream_t s, int n_launch) : h(h_), st(s), n(n_launch) {
        h->phase_begin(phase, st, &rec);
    }
    ~PhaseScope() { h->phase_end(&rec, st, n); }
};
}  // namespace vv10
