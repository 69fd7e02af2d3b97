// Batched molecules (vv10_batch_*): many independent molecules per call, each with its own
// grid, density and trial densities, evaluated with one persistent pair-sum launch per
// quantity and one tensor-core launch per trial-count class, and replayable as a CUDA graph.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "kernels.hpp"
#include "vv10_internal.hpp"

using namespace vv10;

namespace {

size_t a256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

template <class T>
T* at(DevBuf& b, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(b.p) + off);
}

// Device-accessible memory of `device` (device or managed), aligned to `align` bytes.
bool dev_ok(const void* p, int device, size_t align = 8) {
    if (!p) return false;
    if (reinterpret_cast<uintptr_t>(p) % align) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == device);
}

}  // namespace

#define B_CUDA(expr, where)                                 \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)
#define B_TRY(expr)                   \
    do {                              \
        vv10_status s_ = (expr);      \
        if (s_ != VV10_OK) return s_; \
    } while (0)

void vv10_ctx::batch_release() {
    batch_drop_graph();
    BatchState& B = batch;
    DevBuf* bufs[] = {&B.scratch, &B.small, &B.arena, &B.sums, &B.part, &B.eblk, &B.pair_tab,
                      &B.counter, &B.rtgt, &B.splits, &B.acc, &B.maps, &B.tc_tab,
                      &B.f16small, &B.f16tab, &B.f16counter, &B.epi, &B.prep_tab};
    for (DevBuf* b : bufs) {
        if (b->p) cudaFree(b->p);
        b->p = nullptr;
        b->bytes = 0;
    }
    if (B.h_small) cudaFreeHost(B.h_small);
    B.h_small = nullptr;
    B.h_small_bytes = 0;
}

// Forget the recorded batch graph (after the device has finished any replay of it).
void vv10_ctx::batch_drop_graph() {
    if (!batch.graph) return;
    cudaDeviceSynchronize();
    cudaGraphExecDestroy(batch.graph);
    batch.graph = nullptr;
    batch.graph_key.clear();
    batch.graph_P.clear();
}

// Rows per thread and j tiles per split of the batched pair sums: vv10_set_tiles, else the
// autotuner's choice, else 2 (FP32) / 1 (FP64) rows per thread and 32 tiles (8,192 j).
void vv10_ctx::batch_tiles(bool fp64, int* rpt, int* split_tiles) const {
    const TileOverride& o = batch_over[fp64 ? 1 : 0];
    *rpt = o.active && o.rows_per_thread > 0 ? o.rows_per_thread : (fp64 ? 1 : 2);
    *split_tiles = o.active && o.n_split > 0 ? o.n_split : 32;
}

// Task table of the batched pair sums: (molecule, row tile, j-split), largest molecule first;
// at most 8 splits per molecule, each of at least `split_tiles` tiles.
vv10_status vv10_ctx::batch_pair_tables(bool fp64, int rpt, int split_tiles) {
    BatchState& B = batch;
    if (B.pair_tab_fp64 == (fp64 ? 1 : 0) && B.pair_tab_rpt == rpt &&
        B.pair_tab_split_tiles == split_tiles)
        return VV10_OK;
    batch_drop_graph();  // the tables (and possibly their buffers) change under it
    const int rows = pairsum_rows_per_cta(fp64, rpt);
    std::vector<PairMol> mols(B.mol.size());
    std::vector<PairTask> tasks;
    size_t part_bytes = 0, eblk_bytes = 0;
    for (size_t m = 0; m < B.mol.size(); ++m) {
        BatchMol& M = B.mol[m];
        const int64_t ntile = M.nk_pad / kJTile;
        int S = static_cast<int>(
            std::min<int64_t>(8, std::max<int64_t>(1, (ntile + split_tiles - 1) / split_tiles)));
        const int64_t tps = ntile > 0 ? (ntile + S - 1) / S : 1;
        S = static_cast<int>(ntile > 0 ? (ntile + tps - 1) / tps : 1);
        M.n_split = S;
        M.j_per_split = tps * kJTile;
        M.part = part_bytes;
        part_bytes += a256(sizeof(double) * pair_mode_nq(MODE_EUWABC) * S * (M.cap));
        M.nblk = ep_epilogue_blocks(M.nk);
        M.eblk = eblk_bytes;
        eblk_bytes += a256(sizeof(double) * M.nblk);
    }
    B_TRY(ensure(B.part, part_bytes, "batch pair-sum partials"));
    B_TRY(ensure(B.eblk, eblk_bytes, "batch energy partials"));
    for (size_t m = 0; m < B.mol.size(); ++m) {
        const BatchMol& M = B.mol[m];
        PairMol& d = mols[m];
        d.ra32 = M.P.r32a;
        d.rb32 = M.P.r32b;
        d.ra64 = M.P.r64a;
        d.rb64 = M.P.r64b;
        d.nk = M.nk;
        d.nk_pad = M.nk_pad;
        d.j_per_split = M.j_per_split;
        d.n_split = M.n_split;
        d.pad = 0;
        d.part = at<double>(B.part, M.part);
    }
    for (int m : B.order) {
        const BatchMol& M = B.mol[m];
        const int64_t rt = (M.nk + rows - 1) / rows;
        for (int64_t r = 0; r < rt; ++r)
            for (int s = 0; s < M.n_split; ++s) tasks.push_back(PairTask{m, static_cast<int32_t>(r), s, 0});
    }
    B.pair_mols = 0;
    B.pair_tasks = a256(sizeof(PairMol) * mols.size());
    B_TRY(ensure(B.pair_tab, B.pair_tasks + sizeof(PairTask) * (tasks.size() + 1), "batch task table"));
    B_TRY(ensure(B.counter, 64, "batch work counter"));
    // table upload happens outside any stream capture (first use of this configuration)
    B_CUDA(cudaMemcpy(at<char>(B.pair_tab, B.pair_mols), mols.data(), sizeof(PairMol) * mols.size(),
                      cudaMemcpyHostToDevice),
           "upload molecule table");
    if (!tasks.empty())
        B_CUDA(cudaMemcpy(at<char>(B.pair_tab, B.pair_tasks), tasks.data(),
                          sizeof(PairTask) * tasks.size(), cudaMemcpyHostToDevice),
               "upload task table");
    B.n_pair_tasks = static_cast<int>(tasks.size());
    B.pair_tab_fp64 = fp64 ? 1 : 0;
    B.pair_tab_rpt = rpt;
    B.pair_tab_split_tiles = split_tiles;
    return batch_epi_tables();
}

// The molecule table of the batched per-point kernels and each launch's block prefix sums
// (rebuilt with the pair-sum tables and with the tensor-core Hessian layout, outside any
// stream capture).
vv10_status vv10_ctx::batch_epi_tables() {
    BatchState& B = batch;
    const int n_mol = static_cast<int>(B.mol.size());
    const bool tc = !B.tc_classes.empty();    // the split-TF32 Hessian layout
    const bool f16 = !B.f16_classes.empty();  // the split-FP16 one (they share the arenas)
    std::vector<EpiMol> t(n_mol);
    std::vector<int64_t> pe(n_mol + 1, 0), pt(n_mol + 1, 0), pm(n_mol + 1, 0), ph(n_mol + 1, 0);
    for (int m = 0; m < n_mol; ++m) {
        const BatchMol& M = B.mol[m];
        EpiMol& e = t[m];
        e.P = M.P;
        e.part = at<double>(B.part, M.part);
        e.sums = at<double>(B.sums, M.sums);
        e.eblk = at<double>(B.eblk, M.eblk);
        e.cap = M.cap;
        e.off = M.off;
        e.n_split = M.n_split;
        e.nblk = M.nblk;
        pe[m + 1] = pe[m] + M.nblk;
        int64_t ntr = 0, nmx = 0, nhs = 0;
        if ((tc || f16) && M.nk > 0) {
            e.rt = at<double>(B.rtgt, M.rt);
            e.gt = at<double>(B.rtgt, M.gt);
            e.split = at<char>(B.splits, M.split);
            e.split_step = tc ? static_cast<int64_t>(a256(sizeof(float) * M.rows * M.nk_pad) / sizeof(float))
                              : static_cast<int64_t>(a256(sizeof(uint16_t) * 2 * M.rows * M.nk_pad) / sizeof(uint16_t));
            if (f16) e.f16small = at<char>(B.f16small, M.f16small);
            e.acc = at<double>(B.acc, M.acc);
            e.toff = M.toff;
            e.n_t = M.n_t;
            e.rows = static_cast<int32_t>(M.rows);
            ntr = (M.nk_pad / 256) * M.rows;
            nmx = f16 ? (M.nk_pad / 256) * M.n_t : 0;
            nhs = ((M.nk + 255) / 256) * M.n_t;
        }
        pt[m + 1] = pt[m] + ntr;
        pm[m + 1] = pm[m] + nmx;
        ph[m + 1] = ph[m] + nhs;
    }
    const size_t pre_bytes = sizeof(int64_t) * (n_mol + 1);
    B.epi_pre_ep = a256(sizeof(EpiMol) * n_mol);
    B.epi_pre_tr = B.epi_pre_ep + a256(pre_bytes);
    B.epi_pre_mx = B.epi_pre_tr + a256(pre_bytes);
    B.epi_pre_hs = B.epi_pre_mx + a256(pre_bytes);
    B_TRY(ensure(B.epi, B.epi_pre_hs + a256(pre_bytes), "batch molecule table"));
    std::vector<unsigned char> buf(B.epi_pre_hs + pre_bytes, 0);
    std::memcpy(buf.data(), t.data(), sizeof(EpiMol) * n_mol);
    std::memcpy(buf.data() + B.epi_pre_ep, pe.data(), pre_bytes);
    std::memcpy(buf.data() + B.epi_pre_tr, pt.data(), pre_bytes);
    std::memcpy(buf.data() + B.epi_pre_mx, pm.data(), pre_bytes);
    std::memcpy(buf.data() + B.epi_pre_hs, ph.data(), pre_bytes);
    B_CUDA(cudaMemcpy(B.epi.p, buf.data(), buf.size(), cudaMemcpyHostToDevice),
           "upload batch molecule table");
    B.epi_n_ep = pe[n_mol];
    B.epi_n_tr = pt[n_mol];
    B.epi_n_mx = pm[n_mol];
    B.epi_n_hs = ph[n_mol];
    return VV10_OK;
}

vv10_status vv10_ctx::batch_ep(vv10_precision prec, double* energies, double* vrho,
                               double* vgamma, bool with_abc, cudaStream_t st) {
    BatchState& B = batch;
    const bool fp64 = precision_fp64(prec);
    if (autotune & VV10_TUNE_BATCH) B_TRY(tune_batch(fp64, st, false));
    int rpt, split_tiles;
    batch_tiles(fp64, &rpt, &split_tiles);
    B_TRY(batch_pair_tables(fp64, rpt, split_tiles));
    if (vrho) B_CUDA(cudaMemsetAsync(vrho, 0, sizeof(double) * B.n_total, st), "memset vrho");
    if (vgamma) B_CUDA(cudaMemsetAsync(vgamma, 0, sizeof(double) * B.n_total, st), "memset vgamma");
    int* err = static_cast<int*>(dev_err.p);
    {
        PhaseScope ph(this, PH_PAIR_EUW, st, 1);
        B_CUDA(launch_pairsum_batch(at<PairMol>(B.pair_tab, B.pair_mols),
                                    at<PairTask>(B.pair_tab, B.pair_tasks), B.n_pair_tasks,
                                    static_cast<int*>(B.counter.p), with_abc ? MODE_EUWABC : MODE_EUW,
                                    fp64, rpt, n_sm, err, st),
               "batched pair sums");
    }
    const int n_mol = static_cast<int>(B.mol.size());
    const EpiMol* mt = at<EpiMol>(B.epi, 0);
    if (with_abc) {  // A_i, B_i, C_i: quantities 3..5 of each molecule's partial buffer
        PhaseScope ph(this, PH_PAIR_ABC, st, 1);
        B_CUDA(launch_abc_epilogue_batch(mt, at<int64_t>(B.epi, B.epi_pre_ep), n_mol, B.epi_n_ep, st),
               "batched A/B/C epilogue");
    }
    PhaseScope ph(this, PH_EP_EPILOGUE, st, 2);
    B_CUDA(launch_ep_epilogue_batch(mt, at<int64_t>(B.epi, B.epi_pre_ep), n_mol, B.epi_n_ep, vrho,
                                    vgamma, err, st),
           "batched energy epilogue");
    B_CUDA(launch_sum_blocks_batch(mt, n_mol, energies, st), "batched energy sums");
    B.have_euw = true;
    B.have_abc = with_abc;
    B.abc_fp64 = fp64;
    return VV10_OK;
}

vv10_status vv10_ctx::batch_hess(vv10_precision prec, const int32_t* Pt, const double* rho_t,
                                 const double* grad_rho_t, double* f_rho_t, double* f_gamma_t,
                                 cudaStream_t st) {
    BatchState& B = batch;
    const bool fp64 = precision_fp64(prec);
    const size_t n_mol = B.mol.size();
    int* err = static_cast<int*>(dev_err.p);
    // trial offsets in the caller's concatenated arrays, and output clearing
    int64_t toff = 0;
    bool same_P = B.hess_P.size() == n_mol;
    for (size_t m = 0; m < n_mol; ++m) {
        same_P = same_P && B.hess_P[m] == Pt[m];
        B.mol[m].n_t = Pt[m];
        B.mol[m].toff = toff;
        toff += static_cast<int64_t>(Pt[m]) * B.mol[m].n;
    }
    B_CUDA(cudaMemsetAsync(f_rho_t, 0, sizeof(double) * toff, st), "memset f_rho_t");
    B_CUDA(cudaMemsetAsync(f_gamma_t, 0, sizeof(double) * toff, st), "memset f_gamma_t");

    // A_i, B_i, C_i of the delta_ij / w_i terms
    if (!B.have_abc || (fp64 && !B.abc_fp64)) {
        int rpt, split_tiles;
        batch_tiles(fp64, &rpt, &split_tiles);
        B_TRY(batch_pair_tables(fp64, rpt, split_tiles));
        {
            PhaseScope ph(this, PH_PAIR_ABC, st, 1);
            B_CUDA(launch_pairsum_batch(at<PairMol>(B.pair_tab, B.pair_mols),
                                        at<PairTask>(B.pair_tab, B.pair_tasks), B.n_pair_tasks,
                                        static_cast<int*>(B.counter.p), MODE_ABC, fp64, rpt, n_sm,
                                        err, st),
                   "batched A/B/C sums");
        }
        // MODE_ABC writes A/B/C as quantities 0..2 of each molecule's partials
        PhaseScope ph(this, PH_PAIR_ABC, st, static_cast<int>(n_mol));
        for (size_t m = 0; m < n_mol; ++m) {
            BatchMol& M = B.mol[m];
            double* s = at<double>(B.sums, M.sums);
            B_CUDA(launch_abc_epilogue(M.P, at<double>(B.part, M.part), M.n_split, s + 3 * M.cap,
                                       s + 4 * M.cap, s + 5 * M.cap, st),
                   "batched A/B/C epilogue");
        }
        B.have_abc = true;
        B.abc_fp64 = fp64;
    }

    if (fp64) {
        // FP64 baseline: the single-system kernels molecule by molecule, on scratch sized
        // once for the largest molecule (nothing is reallocated between launches)
        size_t tpad = 0, tk = 0, hb = 0;
        std::vector<HessLaunch> cfg(n_mol);
        for (size_t m = 0; m < n_mol; ++m) {
            const BatchMol& M = B.mol[m];
            if (M.nk == 0) continue;
            cfg[m].trials_per_cta = hess_f64_trials_per_cta(M.n_t);
            cfg[m].n_split = hess_f64_default_split(M.P, M.n_t, cfg[m].trials_per_cta, n_sm);
            tpad = std::max(tpad, sizeof(double) * static_cast<size_t>(M.n_t) * M.nk_pad);
            tk = std::max(tk, sizeof(double) * static_cast<size_t>(M.n_t) * M.nk);
            hb = std::max(hb, sizeof(double) * 2 * static_cast<size_t>(cfg[m].n_split) * M.n_t * M.nk_pad);
        }
        if (tpad == 0) return VV10_OK;
        B_TRY(ensure(tu, tpad, "trial u"));
        B_TRY(ensure(ty, tpad, "trial y"));
        B_TRY(ensure(trt, tk, "trial rho at kept points"));
        B_TRY(ensure(tgt, tk, "trial gamma at kept points"));
        B_TRY(ensure(hacc, hb, "contraction partials"));
        for (size_t m = 0; m < n_mol; ++m) {
            BatchMol& M = B.mol[m];
            if (M.nk == 0) continue;
            double* s = at<double>(B.sums, M.sums);
            PhaseScope ph(this, PH_CONTRACT_F64, st, 3);
            B_CUDA(launch_trial_prep(M.P, M.n_t, rho_t + M.toff, grad_rho_t + 3 * M.toff,
                                     static_cast<double*>(tu.p), static_cast<double*>(ty.p),
                                     static_cast<double*>(trt.p), static_cast<double*>(tgt.p), st),
                   "trial prep");
            B_CUDA(launch_hess_f64(M.P, M.n_t, static_cast<double*>(tu.p), static_cast<double*>(ty.p),
                                   cfg[m], static_cast<double*>(hacc.p), err, st),
                   "FP64 contraction");
            B_CUDA(launch_hess_epilogue(M.P, M.n_t, static_cast<double*>(hacc.p), cfg[m].n_split,
                                        M.nk_pad, s + M.cap, s + 2 * M.cap, s + 3 * M.cap,
                                        s + 4 * M.cap, s + 5 * M.cap, static_cast<double*>(trt.p),
                                        static_cast<double*>(tgt.p), f_rho_t + M.toff,
                                        f_gamma_t + M.toff, err, st),
                   "Hessian epilogue");
        }
        return VV10_OK;
    }

    if (prec == VV10_MIXED_F16X3) return batch_hess_f16(same_P, Pt, rho_t, grad_rho_t, f_rho_t, f_gamma_t, st);

    // tensor-core path.  Layout (rebuilt when the trial counts change): per molecule the
    // trial values at kept points, four FP32 trial splits of `rows` rows, the FP64 partial
    // output, four tensor maps; per padded group width one molecule-group table and one
    // task table (row tile x output kind), largest molecules first.
    if (!same_P || B.tc_classes.empty()) {
        batch_drop_graph();
        size_t rtgt = 0, split = 0, acc = 0;
        for (size_t m = 0; m < n_mol; ++m) {
            BatchMol& M = B.mol[m];
            const int cap = tc_cap_for(M.n_t, M.nk);
            M.ng = (M.n_t + cap - 1) / cap;
            M.pg = (M.n_t + M.ng - 1) / M.ng;
            M.ppad = hess_tc_ppad(M.pg);
            M.rows = static_cast<int64_t>(M.ng - 1) * M.pg + M.ppad;
            const size_t nk1 = M.nk > 0 ? M.nk : 1;
            M.rt = rtgt;
            rtgt += a256(sizeof(double) * M.n_t * nk1);
            M.gt = rtgt;
            rtgt += a256(sizeof(double) * M.n_t * nk1);
            M.split = split;
            split += 4 * a256(sizeof(float) * M.rows * M.nk_pad);
            M.acc = acc;
            acc += a256(sizeof(double) * 2 * M.n_t * M.nk_pad);
        }
        B_TRY(ensure(B.rtgt, rtgt, "batch trial values"));
        B_TRY(ensure(B.splits, split > 0 ? split : 256, "batch trial splits"));
        B_TRY(ensure(B.acc, acc > 0 ? acc : 256, "batch contraction partials"));
        std::vector<unsigned char> maps(512 * n_mol, 0);
        for (size_t m = 0; m < n_mol; ++m) {
            BatchMol& M = B.mol[m];
            if (M.nk_pad == 0) continue;
            float* sp = at<float>(B.splits, M.split);
            const size_t step = a256(sizeof(float) * M.rows * M.nk_pad) / sizeof(float);
            if (!hess_tc_make_maps(maps.data() + 512 * m, sp, sp + step, sp + 2 * step, sp + 3 * step,
                                   M.nk_pad, M.rows, M.ppad)) {
                set_error("tensor map encoding failed");
                return VV10_ERR_CUDA;
            }
        }
        B_TRY(ensure(B.maps, maps.size(), "batch tensor maps"));
        B_CUDA(cudaMemcpy(B.maps.p, maps.data(), maps.size(), cudaMemcpyHostToDevice),
               "upload tensor maps");
        std::vector<int> widths;
        for (const BatchMol& M : B.mol)
            if (M.nk > 0 && std::find(widths.begin(), widths.end(), M.ppad) == widths.end())
                widths.push_back(M.ppad);
        std::sort(widths.begin(), widths.end());
        std::vector<unsigned char> tab;
        B.tc_classes.clear();
        for (int ppad : widths) {
            TcClass c;
            c.ppad = ppad;
            std::vector<std::pair<int, int>> groups;  // (molecule, group), largest molecules first
            for (int m : B.order)
                if (B.mol[m].ppad == ppad && B.mol[m].nk > 0)
                    for (int g = 0; g < B.mol[m].ng; ++g) groups.push_back({m, g});
            c.mols = a256(tab.size());
            tab.resize(c.mols + hess_tc_mol_bytes() * groups.size());
            for (size_t k = 0; k < groups.size(); ++k) {
                const BatchMol& M = B.mol[groups[k].first];
                const int t0 = groups[k].second * M.pg;
                const int pn = std::min(M.pg, M.n_t - t0);
                hess_tc_fill_mol(tab.data() + c.mols + hess_tc_mol_bytes() * k, M.P.r32a, M.P.r32b,
                                 M.P.r32p, static_cast<char*>(B.maps.p) + 512 * groups[k].first,
                                 at<double>(B.acc, M.acc), M.nk, M.nk_pad, M.n_t, pn, t0);
            }
            const int kinds = hess_tc_kinds_per_tile(ppad) == 2 ? 1 : 2;
            std::vector<unsigned char> tk;
            int64_t nt = 0;
            for (size_t k = 0; k < groups.size(); ++k) {
                const int64_t rt = (B.mol[groups[k].first].nk + 127) / 128;
                for (int64_t r = 0; r < rt; ++r)
                    for (int kind = 0; kind < kinds; ++kind) {
                        tk.resize(tk.size() + hess_tc_task_bytes());
                        hess_tc_fill_task(tk.data() + hess_tc_task_bytes() * nt, static_cast<int32_t>(k),
                                          static_cast<int32_t>(r), kind);
                        ++nt;
                    }
            }
            c.tasks = a256(tab.size());
            tab.resize(c.tasks + tk.size());
            std::memcpy(tab.data() + c.tasks, tk.data(), tk.size());
            c.n_tasks = nt;
            B.tc_classes.push_back(c);
        }
        B_TRY(ensure(B.tc_tab, tab.size() + 256, "batch tensor-core tables"));
        if (!tab.empty())
            B_CUDA(cudaMemcpy(B.tc_tab.p, tab.data(), tab.size(), cudaMemcpyHostToDevice),
                   "upload tensor-core tables");
        B.hess_P.assign(Pt, Pt + n_mol);
        B.f16_classes.clear();  // the split-FP16 layout shares the arenas: rebuild it when used
        B_TRY(batch_epi_tables());
    }

    // trial values and their split-TF32 cut, every molecule in one launch
    const EpiMol* mt = at<EpiMol>(B.epi, 0);
    {
        PhaseScope ph(this, PH_TRIAL_PREP, st, 1);
        B_CUDA(launch_trial_tc_batch(mt, at<int64_t>(B.epi, B.epi_pre_tr), static_cast<int>(n_mol),
                                     B.epi_n_tr, rho_t, grad_rho_t, st),
               "batched trial values and split");
    }
    B_CUDA(cudaMemsetAsync(B.acc.p, 0, B.acc.bytes, st), "zero contraction partials");
    {
        PhaseScope ph(this, PH_CONTRACT_TC, st, static_cast<int>(B.tc_classes.size()));
        for (const TcClass& c : B.tc_classes)
            B_CUDA(launch_hess_tc_batch(static_cast<char*>(B.tc_tab.p) + c.mols,
                                        static_cast<char*>(B.tc_tab.p) + c.tasks, c.n_tasks, c.ppad,
                                        n_sm, tc_flush, err, st),
                   "batched tensor-core contraction");
    }
    PhaseScope ph(this, PH_HESS_EPILOGUE, st, 1);
    B_CUDA(launch_hess_epilogue_batch(mt, at<int64_t>(B.epi, B.epi_pre_hs), static_cast<int>(n_mol),
                                      B.epi_n_hs, f_rho_t, f_gamma_t, err, st),
           "batched Hessian epilogue");
    return VV10_OK;
}

// The split-FP16 contraction of the batch.  Layout (rebuilt when the trial counts change):
// per molecule the trial values at kept points, its FP16 hi / lo trial tiles [rows][2 nk_pad],
// its column factors, the FP64 partial output and two tensor maps; per padded width one
// molecule-group table and one task table (row tile x output kind), largest molecules first,
// taken by the persistent CTAs from an atomic counter.
vv10_status vv10_ctx::batch_hess_f16(bool same_P, const int32_t* Pt, const double* rho_t,
                                     const double* grad_rho_t, double* f_rho_t, double* f_gamma_t,
                                     cudaStream_t st) {
    BatchState& B = batch;
    const size_t n_mol = B.mol.size();
    int* err = static_cast<int*>(dev_err.p);
    if (!same_P || B.f16_classes.empty()) {
        batch_drop_graph();
        size_t rtgt = 0, split = 0, small = 0, acc = 0;
        for (size_t m = 0; m < n_mol; ++m) {
            BatchMol& M = B.mol[m];
            const int cap = tc_cap_for(M.n_t, M.nk);
            M.ng = (M.n_t + cap - 1) / cap;
            M.pg = (M.n_t + M.ng - 1) / M.ng;
            M.ppad = hess_tc_ppad(M.pg);
            M.rows = static_cast<int64_t>(M.ng - 1) * M.pg + M.ppad;
            const size_t nk1 = M.nk > 0 ? M.nk : 1;
            M.rt = rtgt;
            rtgt += a256(sizeof(double) * M.n_t * nk1);
            M.gt = rtgt;
            rtgt += a256(sizeof(double) * M.n_t * nk1);
            M.split = split;  // hi then lo, [rows][2 nk_pad] FP16 each
            split += 2 * a256(sizeof(uint16_t) * 2 * M.rows * M.nk_pad);
            M.f16small = small;  // colmax [2 n_t] | params [4] | scale [n_t] | col_isc [n_t]
            small += a256(sizeof(unsigned int) * 2 * M.n_t) + 256 + a256(sizeof(float) * M.n_t) +
                     a256(sizeof(double) * M.n_t);
            M.acc = acc;
            acc += a256(sizeof(double) * 2 * M.n_t * M.nk_pad);
        }
        B_TRY(ensure(B.rtgt, rtgt, "batch trial values"));
        B_TRY(ensure(B.splits, split > 0 ? split : 256, "batch FP16 trial tiles"));
        B_TRY(ensure(B.f16small, small > 0 ? small : 256, "batch FP16 trial factors"));
        B_TRY(ensure(B.acc, acc > 0 ? acc : 256, "batch contraction partials"));
        std::vector<unsigned char> maps(256 * n_mol, 0);
        for (size_t m = 0; m < n_mol; ++m) {
            BatchMol& M = B.mol[m];
            if (M.nk_pad == 0) continue;
            char* sp = at<char>(B.splits, M.split);
            const size_t half = a256(sizeof(uint16_t) * 2 * M.rows * M.nk_pad);
            if (!hess_f16_make_maps(maps.data() + 256 * m, sp, sp + half, M.nk_pad, M.rows, M.ppad)) {
                set_error("tensor map encoding failed");
                return VV10_ERR_CUDA;
            }
        }
        B_TRY(ensure(B.maps, maps.size(), "batch tensor maps"));
        B_CUDA(cudaMemcpy(B.maps.p, maps.data(), maps.size(), cudaMemcpyHostToDevice),
               "upload tensor maps");
        std::vector<int> widths;
        for (const BatchMol& M : B.mol)
            if (M.nk > 0 && std::find(widths.begin(), widths.end(), M.ppad) == widths.end())
                widths.push_back(M.ppad);
        std::sort(widths.begin(), widths.end());
        std::vector<unsigned char> tab;
        B.f16_classes.clear();
        for (int ppad : widths) {
            TcClass c;
            c.ppad = ppad;
            std::vector<std::pair<int, int>> groups;  // (molecule, group), largest molecules first
            for (int m : B.order)
                if (B.mol[m].ppad == ppad && B.mol[m].nk > 0)
                    for (int g = 0; g < B.mol[m].ng; ++g) groups.push_back({m, g});
            c.mols = a256(tab.size());
            tab.resize(c.mols + hess_f16_mol_bytes() * groups.size());
            for (size_t k = 0; k < groups.size(); ++k) {
                const BatchMol& M = B.mol[groups[k].first];
                const int t0 = groups[k].second * M.pg;
                const int pn = std::min(M.pg, M.n_t - t0);
                char* sm = at<char>(B.f16small, M.f16small);
                const size_t o_par = a256(sizeof(unsigned int) * 2 * M.n_t);
                const size_t o_isc = o_par + 256 + a256(sizeof(float) * M.n_t);
                hess_f16_fill_mol(tab.data() + c.mols + hess_f16_mol_bytes() * k, M.P.r32a, M.P.r32b,
                                  M.P.r32p, static_cast<char*>(B.maps.p) + 256 * groups[k].first,
                                  at<double>(B.acc, M.acc), reinterpret_cast<const double*>(sm + o_isc),
                                  reinterpret_cast<const float*>(sm + o_par), M.nk, M.nk_pad, M.n_t, pn, t0);
            }
            const int kinds = hess_f16_kinds_per_tile(ppad) == 2 ? 1 : 2;
            std::vector<unsigned char> tk;
            int64_t nt = 0;
            for (size_t k = 0; k < groups.size(); ++k) {
                const int64_t rt = (B.mol[groups[k].first].nk + 127) / 128;
                for (int64_t r = 0; r < rt; ++r)
                    for (int kind = 0; kind < kinds; ++kind) {
                        tk.resize(tk.size() + hess_f16_task_bytes());
                        hess_f16_fill_task(tk.data() + hess_f16_task_bytes() * nt, static_cast<int32_t>(k),
                                           static_cast<int32_t>(r), kind);
                        ++nt;
                    }
            }
            c.tasks = a256(tab.size());
            tab.resize(c.tasks + tk.size());
            std::memcpy(tab.data() + c.tasks, tk.data(), tk.size());
            c.n_tasks = nt;
            B.f16_classes.push_back(c);
        }
        B_TRY(ensure(B.f16tab, tab.size() + 256, "batch split-FP16 tables"));
        if (!tab.empty())
            B_CUDA(cudaMemcpy(B.f16tab.p, tab.data(), tab.size(), cudaMemcpyHostToDevice),
                   "upload split-FP16 tables");
        B_TRY(ensure(B.f16counter, 256, "batch task counter"));
        B.hess_P.assign(Pt, Pt + n_mol);
        B.tc_classes.clear();  // the split-TF32 layout shares the arenas: rebuild it when used
        B_TRY(batch_epi_tables());
    }

    // trial values, column maxima, factors and FP16 tiles of every molecule in three launches
    B_CUDA(cudaMemsetAsync(B.f16small.p, 0, B.f16small.bytes, st), "zero trial column maxima");
    {
        PhaseScope ph(this, PH_TRIAL_PREP, st, 3);
        B_CUDA(launch_f16_trial_batch(at<EpiMol>(B.epi, 0), at<int64_t>(B.epi, B.epi_pre_mx),
                                      at<int64_t>(B.epi, B.epi_pre_tr), static_cast<int>(n_mol),
                                      B.epi_n_mx, B.epi_n_tr, rho_t, grad_rho_t, st),
               "batched FP16 trial tiles");
    }
    B_CUDA(cudaMemsetAsync(B.acc.p, 0, B.acc.bytes, st), "zero contraction partials");
    {
        PhaseScope ph(this, PH_CONTRACT_TC, st, 2 * static_cast<int>(B.f16_classes.size()));
        for (const TcClass& c : B.f16_classes)
            B_CUDA(launch_hess_f16_batch(static_cast<char*>(B.f16tab.p) + c.mols,
                                         static_cast<char*>(B.f16tab.p) + c.tasks, c.n_tasks, c.ppad,
                                         static_cast<int*>(B.f16counter.p), n_sm, tc_flush, err, st),
                   "batched split-FP16 contraction");
    }
    PhaseScope ph(this, PH_HESS_EPILOGUE, st, 1);
    B_CUDA(launch_hess_epilogue_batch(at<EpiMol>(B.epi, 0), at<int64_t>(B.epi, B.epi_pre_hs),
                                      static_cast<int>(n_mol), B.epi_n_hs, f_rho_t, f_gamma_t, err, st),
           "batched Hessian epilogue");
    return VV10_OK;
}

// ---------------------------------------------------------------- ABI

extern "C" {

vv10_status vv10_batch_prepare(vv10_handle h, int32_t n_mol, const int64_t* offsets,
                               const double* xyz, const double* w, const double* rho,
                               const double* grad_rho, const int32_t* atom_of_point,
                               const int32_t* n_atom, vv10_params prm, int64_t* n_kept,
                               void* stream) {
    if (!h) return VV10_ERR_INVALID_ARG;
    h->set_error("");
    if (n_mol < 1 || !offsets || !n_kept || offsets[0] != 0) {
        h->set_error("need n_mol >= 1, offsets[0] == 0 and n_kept");
        return VV10_ERR_INVALID_ARG;
    }
    for (int32_t m = 0; m < n_mol; ++m)
        if (offsets[m + 1] <= offsets[m]) {
            h->set_error("every molecule needs at least one point");
            return VV10_ERR_INVALID_ARG;
        }
    if ((atom_of_point == nullptr) != (n_atom == nullptr)) {
        h->set_error("atom_of_point and n_atom must be given together");
        return VV10_ERR_INVALID_ARG;
    }
    if (!(prm.b > 0.0) || !(prm.C >= 0.0) || !(prm.rho_cut > 0.0)) {
        h->set_error("parameters need b > 0, C >= 0, rho_cut > 0");
        return VV10_ERR_INVALID_ARG;
    }
    if (n_atom)
        for (int32_t m = 0; m < n_mol; ++m)
            if (n_atom[m] < 1 || n_atom[m] > VV10_MAX_ATOMS) {
                h->set_error("n_atom of every molecule must be in [1, VV10_MAX_ATOMS]");
                return VV10_ERR_INVALID_ARG;
            }
    vv10_status s = h->bind();
    if (s != VV10_OK) return s;
    const void* ptrs[] = {xyz, w, rho, grad_rho};
    for (const void* q : ptrs)
        if (!dev_ok(q, h->device)) {
            h->set_error("input arrays must be 8-byte aligned device pointers");
            return VV10_ERR_INVALID_ARG;
        }
    if (atom_of_point && !dev_ok(atom_of_point, h->device, 4)) {
        h->set_error("atom_of_point must be a device pointer");
        return VV10_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BatchState& B = h->batch;
    h->batch_drop_graph();
    B.prepared = B.have_euw = B.have_abc = false;
    B.pair_tab_fp64 = -1;
    B.tc_classes.clear();
    B.f16_classes.clear();
    B.hess_P.clear();
    B.mol.assign(n_mol, BatchMol());
    B.n_total = offsets[n_mol];

    // phase 1: histogram + scan of every molecule into pooled scratch
    std::vector<size_t> sc_off(n_mol);
    size_t sc_bytes = 0;
    for (int32_t m = 0; m < n_mol; ++m) {
        BatchMol& M = B.mol[m];
        M.off = offsets[m];
        M.n = offsets[m + 1] - offsets[m];
        M.n_atom = n_atom ? n_atom[m] : 0;
        const int nblk = prepare_nblk(M.n);
        const int n_keys = (M.n_atom > 0 ? M.n_atom : 1) + 1;
        const size_t Mk = static_cast<size_t>(n_keys) * nblk;
        sc_off[m] = sc_bytes;
        sc_bytes += a256(4 * Mk) + a256(8 * (Mk + n_keys + 1)) + a256(48 * static_cast<size_t>(nblk));
    }
    s = h->ensure(B.scratch, sc_bytes, "batch prepare scratch");
    if (s != VV10_OK) return s;
    s = h->ensure(B.small, 64 * static_cast<size_t>(n_mol), "batch prepare scalars");
    if (s != VV10_OK) return s;
    if (B.h_small_bytes < 64 * static_cast<size_t>(n_mol)) {
        if (B.h_small) cudaFreeHost(B.h_small);
        B.h_small = nullptr;
        B.h_small_bytes = 0;
        if (cudaMallocHost(&B.h_small, 64 * static_cast<size_t>(n_mol)) != cudaSuccess) {
            cudaGetLastError();
            h->set_error("pinned host allocation failed");
            return VV10_ERR_OOM;
        }
        B.h_small_bytes = 64 * static_cast<size_t>(n_mol);
    }
    int* err = static_cast<int*>(h->dev_err.p);
    // one table of every molecule's pointers, and the block prefix sums of both phases
    std::vector<PrepMol> pm(n_mol);
    std::vector<int64_t> pre_blk(n_mol + 1, 0), pre_pts(n_mol + 1, 0);
    int max_keys = 1;
    for (int32_t m = 0; m < n_mol; ++m) {
        BatchMol& M = B.mol[m];
        PrepMol& q = pm[m];
        const int nblk = prepare_nblk(M.n);
        const int n_keys = (M.n_atom > 0 ? M.n_atom : 1) + 1;
        const size_t Mk = static_cast<size_t>(n_keys) * nblk;
        char* base = static_cast<char*>(B.scratch.p) + sc_off[m];
        q.n = M.n;
        q.xyz = xyz + 3 * M.off;
        q.w = w + M.off;
        q.rho = rho + M.off;
        q.grad = grad_rho + 3 * M.off;
        q.atom = atom_of_point ? atom_of_point + M.off : nullptr;
        q.n_atom = M.n_atom;
        q.n_keys = n_keys;
        q.nblk = nblk;
        q.hist = reinterpret_cast<int32_t*>(base);
        q.offs = reinterpret_cast<int64_t*>(base + a256(4 * Mk));
        q.bbox_part = reinterpret_cast<double*>(base + a256(4 * Mk) + a256(8 * (Mk + n_keys + 1)));
        q.center = reinterpret_cast<double*>(static_cast<char*>(B.small.p) + 64 * m);
        q.nk_dev = reinterpret_cast<int64_t*>(static_cast<char*>(B.small.p) + 64 * m + 32);
        pre_blk[m + 1] = pre_blk[m] + (M.n > 0 ? nblk : 0);
        max_keys = std::max(max_keys, n_keys);
    }
    const size_t tab_bytes = a256(sizeof(PrepMol) * n_mol);
    const size_t pre_bytes = sizeof(int64_t) * (n_mol + 1);
    s = h->ensure(B.prep_tab, tab_bytes + 2 * a256(pre_bytes), "batch prepare table");
    if (s != VV10_OK) return s;
    PrepMol* d_pm = static_cast<PrepMol*>(B.prep_tab.p);
    int64_t* d_pre_blk = reinterpret_cast<int64_t*>(static_cast<char*>(B.prep_tab.p) + tab_bytes);
    int64_t* d_pre_pts = reinterpret_cast<int64_t*>(static_cast<char*>(B.prep_tab.p) + tab_bytes + a256(pre_bytes));
    cudaError_t e = cudaMemcpy(d_pm, pm.data(), sizeof(PrepMol) * n_mol, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_pre_blk, pre_blk.data(), pre_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return h->cuda_fail(e, "upload batch prepare table");
    {
        PhaseScope ph(h, PH_PREPARE, st, 2);
        e = launch_prepare_count_batch(d_pm, d_pre_blk, n_mol, pre_blk[n_mol], max_keys,
                                       prm.rho_cut, err, st);
        if (e != cudaSuccess) return h->cuda_fail(e, "batch prepare count");
    }
    e = cudaMemcpyAsync(B.h_small, B.small.p, 64 * static_cast<size_t>(n_mol),
                        cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return h->cuda_fail(e, "read kept counts");
    s = h->check_device_errors(st);  // synchronises
    if (s != VV10_OK) return s;

    // phase 2: per-molecule layout, scatter and per-point quantities
    size_t arena = 0, sums = 0;
    std::vector<size_t> ar_off(n_mol);
    for (int32_t m = 0; m < n_mol; ++m) {
        BatchMol& M = B.mol[m];
        M.nk = *reinterpret_cast<int64_t*>(static_cast<char*>(B.h_small) + 64 * m + 32);
        M.nk_pad = ((M.nk + kJTile - 1) / kJTile) * kJTile;
        M.cap = M.nk_pad > 0 ? M.nk_pad : kJTile;
        const int n_seg = (M.n_atom > 0 ? M.n_atom : 1) + 1;
        ar_off[m] = arena;
        arena += a256(8 * M.cap) + a256(8 * static_cast<size_t>(n_seg)) + a256(4 * M.cap) +
                 a256(8 * F_COUNT * M.cap) + 2 * a256(32 * M.cap) + 2 * a256(16 * M.cap) +
                 a256(32 * M.cap);
        M.sums = sums;
        sums += 6 * a256(8 * M.cap);
    }
    s = h->ensure(B.arena, arena, "batch point blocks");
    if (s != VV10_OK) return s;
    s = h->ensure(B.sums, sums, "batch row sums");
    if (s != VV10_OK) return s;
    const double beta = std::pow(3.0 / (prm.b * prm.b), 0.75) / 32.0;
    for (int32_t m = 0; m < n_mol; ++m) {
        BatchMol& M = B.mol[m];
        const int n_seg = (M.n_atom > 0 ? M.n_atom : 1) + 1;
        char* p = static_cast<char*>(B.arena.p) + ar_off[m];
        int64_t* orig = reinterpret_cast<int64_t*>(p);
        p += a256(8 * M.cap);
        int64_t* seg = reinterpret_cast<int64_t*>(p);
        p += a256(8 * static_cast<size_t>(n_seg));
        int32_t* atom_k = reinterpret_cast<int32_t*>(p);
        p += a256(4 * M.cap);
        double* soa = reinterpret_cast<double*>(p);
        p += a256(8 * F_COUNT * M.cap);
        double4* r64a = reinterpret_cast<double4*>(p);
        p += a256(32 * M.cap);
        double4* r64b = reinterpret_cast<double4*>(p);
        p += a256(32 * M.cap);
        float4* r32a = reinterpret_cast<float4*>(p);
        p += a256(16 * M.cap);
        float4* r32b = reinterpret_cast<float4*>(p);
        p += a256(16 * M.cap);
        float4* r32p = reinterpret_cast<float4*>(p);
        PrepMol& q = pm[m];
        q.nk = M.nk;
        q.nk_pad = M.nk_pad;
        q.orig = orig;
        q.seg = seg;
        q.atom_k = atom_k;
        q.soa = soa;
        q.r64a = r64a;
        q.r64b = r64b;
        q.r32a = r32a;
        q.r32b = r32b;
        q.r32p = r32p;
        pre_pts[m + 1] = pre_pts[m] + M.nk_pad / 256;
        PointsDev& P = M.P;
        P.n = M.n;
        P.nk = M.nk;
        P.nk_pad = M.nk_pad;
        P.n_atom = M.n_atom;
        P.beta = beta;
        P.orig = orig;
        P.seg = seg;
        P.atom = atom_k;
        const double* f = soa;
        const int64_t c = M.cap;
        P.w = f + F_W * c;
        P.rho = f + F_RHO * c;
        P.gx = f + F_GX * c;
        P.gy = f + F_GY * c;
        P.gz = f + F_GZ * c;
        P.om = f + F_OM * c;
        P.ka = f + F_KA * c;
        P.om_r = f + F_OMR * c;
        P.om_g = f + F_OMG * c;
        P.ka_r = f + F_KAR * c;
        P.om_rr = f + F_OMRR * c;
        P.om_rg = f + F_OMRG * c;
        P.om_gg = f + F_OMGG * c;
        P.ka_rr = f + F_KARR * c;
        P.r64a = r64a;
        P.r64b = r64b;
        P.r32a = r32a;
        P.r32b = r32b;
        P.r32p = r32p;
        n_kept[m] = M.nk;
    }
    e = cudaMemcpy(d_pm, pm.data(), sizeof(PrepMol) * n_mol, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_pre_pts, pre_pts.data(), pre_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return h->cuda_fail(e, "upload batch prepare table");
    {
        PhaseScope ph(h, PH_PREPARE, st, 2);
        e = launch_prepare_scatter_batch(d_pm, d_pre_blk, d_pre_pts, n_mol, pre_blk[n_mol],
                                         pre_pts[n_mol], max_keys, prm.rho_cut, prm.b, prm.C, st);
        if (e != cudaSuccess) return h->cuda_fail(e, "batch prepare scatter");
    }
    B.order.resize(n_mol);
    std::iota(B.order.begin(), B.order.end(), 0);
    std::stable_sort(B.order.begin(), B.order.end(),
                     [&](int a, int b) { return B.mol[a].nk > B.mol[b].nk; });
    B.prepared = true;
    return VV10_OK;
}

vv10_status vv10_batch_energy_potential(vv10_handle h, vv10_precision prec, double* energies,
                                        double* vrho, double* vgamma, void* stream) {
    if (!h) return VV10_ERR_INVALID_ARG;
    h->set_error("");
    if (!h->batch.prepared) {
        h->set_error("vv10_batch_prepare has not been called");
        return VV10_ERR_INVALID_ARG;
    }
    if (!precision_known(prec))
        return VV10_ERR_INVALID_ARG;
    vv10_status s = h->bind();
    if (s != VV10_OK) return s;
    if (!dev_ok(energies, h->device) || (vrho && !dev_ok(vrho, h->device)) ||
        (vgamma && !dev_ok(vgamma, h->device))) {
        h->set_error("energies / vrho / vgamma must be device pointers");
        return VV10_ERR_INVALID_ARG;
    }
    return h->batch_ep(prec, energies, vrho, vgamma, (h->options & VV10_OPT_FUSE_HESSIAN_SUMS) != 0,
                       static_cast<cudaStream_t>(stream));
}

vv10_status vv10_batch_hessian_contract(vv10_handle h, vv10_precision prec, const int32_t* P,
                                        const double* rho_t, const double* grad_rho_t,
                                        double* f_rho_t, double* f_gamma_t, void* stream) {
    if (!h) return VV10_ERR_INVALID_ARG;
    h->set_error("");
    if (!h->batch.prepared || !h->batch.have_euw) {
        h->set_error("vv10_batch_prepare and vv10_batch_energy_potential must be called first");
        return VV10_ERR_INVALID_ARG;
    }
    if (prec == VV10_MIXED_BF16X3) {
        h->set_error("the BF16x3 Hessian contraction is not available in this library");
        return VV10_ERR_UNSUPPORTED;
    }
    if (prec == VV10_FP64_TC) {
        h->set_error("the FP64 tensor-core contraction is built for single systems "
                     "(vv10_hessian_contract); a batch takes VV10_FP64");
        return VV10_ERR_UNSUPPORTED;
    }
    if (prec != VV10_FP64 && prec != VV10_MIXED_TF32X3 && prec != VV10_MIXED_F16X3)
        return VV10_ERR_INVALID_ARG;
    if (!P) return VV10_ERR_INVALID_ARG;
    for (size_t m = 0; m < h->batch.mol.size(); ++m)
        if (P[m] < 1 || P[m] > VV10_MAX_TRIALS) {
            h->set_error("every molecule needs 1 <= P <= VV10_MAX_TRIALS");
            return VV10_ERR_INVALID_ARG;
        }
    vv10_status s = h->bind();
    if (s != VV10_OK) return s;
    const void* ptrs[] = {rho_t, grad_rho_t, f_rho_t, f_gamma_t};
    for (const void* q : ptrs)
        if (!dev_ok(q, h->device)) {
            h->set_error("trial and output arrays must be 8-byte aligned device pointers");
            return VV10_ERR_INVALID_ARG;
        }
    return h->batch_hess(prec, P, rho_t, grad_rho_t, f_rho_t, f_gamma_t,
                         static_cast<cudaStream_t>(stream));
}

vv10_status vv10_batch_run(vv10_handle h, vv10_precision prec, const int32_t* P,
                           const double* rho_t, const double* grad_rho_t, double* energies,
                           double* vrho, double* vgamma, double* f_rho_t, double* f_gamma_t,
                           void* stream) {
    if (!h) return VV10_ERR_INVALID_ARG;
    BatchState& B = h->batch;
    if (!B.prepared || !P) {
        h->set_error("vv10_batch_prepare has not been called");
        return VV10_ERR_INVALID_ARG;
    }
    vv10_status s = h->bind();
    if (s != VV10_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const std::vector<const void*> key = {rho_t, grad_rho_t, energies, vrho, vgamma, f_rho_t, f_gamma_t};
    const std::vector<int32_t> Pv(P, P + B.mol.size());
    if (B.graph && B.graph_key == key && B.graph_prec == static_cast<int>(prec) && B.graph_P == Pv) {
        cudaError_t e = cudaGraphLaunch(B.graph, st);
        if (e != cudaSuccess) return h->cuda_fail(e, "graph launch");
        for (int k = 0; k < PH_COUNT; ++k) h->launches[k] += B.graph_launches[k];
        return VV10_OK;
    }
    h->batch_drop_graph();
    // first call for this configuration: run eagerly (allocates, builds the tables) ...
    if (!dev_ok(energies, h->device) || (vrho && !dev_ok(vrho, h->device)) ||
        (vgamma && !dev_ok(vgamma, h->device))) {
        h->set_error("energies / vrho / vgamma must be device pointers");
        return VV10_ERR_INVALID_ARG;
    }
    if (!precision_known(prec))
        return VV10_ERR_INVALID_ARG;
    s = h->batch_ep(prec, energies, vrho, vgamma, true, st);  // A/B/C in the same pass
    if (s != VV10_OK) return s;
    s = vv10_batch_hessian_contract(h, prec, P, rho_t, grad_rho_t, f_rho_t, f_gamma_t, stream);
    if (s != VV10_OK) return s;
    // ... then record the same sequence, which now allocates nothing, as a CUDA graph
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return h->cuda_fail(e, "capture stream");
    const bool prof = h->prof_on;
    int64_t launches[PH_COUNT];
    std::memcpy(launches, h->launches, sizeof(launches));
    h->prof_on = false;  // no event records inside the graph
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) {
        s = h->batch_ep(prec, energies, vrho, vgamma, true, cs);
        if (s == VV10_OK) s = h->batch_hess(prec, P, rho_t, grad_rho_t, f_rho_t, f_gamma_t, cs);
        e = cudaStreamEndCapture(cs, &g);
        if (s == VV10_OK && e == cudaSuccess) e = cudaGraphInstantiate(&B.graph, g, 0);
        if (e != cudaSuccess) B.graph = nullptr;
    }
    if (g) cudaGraphDestroy(g);
    h->prof_on = prof;
    for (int k = 0; k < PH_COUNT; ++k) {  // recording launched nothing: keep the counts per replay
        B.graph_launches[k] = h->launches[k] - launches[k];
        h->launches[k] = launches[k];
    }
    cudaStreamDestroy(cs);
    if (s != VV10_OK) return s;
    if (e != cudaSuccess) return h->cuda_fail(e, "recording the batch graph");
    if (B.graph) {
        B.graph_key = key;
        B.graph_prec = static_cast<int>(prec);
        B.graph_P = Pv;
    }
    return VV10_OK;
}

}  // extern "C"
