// Autotuner (the paper has no counterpart): times the candidate tile shapes of the pair-sum
// kernels and the candidate trial-group widths of the tensor-core contraction on the data a
// handle has prepared, keeps the fastest, and caches the choice for the process.
//
// Free parameters:
//   single-system pair sums (per mode and precision): rows per thread (FP32 1/2/4, FP64 1/2)
//     and the number of j-splits (the SM-count default, half and twice it);
//   batched pair sums (per precision): rows per thread and j tiles per split (16/32/64);
//   contraction: the widest trial group (64, 96, 128, 192 trials).  Up to 64 trials both
//     outputs share one tile generation; wider groups generate the two outputs' tiles
//     separately but issue fewer MMAs per trial, so which is faster depends on P and N.
// Keys: kernel, mode, precision, N bucket = ceil(log2 N_kept) (for a batch that of its
// largest molecule), trial count (contraction) or batch-size bucket, and SM count.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "kernels.hpp"
#include "vv10_internal.hpp"

using namespace vv10;

namespace {

struct Key {
    int kind, mode, fp64, nb, pb, n_sm;
    bool operator<(const Key& o) const {
        return std::tie(kind, mode, fp64, nb, pb, n_sm) < std::tie(o.kind, o.mode, o.fp64, o.nb, o.pb, o.n_sm);
    }
};
std::mutex g_mu;
std::map<Key, std::pair<int, int>>& cache() {
    static std::map<Key, std::pair<int, int>> c;
    return c;
}

// Keeps the handle's launch counters and profiling untouched by the tuning runs.
struct QuietScope {
    vv10_ctx* h;
    bool prof;
    int64_t launches[PH_COUNT];
    explicit QuietScope(vv10_ctx* h_) : h(h_), prof(h_->prof_on) {
        for (int k = 0; k < PH_COUNT; ++k) launches[k] = h->launches[k];
        h->prof_on = false;
    }
    ~QuietScope() {
        for (int k = 0; k < PH_COUNT; ++k) h->launches[k] = launches[k];
        h->prof_on = prof;
    }
};

// Fastest of `reps` timed runs of f (after one untimed run), in milliseconds.
template <class F>
vv10_status best_ms(vv10_ctx* h, cudaStream_t st, int reps, F&& f, float* out) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return h->cuda_fail(cudaGetLastError(), "tuning events");
    }
    vv10_status s = f();
    float best = 3.0e38f;
    for (int r = 0; r < reps && s == VV10_OK; ++r) {
        cudaEventRecord(a, st);
        s = f();
        cudaEventRecord(b, st);
        if (s != VV10_OK) break;
        cudaError_t e = cudaEventSynchronize(b);
        if (e != cudaSuccess) {
            s = h->cuda_fail(e, "tuning run");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s == VV10_OK) s = h->check_device_errors(st);
    *out = best;
    return s;
}

}  // namespace

namespace vv10 {

int n_bucket(int64_t n) {
    int b = 0;
    while ((static_cast<int64_t>(1) << b) < n) ++b;
    return b;
}

bool tune_cache_get(int kind, int mode, int fp64, int nb, int pb, int n_sm, int* v0, int* v1) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = cache().find(Key{kind, mode, fp64, nb, pb, n_sm});
    if (it == cache().end()) return false;
    *v0 = it->second.first;
    *v1 = it->second.second;
    return true;
}

void tune_cache_put(int kind, int mode, int fp64, int nb, int pb, int n_sm, int v0, int v1) {
    std::lock_guard<std::mutex> lk(g_mu);
    cache()[Key{kind, mode, fp64, nb, pb, n_sm}] = {v0, v1};
}

bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;  // unknown: do not time anything
    }
    return cs != cudaStreamCaptureStatusNone;
}

}  // namespace vv10

// Single-system pair sums of one mode: rows per thread x j-splits.
vv10_status vv10_ctx::tune_pairsum(int mode, bool fp64, cudaStream_t st, bool force) {
    TileOverride& o = overrides[mode + kPairModes * (fp64 ? 1 : 0)];
    if (o.manual || P.nk == 0) return VV10_OK;
    const int nb = n_bucket(P.nk);
    if (!force && o.active && o.bucket == nb) return VV10_OK;
    int rpt = 0, ns = 0;
    if (!force && tune_cache_get(TUNE_PAIRSUM, mode, fp64, nb, 0, n_sm, &rpt, &ns)) {
        o = TileOverride{true, false, mode, fp64, rpt, ns, nb};
        return VV10_OK;
    }
    if (stream_capturing(st)) return VV10_OK;
    QuietScope quiet(this);
    const std::vector<int> rpts = fp64 ? std::vector<int>{1, 2} : std::vector<int>{1, 2, 4};
    float best = 3.0e38f;
    int best_r = fp64 ? 1 : 2, best_s = 0;
    for (int r : rpts) {
        const int d = pairsum_default_split(P, mode, fp64, r, n_sm);
        std::vector<int> splits = {d};
        if (d / 2 >= 1) splits.push_back(d / 2);
        splits.push_back(2 * d);
        for (int sp : splits) {
            o = TileOverride{true, false, mode, fp64, r, sp, nb};
            float ms = 0.f;
            int ns_out = 0;
            vv10_status s = best_ms(this, st, 2, [&] { return run_pairsum(mode, fp64, st, &ns_out); }, &ms);
            if (s != VV10_OK) {
                o = TileOverride{};
                return s;
            }
            if (ms < best) {
                best = ms;
                best_r = r;
                best_s = sp;
            }
        }
    }
    o = TileOverride{true, false, mode, fp64, best_r, best_s, nb};
    tune_cache_put(TUNE_PAIRSUM, mode, fp64, nb, 0, n_sm, best_r, best_s);
    return VV10_OK;
}

// Batched pair sums: rows per thread x j tiles per split, timed on the fused energy and
// A/B/C sums (the pass vv10_batch_run makes).
vv10_status vv10_ctx::tune_batch(bool fp64, cudaStream_t st, bool force) {
    BatchState& B = batch;
    TileOverride& o = batch_over[fp64 ? 1 : 0];
    if (o.manual || !B.prepared) return VV10_OK;
    int64_t nk_max = 0, nk_sum = 0;
    for (const BatchMol& M : B.mol) {
        nk_max = M.nk > nk_max ? M.nk : nk_max;
        nk_sum += M.nk;
    }
    if (nk_sum == 0) return VV10_OK;
    const int nb = n_bucket(nk_max), pb = n_bucket(nk_sum);
    if (!force && o.active && o.bucket == nb * 64 + pb) return VV10_OK;
    int rpt = 0, sp = 0;
    if (!force && tune_cache_get(TUNE_BATCH, 0, fp64, nb, pb, n_sm, &rpt, &sp)) {
        o = TileOverride{true, false, 0, fp64, rpt, sp, nb * 64 + pb};
        return VV10_OK;
    }
    if (stream_capturing(st)) return VV10_OK;
    QuietScope quiet(this);
    const std::vector<int> rpts = fp64 ? std::vector<int>{1, 2} : std::vector<int>{1, 2, 4};
    float best = 3.0e38f;
    int best_r = fp64 ? 1 : 2, best_t = 32;
    int* err = static_cast<int*>(dev_err.p);
    for (int r : rpts)
        for (int t : {16, 32, 64}) {
            vv10_status s = batch_pair_tables(fp64, r, t);
            if (s != VV10_OK) return s;
            float ms = 0.f;
            s = best_ms(this, st, 1, [&]() -> vv10_status {
                cudaError_t e = launch_pairsum_batch(
                    reinterpret_cast<PairMol*>(static_cast<char*>(B.pair_tab.p) + B.pair_mols),
                    reinterpret_cast<PairTask*>(static_cast<char*>(B.pair_tab.p) + B.pair_tasks),
                    B.n_pair_tasks, static_cast<int*>(B.counter.p), MODE_EUWABC, fp64, r, n_sm, err, st);
                return e == cudaSuccess ? VV10_OK : cuda_fail(e, "batched pair sums");
            }, &ms);
            if (s != VV10_OK) return s;
            if (ms < best) {
                best = ms;
                best_r = r;
                best_t = t;
            }
        }
    o = TileOverride{true, false, 0, fp64, best_r, best_t, nb * 64 + pb};
    tune_cache_put(TUNE_BATCH, 0, fp64, nb, pb, n_sm, best_r, best_t);
    return VV10_OK;
}

// Widest trial group of the contraction for P trials over nk kept points: vv10_set_tiles,
// else a tuned choice for this (P, N bucket), else 192.
int vv10_ctx::tc_cap_for(int32_t Pn, int64_t nk) const {
    if (tc_cap_manual > 0) return tc_cap_manual;
    int cap = 0, unused = 0;
    if (tune_cache_get(TUNE_TC_CAP, 0, 0, n_bucket(nk), Pn, n_sm, &cap, &unused)) return cap;
    return 192;
}

// Times the split + contraction of the prepared trials for every distinct group layout and
// caches the fastest width (only for P > 64: below that every width gives one group).
vv10_status vv10_ctx::tune_tc_cap(int32_t Pn, cudaStream_t st, int* cap) {
    *cap = tc_cap_for(Pn, P.nk);
    int c0 = 0, unused = 0;
    if (tc_cap_manual > 0 || Pn <= 64 ||
        tune_cache_get(TUNE_TC_CAP, 0, 0, n_bucket(P.nk), Pn, n_sm, &c0, &unused) ||
        stream_capturing(st))
        return VV10_OK;
    QuietScope quiet(this);
    std::vector<std::pair<int, int>> seen;  // (groups, padded width)
    float best = 3.0e38f;
    int best_cap = 192;
    for (int c : {192, 128, 96, 64}) {
        const int ng = (Pn + c - 1) / c;
        const int pg = (Pn + ng - 1) / ng;
        const std::pair<int, int> lay{ng, hess_tc_ppad(pg)};
        bool dup = false;
        for (const auto& x : seen) dup = dup || x == lay;
        if (dup) continue;
        seen.push_back(lay);
        float ms = 0.f;
        vv10_status s = best_ms(this, st, 1, [&] { return tc_contract(Pn, c, st); }, &ms);
        if (s != VV10_OK) return s;
        if (ms < best) {
            best = ms;
            best_cap = c;
        }
    }
    tune_cache_put(TUNE_TC_CAP, 0, 0, n_bucket(P.nk), Pn, n_sm, best_cap, 0);
    *cap = best_cap;
    return VV10_OK;
}
