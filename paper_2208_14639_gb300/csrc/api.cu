// C ABI of the VV10 library: handle, argument validation, buffer management and the
// orchestration of the kernels of each entry point (declared in include/vv10.h).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"
#include "kernels.hpp"
#include "vv10.h"
#include "vv10_internal.hpp"

using namespace vv10;

// ---------------------------------------------------------------- helpers

void vv10_ctx::set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(last_error, sizeof(last_error), fmt, ap);
    va_end(ap);
}

vv10_status vv10_ctx::cuda_fail(cudaError_t e, const char* where) {
    set_error("%s: %s", where, cudaGetErrorString(e));
    cudaGetLastError();  // clear a sticky-free error so later calls can proceed
    return e == cudaErrorMemoryAllocation ? VV10_ERR_OOM : VV10_ERR_CUDA;
}

vv10_status vv10_ctx::ensure(DevBuf& b, size_t bytes, const char* what) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return VV10_OK;
    if (debug_fail_alloc > 0 && --debug_fail_alloc == 0) {
        set_error("allocation of %zu bytes for %s failed (injected)", bytes, what);
        return VV10_ERR_OOM;
    }
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        set_error("cudaMalloc(%zu) for %s: %s", bytes, what, cudaGetErrorString(e));
        return VV10_ERR_OOM;
    }
    b.bytes = bytes;
    return VV10_OK;
}

void vv10_ctx::release_all() {
    batch_release();
    DevBuf* bufs[] = {&prep_hist, &prep_offs, &prep_bbox, &prep_small, &orig, &seg, &atom_k,
                      &soa, &r64a, &r64b, &r32a, &r32b, &r32p, &sumE, &sumU, &sumW, &sumA, &sumB,
                      &sumC, &part, &eblk, &scal, &tu, &ty, &trt, &tgt, &hacc, &gk,
                      &tc_uh, &tc_ul, &tc_yh, &tc_yl, &tc16_bh, &tc16_bl, &tc16_small, &o64_sl, &o64_small, &o64_rec, &hvp_fr, &hvp_fg, &nhess, &chpart, &wdir, &wsplit, &ehalf, &aophik, &aoz, &aom, &aogw, &aofa, &ngpart, &dev_err};
    for (DevBuf* b : bufs) {
        if (b->p) cudaFree(b->p);
        b->p = nullptr;
        b->bytes = 0;
    }
    if (h_pinned) cudaFreeHost(h_pinned);
    h_pinned = nullptr;
    for (ProfRec& r : prof) {
        event_pool.push_back(r.a);
        event_pool.push_back(r.b);
    }
    prof.clear();
    for (cudaEvent_t e : event_pool) cudaEventDestroy(e);
    event_pool.clear();
}

// Pointer must be device-accessible memory of this handle's device (device or managed).
static bool device_ptr_ok(const void* p, int device) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

static bool aligned(const void* p, size_t a) {
    return (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

#define VV10_CHECK_HANDLE(h)                          \
    do {                                              \
        if (!(h)) return VV10_ERR_INVALID_ARG;        \
    } while (0)

#define VV10_CUDA(h, expr, where)                        \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return (h)->cuda_fail(e_, where); \
    } while (0)

#define VV10_TRY(expr)                        \
    do {                                      \
        vv10_status s_ = (expr);              \
        if (s_ != VV10_OK) return s_;         \
    } while (0)

vv10_status vv10_ctx::bind() {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return VV10_OK;
}

// Read and clear the device error word (synchronises the stream).
vv10_status vv10_ctx::check_device_errors(cudaStream_t st) {
    int* herr = reinterpret_cast<int*>(h_pinned) + 8;
    VV10_CUDA(this, cudaMemcpyAsync(herr, dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, st),
              "read error word");
    VV10_CUDA(this, cudaMemsetAsync(dev_err.p, 0, sizeof(int), st), "clear error word");
    VV10_CUDA(this, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    const int v = *herr;
    if (v & DEVERR_TIMEOUT) {
        set_error("a bounded device-side wait gave up");
        return VV10_ERR_TIMEOUT;
    }
    if (v & DEVERR_BAD_ATOM) {
        set_error("atom_of_point holds an index outside [0, n_atom)");
        return VV10_ERR_INVALID_ARG;
    }
    if (v & DEVERR_BAD_INPUT) {
        set_error("non-finite coordinate, weight, density or gradient in the input");
        return VV10_ERR_INVALID_ARG;
    }
    if (v & DEVERR_NONFINITE) {
        set_error("a non-finite value was produced in an output");
        return VV10_ERR_NONFINITE;
    }
    return VV10_OK;
}

PointsDev vv10_ctx::points() const { return P; }

cudaEvent_t vv10_ctx::take_event() {
    if (!event_pool.empty()) {
        cudaEvent_t e = event_pool.back();
        event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void vv10_ctx::phase_begin(int phase, cudaStream_t st, ProfRec* rec) {
    rec->phase = phase;
    rec->a = rec->b = nullptr;
    if (!prof_on) return;
    rec->a = take_event();
    if (rec->a) cudaEventRecord(rec->a, st);
}

void vv10_ctx::phase_end(ProfRec* rec, cudaStream_t st, int n_launch) {
    launches[rec->phase] += n_launch;
    if (!prof_on || !rec->a) return;
    rec->b = take_event();
    if (!rec->b) {
        event_pool.push_back(rec->a);
        return;
    }
    cudaEventRecord(rec->b, st);
    prof.push_back(*rec);
}

// ---------------------------------------------------------------- ABI

extern "C" {

const char* vv10_status_string(vv10_status s) {
    switch (s) {
        case VV10_OK: return "ok";
        case VV10_ERR_INVALID_ARG: return "invalid argument";
        case VV10_ERR_CUDA: return "CUDA error";
        case VV10_ERR_OOM: return "out of device memory";
        case VV10_ERR_TIMEOUT: return "device-side wait timed out";
        case VV10_ERR_NONFINITE: return "non-finite output";
        case VV10_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

const char* vv10_last_error(vv10_handle h) { return h ? h->last_error : "null handle"; }

vv10_status vv10_create(vv10_handle* out, int device) {
    if (!out) return VV10_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VV10_ERR_CUDA;
    }
    if (device < 0 || device >= count) return VV10_ERR_INVALID_ARG;
    vv10_ctx* h = new (std::nothrow) vv10_ctx();
    if (!h) return VV10_ERR_OOM;
    h->device = device;
    vv10_status s = h->bind();
    if (s != VV10_OK) {
        delete h;
        return s;
    }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete h;
        cudaGetLastError();
        return VV10_ERR_CUDA;
    }
    h->n_sm = prop.multiProcessorCount;
    h->cc_major = prop.major;
    h->cc_minor = prop.minor;
    e = cudaMallocHost(&h->h_pinned, 256);
    if (e != cudaSuccess) {
        delete h;
        cudaGetLastError();
        return VV10_ERR_OOM;
    }
    s = h->ensure(h->dev_err, 64, "error word");
    if (s == VV10_OK) {
        e = cudaMemset(h->dev_err.p, 0, 64);
        if (e != cudaSuccess) s = h->cuda_fail(e, "cudaMemset");
    }
    if (s != VV10_OK) {
        h->release_all();
        delete h;
        return s;
    }
    *out = h;
    return VV10_OK;
}

vv10_status vv10_destroy(vv10_handle h) {
    if (!h) return VV10_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    cudaGetLastError();
    h->release_all();
    delete h;
    return VV10_OK;
}

vv10_status vv10_sync(vv10_handle h, void* stream) {
    VV10_CHECK_HANDLE(h);
    VV10_TRY(h->bind());
    return h->check_device_errors(static_cast<cudaStream_t>(stream));
}

vv10_status vv10_prepare_points(vv10_handle h, int64_t n, const double* xyz, const double* w,
                                const double* rho, const double* grad_rho,
                                const int32_t* atom_of_point, int32_t n_atom, vv10_params prm,
                                int64_t* n_kept, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    if (n < 1 || !n_kept) {
        h->set_error("n must be >= 1 and n_kept non-NULL");
        return VV10_ERR_INVALID_ARG;
    }
    if (!(prm.b > 0.0) || !(prm.C >= 0.0) || !(prm.rho_cut > 0.0) || !std::isfinite(prm.b) ||
        !std::isfinite(prm.C) || !std::isfinite(prm.rho_cut)) {
        h->set_error("parameters need b > 0, C >= 0, rho_cut > 0 (finite)");
        return VV10_ERR_INVALID_ARG;
    }
    if (n_atom < 0 || (atom_of_point == nullptr) != (n_atom == 0)) {
        h->set_error("atom_of_point and n_atom must be given together");
        return VV10_ERR_INVALID_ARG;
    }
    if (n_atom > VV10_MAX_ATOMS) {
        h->set_error("n_atom %d exceeds VV10_MAX_ATOMS", n_atom);
        return VV10_ERR_UNSUPPORTED;
    }
    VV10_TRY(h->bind());
    const void* ptrs[] = {xyz, w, rho, grad_rho};
    for (const void* q : ptrs)
        if (!device_ptr_ok(q, h->device) || !aligned(q, 8)) {
            h->set_error("input arrays must be 8-byte aligned device pointers on device %d",
                         h->device);
            return VV10_ERR_INVALID_ARG;
        }
    if (atom_of_point && (!device_ptr_ok(atom_of_point, h->device) || !aligned(atom_of_point, 4))) {
        h->set_error("atom_of_point must be a device pointer");
        return VV10_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    h->prepared = false;
    h->have_euw = false;
    h->have_abc = false;

    const int nblk = prepare_nblk(n);
    const int n_keys = (n_atom > 0 ? n_atom : 1) + 1;
    const int64_t M = static_cast<int64_t>(n_keys) * nblk;
    VV10_TRY(h->ensure(h->prep_hist, sizeof(int32_t) * M, "prepare histogram"));
    VV10_TRY(h->ensure(h->prep_offs, sizeof(int64_t) * (M + n_keys + 1), "prepare offsets"));
    VV10_TRY(h->ensure(h->prep_bbox, sizeof(double) * 6 * nblk, "prepare bbox"));
    VV10_TRY(h->ensure(h->prep_small, 64, "prepare scalars"));
    PrepareScratch ps;
    ps.hist = static_cast<int32_t*>(h->prep_hist.p);
    ps.offs = static_cast<int64_t*>(h->prep_offs.p);
    ps.bbox_part = static_cast<double*>(h->prep_bbox.p);
    ps.center = static_cast<double*>(h->prep_small.p);
    ps.nk_dev = reinterpret_cast<int64_t*>(static_cast<double*>(h->prep_small.p) + 4);
    int* err = static_cast<int*>(h->dev_err.p);
    {
        PhaseScope ph(h, PH_PREPARE, st, 2);
        VV10_CUDA(h, launch_prepare_count(n, xyz, w, rho, grad_rho, atom_of_point, n_atom,
                                          prm.rho_cut, ps, err, st),
                  "prepare count");
    }
    int64_t* hnk = reinterpret_cast<int64_t*>(h->h_pinned);
    VV10_CUDA(h, cudaMemcpyAsync(hnk, ps.nk_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st),
              "read n_kept");
    VV10_TRY(h->check_device_errors(st));  // synchronises
    const int64_t nk = *hnk;
    const int64_t nk_pad = ((nk + kJTile - 1) / kJTile) * kJTile;
    const int64_t cap = nk_pad > 0 ? nk_pad : kJTile;
    const int n_seg = (n_atom > 0 ? n_atom : 1) + 1;
    VV10_TRY(h->ensure(h->orig, sizeof(int64_t) * cap, "kept index map"));
    VV10_TRY(h->ensure(h->seg, sizeof(int64_t) * n_seg, "atom segments"));
    VV10_TRY(h->ensure(h->atom_k, sizeof(int32_t) * cap, "kept atoms"));
    VV10_TRY(h->ensure(h->soa, sizeof(double) * F_COUNT * cap, "point arrays"));
    VV10_TRY(h->ensure(h->r64a, sizeof(double4) * cap, "FP64 records"));
    VV10_TRY(h->ensure(h->r64b, sizeof(double4) * cap, "FP64 records"));
    VV10_TRY(h->ensure(h->r32a, sizeof(float4) * cap, "FP32 records"));
    VV10_TRY(h->ensure(h->r32b, sizeof(float4) * cap, "FP32 records"));
    VV10_TRY(h->ensure(h->r32p, sizeof(float4) * 2 * cap, "pair-packed FP32 records"));
    PhaseScope ph_scatter(h, PH_PREPARE, st, nk_pad > 0 ? 2 : 1);
    VV10_CUDA(h, launch_prepare_scatter(n, xyz, w, rho, grad_rho, atom_of_point, n_atom,
                                        prm.rho_cut, prm.b, prm.C, ps, nk, nk_pad,
                                        static_cast<int64_t*>(h->orig.p),
                                        static_cast<int64_t*>(h->seg.p),
                                        static_cast<int32_t*>(h->atom_k.p),
                                        static_cast<double*>(h->soa.p),
                                        static_cast<double4*>(h->r64a.p),
                                        static_cast<double4*>(h->r64b.p),
                                        static_cast<float4*>(h->r32a.p),
                                        static_cast<float4*>(h->r32b.p),
                                        static_cast<float4*>(h->r32p.p), st),
              "prepare scatter");
    PointsDev& P = h->P;
    P.n = n;
    P.nk = nk;
    P.nk_pad = nk_pad;
    P.n_atom = n_atom;
    P.beta = std::pow(3.0 / (prm.b * prm.b), 0.75) / 32.0;  // beta of Sec. II.A
    P.orig = static_cast<const int64_t*>(h->orig.p);
    P.seg = static_cast<const int64_t*>(h->seg.p);
    P.atom = static_cast<const int32_t*>(h->atom_k.p);
    const double* f = static_cast<const double*>(h->soa.p);
    P.w = f + F_W * cap;
    P.rho = f + F_RHO * cap;
    P.gx = f + F_GX * cap;
    P.gy = f + F_GY * cap;
    P.gz = f + F_GZ * cap;
    P.om = f + F_OM * cap;
    P.ka = f + F_KA * cap;
    P.om_r = f + F_OMR * cap;
    P.om_g = f + F_OMG * cap;
    P.ka_r = f + F_KAR * cap;
    P.om_rr = f + F_OMRR * cap;
    P.om_rg = f + F_OMRG * cap;
    P.om_gg = f + F_OMGG * cap;
    P.ka_rr = f + F_KARR * cap;
    P.r64a = static_cast<const double4*>(h->r64a.p);
    P.r64b = static_cast<const double4*>(h->r64b.p);
    P.r32a = static_cast<const float4*>(h->r32a.p);
    P.r32b = static_cast<const float4*>(h->r32b.p);
    P.r32p = static_cast<const float4*>(h->r32p.p);
    h->soa_ld = cap;
    h->prm = prm;
    h->prepared = true;
    *n_kept = nk;
    return VV10_OK;
}

}  // extern "C"

// SoA arrays are laid out with leading dimension soa_ld (= nk_pad, or kJTile when empty);
// kernels index them with nk_pad, so keep the two equal.
static_assert(kJTile > 0, "tile");

vv10_status vv10_ctx::require_prepared() {
    if (!prepared) {
        set_error("vv10_prepare_points has not been called on this handle");
        return VV10_ERR_INVALID_ARG;
    }
    return VV10_OK;
}

vv10_status vv10_ctx::run_pairsum(int mode, bool fp64, cudaStream_t st, int* n_split_out) {
    if (autotune & VV10_TUNE_PAIRSUMS) VV10_TRY(tune_pairsum(mode, fp64, st, false));
    const int nq = pair_mode_nq(mode);
    PairLaunch cfg;
    const TileChoice tc = tiles_for(mode, fp64);
    cfg.rows_per_thread = tc.rows_per_thread;
    cfg.n_split = tc.n_split > 0 ? tc.n_split : pairsum_default_split(P, mode, fp64, cfg.rows_per_thread, n_sm);
    if (debug_stall) {
        cfg.stall = 1;
        debug_stall = 0;
    }
    const int ns = pairsum_split_count(P.nk_pad, cfg.n_split);  // the splits the launch uses
    VV10_TRY(ensure(part, sizeof(double) * nq * static_cast<size_t>(ns) * (P.nk_pad > 0 ? P.nk_pad : 1),
                    "pair-sum partials"));
    {
        PhaseScope ph(this, (mode == MODE_EUW || mode == MODE_EUWABC || mode == MODE_EUWABCG) ? PH_PAIR_EUW
                            : (mode == MODE_ABC ? PH_PAIR_ABC : PH_PAIR_GRAD),
                      st, 1);
        VV10_CUDA(this, launch_pairsum(P, mode, fp64, cfg, static_cast<double*>(part.p),
                                       static_cast<int*>(dev_err.p), st),
                  "pair-sum kernel");
    }
    *n_split_out = ns;
    return VV10_OK;
}

// Tiles of a pair-sum mode: its own override (fixed or tuned), else (fused mode) the
// energy sums' override, else 2 (FP32) / 1 (FP64) rows per thread and SM-derived splits.
TileChoice vv10_ctx::tiles_for(int mode, bool fp64) const {
    TileChoice t;
    t.rows_per_thread = fp64 ? 1 : 2;
    t.n_split = 0;
    const TileOverride& o = overrides[mode + kPairModes * (fp64 ? 1 : 0)];
    const TileOverride& e = overrides[MODE_EUW + kPairModes * (fp64 ? 1 : 0)];
    const bool fused = (mode == MODE_EUWABC || mode == MODE_EUWABCG);
    const TileOverride* use = o.active ? &o : ((fused && e.active) ? &e : nullptr);
    if (use) {
        t.rows_per_thread = use->rows_per_thread;
        t.n_split = use->n_split;
    }
    return t;
}

extern "C" {

vv10_status vv10_energy_potential(vv10_handle h, vv10_precision prec, double* energy,
                                  double* vrho, double* vgamma, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (!precision_known(prec)) {
        h->set_error("unknown precision %d", static_cast<int>(prec));
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    if ((vrho && (!device_ptr_ok(vrho, h->device) || !aligned(vrho, 8))) ||
        (vgamma && (!device_ptr_ok(vgamma, h->device) || !aligned(vgamma, 8)))) {
        h->set_error("vrho / vgamma must be 8-byte aligned device pointers");
        return VV10_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool fp64 = precision_fp64(prec);
    PointsDev& P = h->P;
    const size_t nkb = sizeof(double) * static_cast<size_t>(h->soa_ld);
    VV10_TRY(h->ensure(h->sumE, nkb, "E_i"));
    VV10_TRY(h->ensure(h->sumU, nkb, "U_i"));
    VV10_TRY(h->ensure(h->sumW, nkb, "W_i"));
    const int nblk = ep_epilogue_blocks(P.nk);
    VV10_TRY(h->ensure(h->eblk, sizeof(double) * nblk, "energy partials"));
    VV10_TRY(h->ensure(h->scal, 64, "energy"));
    if (vrho) VV10_CUDA(h, cudaMemsetAsync(vrho, 0, sizeof(double) * P.n, st), "memset vrho");
    if (vgamma) VV10_CUDA(h, cudaMemsetAsync(vgamma, 0, sizeof(double) * P.n, st), "memset vgamma");
    double* escal = static_cast<double*>(h->scal.p);
    const bool fuse = (h->options & VV10_OPT_FUSE_HESSIAN_SUMS) != 0;
    if (fuse) {
        VV10_TRY(h->ensure(h->sumA, nkb, "A_i"));
        VV10_TRY(h->ensure(h->sumB, nkb, "B_i"));
        VV10_TRY(h->ensure(h->sumC, nkb, "C_i"));
    }
    if (P.nk > 0) {
        int ns = 1;
        VV10_TRY(h->run_pairsum(fuse ? MODE_EUWABC : MODE_EUW, fp64, st, &ns));
        if (fuse) {  // A_i, B_i, C_i are the partial buffer's quantities 3..5
            PhaseScope ph(h, PH_PAIR_ABC, st, 1);
            VV10_CUDA(h, launch_abc_epilogue(P, static_cast<double*>(h->part.p) + 3 * static_cast<size_t>(ns) * P.nk_pad,
                                             ns, static_cast<double*>(h->sumA.p),
                                             static_cast<double*>(h->sumB.p),
                                             static_cast<double*>(h->sumC.p), st),
                      "A/B/C epilogue");
        }
        PhaseScope ph(h, PH_EP_EPILOGUE, st, 2);
        VV10_CUDA(h, launch_ep_epilogue(P, static_cast<double*>(h->part.p), ns,
                                        static_cast<double*>(h->sumE.p),
                                        static_cast<double*>(h->sumU.p),
                                        static_cast<double*>(h->sumW.p), vrho, vgamma,
                                        static_cast<double*>(h->eblk.p),
                                        static_cast<int*>(h->dev_err.p), st),
                  "energy epilogue");
        VV10_CUDA(h, launch_sum_blocks(static_cast<double*>(h->eblk.p), nblk, escal, st),
                  "energy sum");
    } else {
        VV10_CUDA(h, cudaMemsetAsync(escal, 0, sizeof(double), st), "zero energy");
    }
    h->have_euw = true;
    h->have_abc = fuse && P.nk > 0;
    h->abc_fp64 = fp64;
    h->euw_fp64 = fp64;
    if (energy) {
        double* he = reinterpret_cast<double*>(h->h_pinned) + 2;
        VV10_CUDA(h, cudaMemcpyAsync(he, escal, sizeof(double), cudaMemcpyDeviceToHost, st),
                  "read energy");
        VV10_TRY(h->check_device_errors(st));  // synchronises
        *energy = *he;
    }
    return VV10_OK;
}

vv10_status vv10_weight_grad(vv10_handle h, double* dEdw, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (!h->have_euw) {
        h->set_error("vv10_energy_potential must be called first");
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    if (!device_ptr_ok(dEdw, h->device) || !aligned(dEdw, 8)) {
        h->set_error("dEdw must be an 8-byte aligned device pointer");
        return VV10_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    VV10_CUDA(h, cudaMemsetAsync(dEdw, 0, sizeof(double) * h->P.n, st), "memset dEdw");
    VV10_CUDA(h, launch_weight_grad(h->P, static_cast<double*>(h->sumE.p), dEdw, st),
              "weight gradient");
    return VV10_OK;
}

vv10_status vv10_nuclear_gradient(vv10_handle h, int32_t P_dir, const double* rho_t,
                                  const double* grad_rho_t, const double* w_t, double* out,
                                  void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (!h->have_euw) {
        h->set_error("vv10_energy_potential must be called first");
        return VV10_ERR_INVALID_ARG;
    }
    if (P_dir < 1 || P_dir > VV10_MAX_TRIALS) {
        h->set_error("P must be in [1, VV10_MAX_TRIALS]");
        return P_dir < 1 ? VV10_ERR_INVALID_ARG : VV10_ERR_UNSUPPORTED;
    }
    if ((rho_t != nullptr) != (grad_rho_t != nullptr) || (!rho_t && !w_t)) {
        h->set_error("give rho_t with grad_rho_t, w_t, or both");
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    const void* ptrs[] = {rho_t, grad_rho_t, w_t, out};
    for (const void* q : ptrs)
        if (q && (!device_ptr_ok(q, h->device) || !aligned(q, 8))) {
            h->set_error("arrays must be 8-byte aligned device pointers");
            return VV10_ERR_INVALID_ARG;
        }
    if (!out) {
        h->set_error("out is required");
        return VV10_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t np = static_cast<size_t>(P_dir) * static_cast<size_t>(ngrad_blocks(h->P.nk));
    VV10_TRY(h->ensure(h->ngpart, sizeof(double) * np, "nuclear-gradient partials"));
    PhaseScope ph(h, PH_NUCLEAR_GRADIENT, st, h->P.nk > 0 ? 2 : 0);
    VV10_CUDA(h, launch_nuclear_gradient(h->P, static_cast<double*>(h->sumE.p),
                                         static_cast<double*>(h->sumU.p), static_cast<double*>(h->sumW.p),
                                         P_dir, rho_t, grad_rho_t, w_t,
                                         static_cast<double*>(h->ngpart.p), out, st),
              "nuclear gradient terms");
    return VV10_OK;
}

vv10_status vv10_nuclear_hessian(vv10_handle h, vv10_precision prec, const double* rho_a,
                                 const double* grad_rho_a, const double* rho_ab,
                                 const double* grad_rho_ab, const double* w_a, const double* w_ab,
                                 double* H, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (!precision_known(prec)) {
        h->set_error("unknown precision %d", static_cast<int>(prec));
        return VV10_ERR_INVALID_ARG;
    }
    if (h->P.n_atom < 1) {
        h->set_error("the nuclear Hessian needs atom_of_point at prepare time");
        return VV10_ERR_INVALID_ARG;
    }
    const int32_t np = 3 * h->P.n_atom;
    if (np > VV10_MAX_TRIALS) {
        h->set_error("3 n_atom must not exceed VV10_MAX_TRIALS");
        return VV10_ERR_UNSUPPORTED;
    }
    VV10_TRY(h->bind());
    const void* ptrs[] = {rho_a, grad_rho_a, rho_ab, grad_rho_ab, w_a, w_ab, H};
    for (const void* q : ptrs)
        if (!q || !device_ptr_ok(q, h->device) || !aligned(q, 8)) {
            h->set_error("every array must be an 8-byte aligned device pointer");
            return VV10_ERR_INVALID_ARG;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = h->P.n;
    const size_t pn = static_cast<size_t>(np) * static_cast<size_t>(n > 0 ? n : 1);
    const size_t na2 = static_cast<size_t>(h->P.n_atom) * h->P.n_atom * 9;
    const size_t nparts = static_cast<size_t>(np) * np * nhess_blocks(h->P.nk);
    // scratch: f^rho, f^gamma [n] | f^{rho,a}, f^{gamma,a}, E/U/W^{aw} [P][n] | E/U/W^{a,gr}
    // [3][n][P] | E^{AB}_{gr,gr} | block partials
    const size_t nn = static_cast<size_t>(n > 0 ? n : 1);
    const size_t total = 2 * nn + 5 * pn + 3 * pn + na2 + nparts;
    VV10_TRY(h->ensure(h->nhess, sizeof(double) * total, "nuclear-Hessian scratch"));
    double* base = static_cast<double*>(h->nhess.p);
    double* vr = base;
    double* vg = vr + nn;
    double* fr = vg + nn;
    double* fg = fr + pn;
    double* Ew = fg + pn;
    double* Uw = Ew + pn;
    double* Ww = Uw + pn;
    double* euw = Ww + pn;
    double* Hgg = euw + 3 * pn;
    double* part = Hgg + na2;
    // the pair sums, each from this library's own entry point in the requested precision
    VV10_TRY(vv10_energy_potential(h, prec, nullptr, vr, vg, stream));
    VV10_TRY(vv10_hessian_contract(h, prec, np, rho_a, grad_rho_a, fr, fg, stream));
    VV10_TRY(vv10_weight_response(h, prec, np, w_a, Ew, Uw, Ww, stream));
    VV10_TRY(vv10_coord_grad(h, prec, nullptr, nullptr, euw, stream));
    VV10_TRY(vv10_coord_hessian(h, prec, Hgg, nullptr, stream));
    NucHessIn in;
    in.P = np;
    in.rho_a = rho_a;
    in.grad_rho_a = grad_rho_a;
    in.rho_ab = rho_ab;
    in.grad_rho_ab = grad_rho_ab;
    in.w_a = w_a;
    in.w_ab = w_ab;
    in.f_rho_a = fr;
    in.f_gamma_a = fg;
    in.E_w = Ew;
    in.U_w = Uw;
    in.W_w = Ww;
    in.EUW_gr = euw;
    in.vrho = vr;
    in.vgamma = vg;
    in.sumE = static_cast<const double*>(h->sumE.p);
    PhaseScope ph(h, PH_NUCLEAR_GRADIENT, st, 2);
    VV10_CUDA(h, launch_nuclear_hessian(h->P, in, Hgg, part, H, st), "nuclear Hessian assembly");
    return VV10_OK;
}

vv10_status vv10_hessian_vector_product(vv10_handle h, vv10_precision prec, int32_t P_trials,
                                        const double* rho_t, const double* grad_rho_t,
                                        double* hv_rho, double* hv_grad, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (!h->have_euw) {
        h->set_error("vv10_energy_potential must be called first (it provides U_i, W_i)");
        return VV10_ERR_INVALID_ARG;
    }
    if (P_trials < 1 || P_trials > VV10_MAX_TRIALS) {
        h->set_error("P must be in [1, VV10_MAX_TRIALS]");
        return P_trials < 1 ? VV10_ERR_INVALID_ARG : VV10_ERR_UNSUPPORTED;
    }
    if (!precision_known(prec)) {
        h->set_error("unknown precision %d", static_cast<int>(prec));
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    const void* ptrs[] = {rho_t, grad_rho_t, hv_rho, hv_grad};
    for (const void* q : ptrs)
        if (!device_ptr_ok(q, h->device) || !aligned(q, 8)) {
            h->set_error("trial and output arrays must be 8-byte aligned device pointers");
            return VV10_ERR_INVALID_ARG;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t pn = static_cast<size_t>(P_trials) * static_cast<size_t>(h->P.n);
    VV10_TRY(h->ensure(h->hvp_fr, sizeof(double) * pn, "Hessian-vector product scratch"));
    VV10_TRY(h->ensure(h->hvp_fg, sizeof(double) * pn, "Hessian-vector product scratch"));
    double* fr = static_cast<double*>(h->hvp_fr.p);
    double* fg = static_cast<double*>(h->hvp_fg.p);
    VV10_TRY(h->hessian(prec, P_trials, rho_t, grad_rho_t, fr, fg, st));
    VV10_CUDA(h, cudaMemsetAsync(hv_rho, 0, sizeof(double) * pn, st), "memset hv_rho");
    VV10_CUDA(h, cudaMemsetAsync(hv_grad, 0, 3 * sizeof(double) * pn, st), "memset hv_grad");
    PhaseScope ph(h, PH_HESS_EPILOGUE, st, 1);
    VV10_CUDA(h, launch_hvp_assemble(h->P, P_trials, static_cast<double*>(h->sumW.p), fr, fg,
                                     grad_rho_t, hv_rho, hv_grad, st),
              "Hessian-vector product");
    return VV10_OK;
}

vv10_status vv10_hessian_contract(vv10_handle h, vv10_precision prec, int32_t P_trials,
                                  const double* rho_t, const double* grad_rho_t,
                                  double* f_rho_t, double* f_gamma_t, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (!h->have_euw) {
        h->set_error("vv10_energy_potential must be called first (it provides U_i, W_i)");
        return VV10_ERR_INVALID_ARG;
    }
    if (P_trials < 1 || P_trials > VV10_MAX_TRIALS) {
        h->set_error("P must be in [1, VV10_MAX_TRIALS]");
        return P_trials < 1 ? VV10_ERR_INVALID_ARG : VV10_ERR_UNSUPPORTED;
    }
    if (!precision_known(prec)) {
        h->set_error("unknown precision %d", static_cast<int>(prec));
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    const void* ptrs[] = {rho_t, grad_rho_t, f_rho_t, f_gamma_t};
    for (const void* q : ptrs)
        if (!device_ptr_ok(q, h->device) || !aligned(q, 8)) {
            h->set_error("trial and output arrays must be 8-byte aligned device pointers");
            return VV10_ERR_INVALID_ARG;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return h->hessian(prec, P_trials, rho_t, grad_rho_t, f_rho_t, f_gamma_t, st);
}

vv10_status vv10_coord_grad(vv10_handle h, vv10_precision prec, double* grad_points,
                            double* grad_atoms, double* EUW_Bgr, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (!precision_known(prec)) {
        h->set_error("unknown precision %d", static_cast<int>(prec));
        return VV10_ERR_INVALID_ARG;
    }
    if ((grad_atoms || EUW_Bgr) && h->P.n_atom == 0) {
        h->set_error("atom outputs need atom_of_point at prepare time");
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    void* outs[] = {grad_points, grad_atoms, EUW_Bgr};
    for (void* q : outs)
        if (q && (!device_ptr_ok(q, h->device) || !aligned(q, 8))) {
            h->set_error("outputs must be 8-byte aligned device pointers");
            return VV10_ERR_INVALID_ARG;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool fp64 = precision_fp64(prec);
    PointsDev& P = h->P;
    if (grad_points) VV10_CUDA(h, cudaMemsetAsync(grad_points, 0, sizeof(double) * 3 * P.n, st), "memset");
    if (grad_atoms) VV10_CUDA(h, cudaMemsetAsync(grad_atoms, 0, sizeof(double) * 3 * P.n_atom, st), "memset");
    if (EUW_Bgr)
        VV10_CUDA(h, cudaMemsetAsync(EUW_Bgr, 0, sizeof(double) * 9 * P.n * P.n_atom, st), "memset");
    if (P.nk == 0) return VV10_OK;
    if (EUW_Bgr) {
        // one pass gives the atom-resolved terms and, summed over atoms, the point gradient
        const bool want_grad = grad_points || grad_atoms;
        if (want_grad) VV10_TRY(h->ensure(h->gk, sizeof(double) * 3 * h->soa_ld, "kept gradient"));
        {
            PhaseScope ph(h, PH_ATOM_RESOLVED, st, 1);
            VV10_CUDA(h, launch_atom_resolved(P, fp64, EUW_Bgr,
                                              want_grad ? static_cast<double*>(h->gk.p) : nullptr,
                                              grad_points, nullptr, static_cast<int*>(h->dev_err.p), st),
                      "atom-resolved terms");
        }
        if (grad_atoms) {
            PhaseScope ph(h, PH_GRAD_EPILOGUE, st, 1);
            VV10_CUDA(h, launch_atom_sums(P, static_cast<double*>(h->gk.p), grad_atoms, st),
                      "atom sums");
        }
        return VV10_OK;
    }
    if (grad_points || grad_atoms) {
        int ns = 1;
        VV10_TRY(h->run_pairsum(MODE_GRAD, fp64, st, &ns));
        VV10_TRY(h->ensure(h->gk, sizeof(double) * 3 * h->soa_ld, "kept gradient"));
        PhaseScope ph(h, PH_GRAD_EPILOGUE, st, grad_atoms ? 2 : 1);
        VV10_CUDA(h, launch_grad_epilogue(P, static_cast<double*>(h->part.p), ns,
                                          static_cast<double*>(h->gk.p), grad_points, st),
                  "gradient epilogue");
        if (grad_atoms)
            VV10_CUDA(h, launch_atom_sums(P, static_cast<double*>(h->gk.p), grad_atoms, st),
                      "atom sums");
    }
    return VV10_OK;
}

vv10_status vv10_coord_hessian(vv10_handle h, vv10_precision prec, double* E_grgr,
                               double* D_points, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (!precision_known(prec)) {
        h->set_error("unknown precision %d", static_cast<int>(prec));
        return VV10_ERR_INVALID_ARG;
    }
    if (h->P.n_atom == 0) {
        h->set_error("the grid-grid Hessian needs atom_of_point at prepare time");
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    void* outs[] = {E_grgr, D_points};
    for (void* q : outs)
        if (q && (!device_ptr_ok(q, h->device) || !aligned(q, 8))) {
            h->set_error("outputs must be 8-byte aligned device pointers");
            return VV10_ERR_INVALID_ARG;
        }
    if (!E_grgr && !D_points) return VV10_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool fp64 = precision_fp64(prec);
    PointsDev& P = h->P;
    const size_t na = static_cast<size_t>(P.n_atom);
    // chunk offsets, per-task partials, then room for the blocks when only D_i^B is asked for
    const size_t n_off = (na + 1 + 1) & ~static_cast<size_t>(1);  // keeps part 16-byte aligned
    const size_t n_part = 6 * na * static_cast<size_t>(coord_hessian_chunk_bound(P.nk, P.n_atom));
    VV10_TRY(h->ensure(h->chpart, sizeof(double) * (n_off + n_part + (E_grgr ? 0 : 9 * na * na)),
                       "grid-grid Hessian partials"));
    int64_t* off = static_cast<int64_t*>(h->chpart.p);
    double* part = static_cast<double*>(h->chpart.p) + n_off;
    double* E = E_grgr ? E_grgr : part + n_part;
    if (D_points)
        VV10_CUDA(h, cudaMemsetAsync(D_points, 0, sizeof(double) * 9 * na * P.n, st), "memset");
    PhaseScope ph(h, PH_COORD_HESSIAN, st, (P.nk > 0 && P.n_atom > 1) ? 3 : 2);
    VV10_CUDA(h, launch_coord_hessian(P, fp64, off, part, E, D_points, st), "grid-grid Hessian");
    return VV10_OK;
}

vv10_status vv10_weight_response(vv10_handle h, vv10_precision prec, int32_t P,
                                 const double* w_t, double* E_t, double* U_t, double* W_t,
                                 void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (!precision_known(prec)) {
        h->set_error("unknown precision %d", static_cast<int>(prec));
        return VV10_ERR_INVALID_ARG;
    }
    if (P < 1 || P > VV10_MAX_TRIALS) {
        h->set_error("P must be in [1, VV10_MAX_TRIALS]");
        return P < 1 ? VV10_ERR_INVALID_ARG : VV10_ERR_UNSUPPORTED;
    }
    VV10_TRY(h->bind());
    if (!device_ptr_ok(w_t, h->device) || !aligned(w_t, 8)) {
        h->set_error("w_t must be an 8-byte aligned device pointer");
        return VV10_ERR_INVALID_ARG;
    }
    void* outs[] = {E_t, U_t, W_t};
    for (void* q : outs)
        if (q && (!device_ptr_ok(q, h->device) || !aligned(q, 8))) {
            h->set_error("outputs must be 8-byte aligned device pointers");
            return VV10_ERR_INVALID_ARG;
        }
    if (!E_t && !U_t && !W_t) return VV10_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PointsDev& Pd = h->P;
    const size_t pn = static_cast<size_t>(P) * static_cast<size_t>(Pd.n);
    for (void* q : outs)
        if (q) VV10_CUDA(h, cudaMemsetAsync(q, 0, sizeof(double) * pn, st), "memset");
    if (Pd.nk == 0) return VV10_OK;
    VV10_TRY(h->ensure(h->wdir, sizeof(double) * static_cast<size_t>(P) * Pd.nk_pad,
                       "weight directions"));
    double* yk = static_cast<double*>(h->wdir.p);
    if (!precision_fp64(prec) && P > 4) {
        // tensor cores (below 5 directions a 32-wide MMA is mostly padding)
        int ng = 0, ppad = 0;
        weight_tc_groups(P, &ng, &ppad);
        const int32_t rows = ng * ppad;
        const size_t nsplit = static_cast<size_t>(rows) * static_cast<size_t>(Pd.nk_pad);
        VV10_TRY(h->ensure(h->wsplit, 2 * sizeof(float) * nsplit, "weight direction split"));
        float* yh = static_cast<float*>(h->wsplit.p);
        PhaseScope ph(h, PH_WEIGHT_RESPONSE, st, 3);
        VV10_CUDA(h, launch_weight_dirs(Pd, P, w_t, yk, st), "weight directions");
        VV10_CUDA(h, launch_weight_split(yk, P, rows, Pd.nk_pad, yh, yh + nsplit, st),
                  "weight direction split");
        VV10_CUDA(h, launch_weight_tc(Pd, P, yh, yh + nsplit, rows, E_t, U_t, W_t, h->n_sm,
                                      static_cast<int*>(h->dev_err.p), st),
                  "weight-derivative sums (tensor cores)");
        return VV10_OK;
    }
    PhaseScope ph(h, PH_WEIGHT_RESPONSE, st, 2);
    VV10_CUDA(h, launch_weight_dirs(Pd, P, w_t, yk, st), "weight directions");
    VV10_CUDA(h, launch_weight_response(Pd, precision_fp64(prec), P, yk, E_t, U_t, W_t, st),
              "weight-derivative sums");
    return VV10_OK;
}

vv10_status vv10_energy(vv10_handle h, vv10_precision prec, double* energy, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (!precision_known(prec)) {
        h->set_error("unknown precision %d", static_cast<int>(prec));
        return VV10_ERR_INVALID_ARG;
    }
    if (!energy) {
        h->set_error("energy must be a host pointer");
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool fp64 = precision_fp64(prec);
    const int grid = energy_half_grid(fp64, h->n_sm);
    VV10_TRY(h->ensure(h->ehalf, sizeof(double) * (static_cast<size_t>(grid) + 8), "energy partials"));
    double* dev_e = static_cast<double*>(h->ehalf.p) + grid;  // after the per-CTA totals
    {
        PhaseScope ph(h, PH_ENERGY_HALF, st, h->P.nk > 0 ? 2 : 0);
        VV10_CUDA(h, launch_energy_half(h->P, fp64, grid, static_cast<double*>(h->ehalf.p), dev_e, st),
                  "energy");
    }
    double* he = reinterpret_cast<double*>(h->h_pinned) + 2;
    VV10_CUDA(h, cudaMemcpyAsync(he, dev_e, sizeof(double), cudaMemcpyDeviceToHost, st), "read energy");
    VV10_TRY(h->check_device_errors(st));  // synchronises
    *energy = *he;
    return VV10_OK;
}

// Shared part of vv10_fock_matrix and vv10_orbital_hessian.
static vv10_status ao_assemble(vv10_handle h, int32_t nbf, const double* phi, const double* dphi,
                               int32_t n_ch, const double* s, const double* fg, const double* vg,
                               const double* gt, double* out, void* stream) {
    PointsDev& P = h->P;
    if (nbf < 1 || nbf > VV10_MAX_BASIS) {
        h->set_error("nbf must be in [1, VV10_MAX_BASIS]");
        return nbf < 1 ? VV10_ERR_INVALID_ARG : VV10_ERR_UNSUPPORTED;
    }
    const void* ins[] = {phi, dphi, s, fg, out};
    for (const void* q : ins)
        if (!device_ptr_ok(q, h->device) || !aligned(q, 8)) {
            h->set_error("arrays must be 8-byte aligned device pointers");
            return VV10_ERR_INVALID_ARG;
        }
    if ((vg != nullptr) != (gt != nullptr) ||
        (vg && (!device_ptr_ok(vg, h->device) || !device_ptr_ok(gt, h->device)))) {
        h->set_error("vgamma and grad_rho_t must be device pointers");
        return VV10_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nk = static_cast<size_t>(P.nk > 0 ? P.nk : 1);
    const int64_t chunk = ao_channels_per_chunk(P.nk, nbf, n_ch, size_t(1) << 30);
    VV10_TRY(h->ensure(h->aophik, sizeof(double) * nk * nbf, "gathered basis values"));
    VV10_TRY(h->ensure(h->aoz, sizeof(double) * nk * nbf * chunk, "assembly operand"));
    VV10_TRY(h->ensure(h->aom, sizeof(double) * static_cast<size_t>(nbf) * nbf * chunk, "assembly products"));
    const size_t gw = ao_gemm_work_elems(nbf, chunk, h->n_sm);
    VV10_TRY(h->ensure(h->aogw, sizeof(double) * gw, "assembly product partials"));
    const AoGemm g{static_cast<double*>(h->aogw.p), gw, h->n_sm};
    PhaseScope ph(h, PH_AO_ASSEMBLY, st, P.nk > 0 ? 1 + 4 * static_cast<int>((n_ch + chunk - 1) / chunk) : 0);
    VV10_CUDA(h, launch_ao_assemble(P, g, nbf, phi, dphi, n_ch, s, fg, vg, gt, chunk,
                                    static_cast<double*>(h->aophik.p), static_cast<double*>(h->aoz.p),
                                    static_cast<double*>(h->aom.p), out, st),
              "AO assembly");
    return VV10_OK;
}

vv10_status vv10_fock_matrix(vv10_handle h, int32_t nbf, const double* phi, const double* grad_phi,
                             const double* vrho, const double* vgamma, double* F, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    VV10_TRY(h->bind());
    return ao_assemble(h, nbf, phi, grad_phi, 1, vrho, vgamma, nullptr, nullptr, F, stream);
}

vv10_status vv10_orbital_hessian(vv10_handle h, int32_t nbf, const double* phi,
                                 const double* grad_phi, int32_t P_trials, const double* f_rho_t,
                                 const double* f_gamma_t, const double* grad_rho_t,
                                 const double* vgamma, double* G, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (P_trials < 1 || P_trials > VV10_MAX_TRIALS) {
        h->set_error("P must be in [1, VV10_MAX_TRIALS]");
        return P_trials < 1 ? VV10_ERR_INVALID_ARG : VV10_ERR_UNSUPPORTED;
    }
    if (!vgamma || !grad_rho_t) {
        h->set_error("vgamma and grad_rho_t are required");
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    return ao_assemble(h, nbf, phi, grad_phi, P_trials, f_rho_t, f_gamma_t, vgamma, grad_rho_t, G,
                       stream);
}

vv10_status vv10_fock_derivative(vv10_handle h, int32_t nbf, const double* phi,
                                 const double* grad_phi, const double* hess_phi,
                                 const int32_t* bf_atom, const double* vrho, const double* vgamma,
                                 const double* f_rho_a, const double* f_gamma_a,
                                 const double* grad_rho_a, const double* w_a, const double* E_w,
                                 const double* U_w, const double* W_w, const double* EUW_gr,
                                 double* FA, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    PointsDev& P = h->P;
    if (P.n_atom == 0) {
        h->set_error("the nuclear derivative of the Fock matrix needs atom_of_point at prepare time");
        return VV10_ERR_INVALID_ARG;
    }
    if (nbf < 1 || nbf > VV10_MAX_BASIS) {
        h->set_error("nbf must be in [1, VV10_MAX_BASIS]");
        return nbf < 1 ? VV10_ERR_INVALID_ARG : VV10_ERR_UNSUPPORTED;
    }
    const void* ins[] = {phi, grad_phi, hess_phi, vrho, vgamma, f_rho_a, f_gamma_a, grad_rho_a,
                         w_a, E_w, U_w, W_w, EUW_gr, FA};
    for (const void* q : ins)
        if (!device_ptr_ok(q, h->device) || !aligned(q, 8)) {
            h->set_error("arrays must be 8-byte aligned device pointers");
            return VV10_ERR_INVALID_ARG;
        }
    if (!device_ptr_ok(bf_atom, h->device) || !aligned(bf_atom, 4)) {
        h->set_error("bf_atom must be a 4-byte aligned device pointer");
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (stream_capturing(st)) {
        h->set_error("vv10_fock_derivative reads the atom segments on the host and cannot be captured");
        return VV10_ERR_INVALID_ARG;
    }
    const int32_t n_dir = 3 * P.n_atom;
    const size_t nk = static_cast<size_t>(P.nk > 0 ? P.nk : 1);
    const size_t nn = static_cast<size_t>(nbf) * nbf;
    const int64_t chunk = ao_channels_per_chunk(P.nk, nbf, n_dir, size_t(1) << 30);
    VV10_TRY(h->ensure(h->aophik, sizeof(double) * nk * nbf, "gathered basis values"));
    VV10_TRY(h->ensure(h->aoz, sizeof(double) * nk * nbf * chunk, "assembly operand"));
    VV10_TRY(h->ensure(h->aom, sizeof(double) * nn * chunk, "assembly products"));
    VV10_TRY(h->ensure(h->aofa, sizeof(double) * (4 * nk * nbf + 2 * nn), "basis-derivative factors"));
    const size_t gw = ao_gemm_work_elems(nbf, chunk, h->n_sm);
    VV10_TRY(h->ensure(h->aogw, sizeof(double) * gw, "assembly product partials"));
    const AoGemm g{static_cast<double*>(h->aogw.p), gw, h->n_sm};
    std::vector<int64_t> seg(static_cast<size_t>(P.n_atom) + 1);
    VV10_CUDA(h, cudaMemcpyAsync(seg.data(), P.seg, sizeof(int64_t) * seg.size(),
                                 cudaMemcpyDeviceToHost, st), "atom segments");
    VV10_CUDA(h, cudaStreamSynchronize(st), "atom segments");
    FockDerivIn in{nbf, phi, grad_phi, hess_phi, bf_atom, vrho, vgamma, f_rho_a, f_gamma_a,
                   grad_rho_a, w_a, E_w, U_w, W_w, EUW_gr};
    double* fa = static_cast<double*>(h->aofa.p);
    // launches: gather, right factor, per chunk (Z, product, its split sum, symmetrisation),
    // per direction c (left factor, product + split sum, per atom product + split sum and
    // the basis-derivative update)
    const int n_launch =
        P.nk > 0 ? 2 + 4 * static_cast<int>((n_dir + chunk - 1) / chunk) + 3 * (3 + 3 * P.n_atom) : 0;
    PhaseScope ph(h, PH_AO_ASSEMBLY, st, n_launch);
    VV10_CUDA(h, launch_fock_derivative(P, g, in, seg.data(), chunk,
                                        static_cast<double*>(h->aophik.p),
                                        static_cast<double*>(h->aoz.p),
                                        static_cast<double*>(h->aom.p), fa, fa + 4 * nk * nbf, FA,
                                        st),
              "nuclear derivative of the Fock matrix");
    return VV10_OK;
}

}  // extern "C"

// The single pass over the pairs of vv10_evaluate.  With EUW_Bgr the atom-resolved kernel
// forms the six row sums (E/U/W and A/B/C), the atom-resolved terms and the point gradient;
// without it the pair-sum mode MODE_EUWABCG forms the six row sums and the gradient.  Then
// the E/U/W and A/B/C epilogues (energy, f^rho, f^gamma), the gradient epilogue and the atom
// sums.  Leaves the row sums cached as the energy call would.
static vv10_status evaluate_single_pass(vv10_handle h, bool fp64, double* vrho, double* vgamma,
                                        double* grad_points, double* grad_atoms, double* EUW_Bgr,
                                        cudaStream_t st) {
    PointsDev& P = h->P;
    const bool resolved = (EUW_Bgr != nullptr);
    const size_t nkb = sizeof(double) * static_cast<size_t>(h->soa_ld);
    DevBuf* sums[] = {&h->sumE, &h->sumU, &h->sumW, &h->sumA, &h->sumB, &h->sumC};
    for (DevBuf* b : sums) VV10_TRY(h->ensure(*b, nkb, "row sums"));
    const int nblk = ep_epilogue_blocks(P.nk);
    VV10_TRY(h->ensure(h->eblk, sizeof(double) * nblk, "energy partials"));
    VV10_TRY(h->ensure(h->scal, 64, "energy"));
    VV10_TRY(h->ensure(h->gk, 3 * nkb, "kept gradient"));
    if (resolved) VV10_TRY(h->ensure(h->part, 6 * nkb, "pair-sum partials"));
    if (vrho) VV10_CUDA(h, cudaMemsetAsync(vrho, 0, sizeof(double) * P.n, st), "memset vrho");
    if (vgamma) VV10_CUDA(h, cudaMemsetAsync(vgamma, 0, sizeof(double) * P.n, st), "memset vgamma");
    if (grad_points) VV10_CUDA(h, cudaMemsetAsync(grad_points, 0, sizeof(double) * 3 * P.n, st), "memset");
    if (grad_atoms) VV10_CUDA(h, cudaMemsetAsync(grad_atoms, 0, sizeof(double) * 3 * P.n_atom, st), "memset");
    if (resolved)
        VV10_CUDA(h, cudaMemsetAsync(EUW_Bgr, 0, sizeof(double) * 9 * P.n * P.n_atom, st), "memset");
    double* escal = static_cast<double*>(h->scal.p);
    double* gk = static_cast<double*>(h->gk.p);
    int* err = static_cast<int*>(h->dev_err.p);
    if (P.nk > 0) {
        int ns = 1;
        if (resolved) {
            PhaseScope ph(h, PH_ATOM_RESOLVED, st, 1);
            VV10_CUDA(h, launch_atom_resolved(P, fp64, EUW_Bgr, gk, grad_points,
                                              static_cast<double*>(h->part.p), err, st),
                      "fused pair pass");
        } else {
            VV10_TRY(h->run_pairsum(MODE_EUWABCG, fp64, st, &ns));
        }
        double* part = static_cast<double*>(h->part.p);
        const size_t blk = static_cast<size_t>(ns) * static_cast<size_t>(P.nk_pad);
        {
            PhaseScope ph(h, PH_EP_EPILOGUE, st, (resolved && grad_atoms) ? 4 : 3);
            VV10_CUDA(h, launch_ep_epilogue(P, part, ns, static_cast<double*>(h->sumE.p),
                                            static_cast<double*>(h->sumU.p),
                                            static_cast<double*>(h->sumW.p), vrho, vgamma,
                                            static_cast<double*>(h->eblk.p), err, st),
                      "energy epilogue");
            VV10_CUDA(h, launch_sum_blocks(static_cast<double*>(h->eblk.p), nblk, escal, st), "energy sum");
            VV10_CUDA(h, launch_abc_epilogue(P, part + 3 * blk, ns, static_cast<double*>(h->sumA.p),
                                             static_cast<double*>(h->sumB.p),
                                             static_cast<double*>(h->sumC.p), st),
                      "A/B/C epilogue");
            if (resolved && grad_atoms)
                VV10_CUDA(h, launch_atom_sums(P, gk, grad_atoms, st), "atom sums");
        }
        if (!resolved) {
            PhaseScope ph(h, PH_GRAD_EPILOGUE, st, grad_atoms ? 2 : 1);
            VV10_CUDA(h, launch_grad_epilogue(P, part + 6 * blk, ns, gk, grad_points, st),
                      "gradient epilogue");
            if (grad_atoms) VV10_CUDA(h, launch_atom_sums(P, gk, grad_atoms, st), "atom sums");
        }
    } else {
        VV10_CUDA(h, cudaMemsetAsync(escal, 0, sizeof(double), st), "zero energy");
    }
    h->have_euw = true;
    h->euw_fp64 = fp64;
    h->have_abc = P.nk > 0;
    h->abc_fp64 = fp64;
    return VV10_OK;
}

extern "C" {

vv10_status vv10_evaluate(vv10_handle h, vv10_precision prec, int32_t P_trials,
                          const double* rho_t, const double* grad_rho_t, double* energy,
                          double* vrho, double* vgamma, double* f_rho_t, double* f_gamma_t,
                          double* grad_points, double* grad_atoms, double* EUW_Bgr,
                          void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    VV10_TRY(h->require_prepared());
    if (!precision_known(prec)) {
        h->set_error("unknown precision %d", static_cast<int>(prec));
        return VV10_ERR_INVALID_ARG;
    }
    if (P_trials < 0 || P_trials > VV10_MAX_TRIALS) {
        h->set_error("P must be in [0, VV10_MAX_TRIALS]");
        return P_trials < 0 ? VV10_ERR_INVALID_ARG : VV10_ERR_UNSUPPORTED;
    }
    if (P_trials > 0 && prec == VV10_MIXED_BF16X3) {
        h->set_error("the BF16x3 Hessian contraction is not available in this library");
        return VV10_ERR_UNSUPPORTED;
    }
    if ((grad_atoms || EUW_Bgr) && h->P.n_atom == 0) {
        h->set_error("atom outputs need atom_of_point at prepare time");
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    void* outs[] = {vrho, vgamma, grad_points, grad_atoms, EUW_Bgr};
    for (void* q : outs)
        if (q && (!device_ptr_ok(q, h->device) || !aligned(q, 8))) {
            h->set_error("outputs must be 8-byte aligned device pointers");
            return VV10_ERR_INVALID_ARG;
        }
    if (P_trials > 0) {
        const void* ptrs[] = {rho_t, grad_rho_t, f_rho_t, f_gamma_t};
        for (const void* q : ptrs)
            if (!device_ptr_ok(q, h->device) || !aligned(q, 8)) {
                h->set_error("trial and output arrays must be 8-byte aligned device pointers");
                return VV10_ERR_INVALID_ARG;
            }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool fp64 = precision_fp64(prec);
    if (EUW_Bgr || grad_points || grad_atoms) {
        VV10_TRY(evaluate_single_pass(h, fp64, vrho, vgamma, grad_points, grad_atoms, EUW_Bgr, st));
        if (P_trials > 0) VV10_TRY(h->hessian(prec, P_trials, rho_t, grad_rho_t, f_rho_t, f_gamma_t, st));
    } else {
        // the energy call, with the A/B/C sums formed in its pass when the contraction follows
        const int saved = h->options;
        if (P_trials > 0) h->options |= VV10_OPT_FUSE_HESSIAN_SUMS;
        vv10_status s = vv10_energy_potential(h, prec, nullptr, vrho, vgamma, stream);
        h->options = saved;
        VV10_TRY(s);
        if (P_trials > 0) VV10_TRY(h->hessian(prec, P_trials, rho_t, grad_rho_t, f_rho_t, f_gamma_t, st));
    }
    if (energy) {
        double* he = reinterpret_cast<double*>(h->h_pinned) + 2;
        VV10_CUDA(h, cudaMemcpyAsync(he, h->scal.p, sizeof(double), cudaMemcpyDeviceToHost, st),
                  "read energy");
        VV10_TRY(h->check_device_errors(st));  // synchronises
        *energy = *he;
    }
    return VV10_OK;
}

vv10_status vv10_profile_enable(vv10_handle h, int on) {
    VV10_CHECK_HANDLE(h);
    h->prof_on = (on != 0);
    return VV10_OK;
}

vv10_status vv10_profile_read(vv10_handle h, int n, double* ms, int64_t* launches) {
    VV10_CHECK_HANDLE(h);
    if (n < 0 || n > VV10_N_PHASES) return VV10_ERR_INVALID_ARG;
    VV10_TRY(h->bind());
    VV10_CUDA(h, cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    double acc[PH_COUNT] = {0};
    for (ProfRec& r : h->prof) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) acc[r.phase] += t;
        else cudaGetLastError();
        h->event_pool.push_back(r.a);
        h->event_pool.push_back(r.b);
    }
    h->prof.clear();
    for (int k = 0; k < n; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = h->launches[k];
    }
    for (int k = 0; k < PH_COUNT; ++k) h->launches[k] = 0;
    return VV10_OK;
}

const char* vv10_profile_phase_name(int phase) {
    static const char* names[PH_COUNT] = {
        "prepare", "pair_sums_EUW", "energy_epilogue", "pair_sums_ABC", "trial_prep",
        "contraction_fp64", "contraction_tensor_core", "hessian_epilogue", "pair_sums_grad",
        "grad_epilogue", "atom_resolved", "coord_hessian", "weight_response", "energy_half", "ao_assembly", "nuclear_gradient"};
    return (phase >= 0 && phase < PH_COUNT) ? names[phase] : "unknown";
}

vv10_status vv10_debug_inject(vv10_handle h, int what, int64_t value) {
    VV10_CHECK_HANDLE(h);
    switch (what) {
        case VV10_DEBUG_FAIL_ALLOC:
            h->debug_fail_alloc = static_cast<int>(value);
            return VV10_OK;
        case VV10_DEBUG_STALL_COPY:
            h->debug_stall = static_cast<int>(value);
            return VV10_OK;
        default:
            return VV10_ERR_INVALID_ARG;
    }
}

vv10_status vv10_set_tiles(vv10_handle h, int what, int rows_per_thread, int n_split) {
    VV10_CHECK_HANDLE(h);
    if (what < 0 || what > 8 || rows_per_thread < 0 || n_split < 0) return VV10_ERR_INVALID_ARG;
    if (what == 8) {  // widest trial group of the tensor-core contraction; j-chunk size
        if (rows_per_thread != 0 && (rows_per_thread < 32 || rows_per_thread > 192)) {
            h->set_error("the trial-group width must be 0 or in [32, 192]");
            return VV10_ERR_INVALID_ARG;
        }
        if (n_split != 0 && (n_split < 4 || n_split > 96)) {
            h->set_error("the j-chunk size must be 0 or in [4, 96] MB");
            return VV10_ERR_INVALID_ARG;
        }
        h->tc_cap_manual = rows_per_thread;
        h->tc_chunk_mb = n_split;
        h->batch.tc_classes.clear();  // rebuild the batch layouts with the new width
        h->batch.f16_classes.clear();
        h->batch_drop_graph();
        return VV10_OK;
    }
    const bool fp64 = what >= 6 ? what == 7 : what >= 3;
    const int max_rpt = fp64 ? 2 : 4;
    if (rows_per_thread != 0 && rows_per_thread != 1 && rows_per_thread != 2 &&
        rows_per_thread != max_rpt) {
        h->set_error("rows_per_thread must be 0, 1, 2 or %d", max_rpt);
        return VV10_ERR_INVALID_ARG;
    }
    TileOverride& o = what >= 6 ? h->batch_over[what - 6] : h->overrides[what % 3 + kPairModes * (what >= 3)];
    o = TileOverride{};
    o.mode = what >= 6 ? 0 : what % 3;
    o.fp64 = what >= 6 ? what == 7 : what >= 3;
    o.active = rows_per_thread > 0;
    o.manual = o.active;
    o.rows_per_thread = rows_per_thread;
    o.n_split = n_split;
    h->batch_drop_graph();  // a recorded batch graph holds the old tiles
    return VV10_OK;
}

vv10_status vv10_get_tiles(vv10_handle h, int what, int* rows_per_thread, int* n_split) {
    VV10_CHECK_HANDLE(h);
    if (what < 0 || what > 8 || !rows_per_thread || !n_split) return VV10_ERR_INVALID_ARG;
    if (what == 8) {
        *rows_per_thread = h->tc_cap_manual > 0 ? h->tc_cap_manual : h->tc_cap_last;
        *n_split = h->tc_chunk_mb > 0 ? h->tc_chunk_mb
                                      : static_cast<int>(hess_f16_default_chunk_bytes() >> 20);
    } else if (what >= 6) {
        h->batch_tiles(what == 7, rows_per_thread, n_split);
    } else {
        const TileChoice t = h->tiles_for(what % 3, what >= 3);
        *rows_per_thread = t.rows_per_thread;
        *n_split = t.n_split;
    }
    return VV10_OK;
}

vv10_status vv10_set_options(vv10_handle h, int flags) {
    VV10_CHECK_HANDLE(h);
    if (flags & ~VV10_OPT_FUSE_HESSIAN_SUMS) return VV10_ERR_INVALID_ARG;
    h->options = flags;
    return VV10_OK;
}

vv10_status vv10_set_autotune(vv10_handle h, int flags) {
    VV10_CHECK_HANDLE(h);
    if (flags & ~(VV10_TUNE_PAIRSUMS | VV10_TUNE_BATCH | VV10_TUNE_CONTRACTION))
        return VV10_ERR_INVALID_ARG;
    h->autotune = flags;
    return VV10_OK;
}

vv10_status vv10_autotune(vv10_handle h, vv10_precision prec, int what, void* stream) {
    VV10_CHECK_HANDLE(h);
    h->set_error("");
    if (!precision_known(prec))
        return VV10_ERR_INVALID_ARG;
    if (what & ~(VV10_TUNE_PAIRSUMS | VV10_TUNE_BATCH)) {
        h->set_error("vv10_autotune tunes VV10_TUNE_PAIRSUMS and VV10_TUNE_BATCH; the contraction "
                     "width is tuned on first use (vv10_set_autotune)");
        return VV10_ERR_INVALID_ARG;
    }
    VV10_TRY(h->bind());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (stream_capturing(st)) {
        h->set_error("vv10_autotune cannot run while the stream is being captured");
        return VV10_ERR_INVALID_ARG;
    }
    const bool fp64 = precision_fp64(prec);
    if (what & VV10_TUNE_PAIRSUMS) {
        VV10_TRY(h->require_prepared());
        for (int mode = 0; mode < 3; ++mode) VV10_TRY(h->tune_pairsum(mode, fp64, st, true));
        if (h->options & VV10_OPT_FUSE_HESSIAN_SUMS)
            VV10_TRY(h->tune_pairsum(MODE_EUWABC, fp64, st, true));
    }
    if (what & VV10_TUNE_BATCH) {
        if (!h->batch.prepared) {
            h->set_error("vv10_batch_prepare has not been called on this handle");
            return VV10_ERR_INVALID_ARG;
        }
        VV10_TRY(h->tune_batch(fp64, st, true));
    }
    return h->check_device_errors(st);
}

}  // extern "C"
