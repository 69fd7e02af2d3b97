// vv10_energy_potential_noalloc: the energy/potential path for callers that cannot
// allocate device memory -- a host that gave (nearly) all device memory to another
// allocator up front (a preallocating array runtime, a custom arena), or a plug-in that is
// only ever handed buffers and has no allocator of its own to call.
// All of its scratch lives in the file-scope array below, which every GPU that loads
// this library holds (about 11 MB) until the process exits; the call allocates nothing.
// A device-side failure (a non-finite input, a bounded wait that gave up) leaves NaN in
// the energy and in every potential value it writes, so it cannot pass for a result.
//
// It uses the same pair-sum kernel as vv10_energy_potential, but skips the compaction
// step: every one of the n points is a row and a column, and points below the density
// cutoff are given a zero weight-density product so that they add nothing to any sum.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "kernels.hpp"
#include "vv10.h"

namespace vv10 {

constexpr int64_t kNaMaxPoints = VV10_NOALLOC_MAX_POINTS;
constexpr int kNaMaxSplit = 8;
constexpr int64_t kNaPad = ((kNaMaxPoints + kJTile - 1) / kJTile) * kJTile;
// The point and epilogue kernels run n_pad / 256 blocks of 256 threads and the energy has
// n_pad / 256 block partials: whole blocks only while the j tile is a multiple of 256.
static_assert(kJTile % 256 == 0, "n_pad must be a whole number of 256-thread blocks");

// Scratch layout (bytes, every block 256-aligned):
//   r64a, r64b   2 x 32 x kNaPad   FP64 pair records
//   r32a, r32b   2 x 16 x kNaPad   FP32 pair records
//   soa          6 x 8 x kNaPad    w, rho, kappa', omega_rho, omega_gamma, keep flag
//   orig         8 x kNaPad        identity index map
//   part         3 x kNaMaxSplit x 8 x kNaPad   pair-sum partials
//   eblk         8 x kNaPad / 256  energy block partials
//   misc         256               recentring origin, error word
constexpr size_t kNaOffR64a = 0;
constexpr size_t kNaOffR64b = kNaOffR64a + 32 * kNaPad;
constexpr size_t kNaOffR32a = kNaOffR64b + 32 * kNaPad;
constexpr size_t kNaOffR32b = kNaOffR32a + 16 * kNaPad;
constexpr size_t kNaOffSoa = kNaOffR32b + 16 * kNaPad;
constexpr size_t kNaOffOrig = kNaOffSoa + 6 * 8 * kNaPad;
constexpr size_t kNaOffPart = kNaOffOrig + 8 * kNaPad;
constexpr size_t kNaOffEblk = kNaOffPart + 3 * kNaMaxSplit * 8 * kNaPad;
constexpr size_t kNaOffMisc = kNaOffEblk + 8 * (kNaPad / 256);
constexpr size_t kNaBytes = ((kNaOffMisc + 256 + 255) / 256) * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Recentring origin: midpoint of the bounding box of the points that pass the cutoff.
__global__ void __launch_bounds__(1024)
k_na_center(int64_t n, const double* __restrict__ xyz, const double* __restrict__ rho,
            double rho_cut, double* __restrict__ center) {
    __shared__ double sh[6][32];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        if (!(rho[i] >= rho_cut)) continue;
        for (int d = 0; d < 3; ++d) {
            mn[d] = fmin(mn[d], xyz[3 * i + d]);
            mx[d] = fmax(mx[d], xyz[3 * i + d]);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = 0; d < 3; ++d) {
        double a = mn[d], b = mx[d];
        for (int o = 16; o > 0; o >>= 1) {
            a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) {
            sh[d][wid] = a;
            sh[3 + d][wid] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double a = INFINITY, b = -INFINITY;
        for (int w = 0; w < 32; ++w) {
            a = fmin(a, sh[threadIdx.x][w]);
            b = fmax(b, sh[3 + threadIdx.x][w]);
        }
        center[threadIdx.x] = (a <= b) ? 0.5 * (a + b) : 0.0;
    }
}

// Per-point quantities of Sec. II.A for all n points (no compaction); a point below the
// cutoff gets c = 0 (adds nothing as a column) and keep = 0 (zero outputs as a row).
__global__ void __launch_bounds__(256)
k_na_points(int64_t n, int64_t n_pad, const double* __restrict__ xyz, const double* __restrict__ w,
            const double* __restrict__ rho, const double* __restrict__ grad, double b, double C,
            double rho_cut, const double* __restrict__ center, double4* __restrict__ r64a,
            double4* __restrict__ r64b, float4* __restrict__ r32a, float4* __restrict__ r32b,
            double* __restrict__ soa, int64_t* __restrict__ orig, int* __restrict__ err) {
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= n_pad) return;
    double* f = soa;
    if (p < n) {  // a non-finite input is an error, not a point below the cutoff
        bool finite = isfinite(rho[p]) && isfinite(w[p]);
        for (int d = 0; d < 3; ++d) finite = finite && isfinite(xyz[3 * p + d]) && isfinite(grad[3 * p + d]);
        if (!finite) atomicOr(err, DEVERR_BAD_INPUT);
    }
    const bool keep = p < n && rho[p] >= rho_cut;
    if (!keep) {
        const double x = p < n ? xyz[3 * p] : 0.0, y = p < n ? xyz[3 * p + 1] : 0.0,
                     z = p < n ? xyz[3 * p + 2] : 0.0;
        r64a[p] = make_double4(x, y, z, 0.0);
        r64b[p] = make_double4(1.0, 1.0, 0.0, 0.0);
        r32a[p] = make_float4(static_cast<float>(x - center[0]), static_cast<float>(y - center[1]),
                              static_cast<float>(z - center[2]), 0.f);
        r32b[p] = make_float4(1.f, 1.f, 0.f, 0.f);
        for (int k = 0; k < 6; ++k) f[k * n_pad + p] = 0.0;
        orig[p] = p;
        return;
    }
    const double r = rho[p];
    const double gx = grad[3 * p], gy = grad[3 * p + 1], gz = grad[3 * p + 2];
    const double gam = gx * gx + gy * gy + gz * gz;
    const double pi = 3.141592653589793238462643383279502884;
    const double ir = 1.0 / r, ir2 = ir * ir, ir4 = ir2 * ir2;
    const double Q = C * gam * gam * ir4 + (4.0 * pi / 3.0) * r;  // omega^2
    const double Qr = -4.0 * C * gam * gam * ir4 * ir + 4.0 * pi / 3.0;
    const double Qg = 2.0 * C * gam * ir4;
    const double om = sqrt(Q);
    const double ka = b * 1.5 * pi * pow(r / (9.0 * pi), 1.0 / 6.0);
    const double om_r = 0.5 * Qr / om, om_g = 0.5 * Qg / om, ka_r = ka * ir / 6.0;
    const double cj = -1.5 * w[p] * r;
    const double x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
    r64a[p] = make_double4(x, y, z, cj);
    r64b[p] = make_double4(om, ka, r * ka_r, r * om_r);
    r32a[p] = make_float4(static_cast<float>(x - center[0]), static_cast<float>(y - center[1]),
                          static_cast<float>(z - center[2]), static_cast<float>(cj));
    r32b[p] = make_float4(static_cast<float>(om), static_cast<float>(ka),
                          static_cast<float>(r * ka_r), static_cast<float>(r * om_r));
    f[0 * n_pad + p] = w[p];
    f[1 * n_pad + p] = r;
    f[2 * n_pad + p] = ka_r;
    f[3 * n_pad + p] = om_r;
    f[4 * n_pad + p] = om_g;
    f[5 * n_pad + p] = 1.0;
    orig[p] = p;
}

// f^rho, f^gamma and energy block partials; rows below the cutoff get zeros.  If an
// earlier kernel of this call set the error word, every output is NaN instead.
__global__ void __launch_bounds__(256)
k_na_epilogue(int64_t n, int64_t n_pad, double beta, const double* __restrict__ part, int n_split,
              const double* __restrict__ soa, const int* __restrict__ err,
              double* __restrict__ vrho, double* __restrict__ vgamma, double* __restrict__ eblk) {
    __shared__ double sh[8];
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool failed = *err != 0;
    double ei = 0.0;
    if (p < n) {
        double e = 0.0, u = 0.0, wv = 0.0;
        for (int k = 0; k < n_split; ++k) {
            e += part[(0 * static_cast<int64_t>(n_split) + k) * n_pad + p];
            u -= part[(1 * static_cast<int64_t>(n_split) + k) * n_pad + p];
            wv -= part[(2 * static_cast<int64_t>(n_split) + k) * n_pad + p];
        }
        const double keep = soa[5 * n_pad + p];
        const double r = soa[1 * n_pad + p];
        double fr = 0.0, fg = 0.0;
        if (keep != 0.0) {
            fr = beta + e + r * (soa[2 * n_pad + p] * u + soa[3 * n_pad + p] * wv);
            fg = r * soa[4 * n_pad + p] * wv;
            ei = soa[0 * n_pad + p] * r * (beta + 0.5 * e);
        }
        if (failed) fr = fg = NAN;
        if (vrho) vrho[p] = fr;
        if (vgamma) vgamma[p] = fg;
    }
    const double s = block_sum(ei, sh);
    if (threadIdx.x == 0) eblk[blockIdx.x] = failed ? NAN : s;
}

// Per-device address of the scratch array, looked up once (with that device current).
static std::mutex g_na_mutex;
static unsigned char* g_na_addr[64] = {nullptr};

static cudaError_t na_scratch(int device, unsigned char** out) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_addr[device] = static_cast<unsigned char*>(ptr);
    }
    *out = g_na_addr[device];
    return cudaSuccess;
}

static bool na_device_ptr(const void* p, int device) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (reinterpret_cast<uintptr_t>(p) % 8) return false;
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == device);
}

}  // namespace vv10

using namespace vv10;

extern "C" vv10_status vv10_energy_potential_noalloc(int64_t n, const double* xyz, const double* w,
                                                     const double* rho, const double* grad_rho,
                                                     vv10_params prm, vv10_precision prec,
                                                     double* energy, double* vrho, double* vgamma,
                                                     void* stream) {
    if (n < 1) return VV10_ERR_INVALID_ARG;
    if (n > kNaMaxPoints) return VV10_ERR_UNSUPPORTED;
    if (!precision_known(prec))
        return VV10_ERR_INVALID_ARG;
    if (!(prm.b > 0.0) || !(prm.C >= 0.0) || !(prm.rho_cut > 0.0) || !std::isfinite(prm.b) ||
        !std::isfinite(prm.C) || !std::isfinite(prm.rho_cut))
        return VV10_ERR_INVALID_ARG;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return VV10_ERR_CUDA;
    }
    const void* in[] = {xyz, w, rho, grad_rho, energy};
    for (const void* q : in)
        if (!na_device_ptr(q, device)) return VV10_ERR_INVALID_ARG;
    if ((vrho && !na_device_ptr(vrho, device)) || (vgamma && !na_device_ptr(vgamma, device)))
        return VV10_ERR_INVALID_ARG;
    unsigned char* base = nullptr;
    if (na_scratch(device, &base) != cudaSuccess) {
        cudaGetLastError();
        return VV10_ERR_CUDA;
    }
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return VV10_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool fp64 = precision_fp64(prec);
    const int64_t n_pad = ((n + kJTile - 1) / kJTile) * kJTile;
    double4* r64a = reinterpret_cast<double4*>(base + kNaOffR64a);
    double4* r64b = reinterpret_cast<double4*>(base + kNaOffR64b);
    float4* r32a = reinterpret_cast<float4*>(base + kNaOffR32a);
    float4* r32b = reinterpret_cast<float4*>(base + kNaOffR32b);
    double* soa = reinterpret_cast<double*>(base + kNaOffSoa);
    int64_t* orig = reinterpret_cast<int64_t*>(base + kNaOffOrig);
    double* part = reinterpret_cast<double*>(base + kNaOffPart);
    double* eblk = reinterpret_cast<double*>(base + kNaOffEblk);
    double* center = reinterpret_cast<double*>(base + kNaOffMisc);
    int* err = reinterpret_cast<int*>(base + kNaOffMisc + 64);

    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);  // error word starts clear
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VV10_ERR_CUDA;
    }
    k_na_center<<<1, 1024, 0, st>>>(n, xyz, rho, prm.rho_cut, center);
    k_na_points<<<static_cast<unsigned>(n_pad / 256), 256, 0, st>>>(
        n, n_pad, xyz, w, rho, grad_rho, prm.b, prm.C, prm.rho_cut, center, r64a, r64b, r32a,
        r32b, soa, orig, err);
    PointsDev P;
    P.n = n;
    P.nk = n;
    P.nk_pad = n_pad;
    P.beta = std::pow(3.0 / (prm.b * prm.b), 0.75) / 32.0;  // beta of Sec. II.A
    P.orig = orig;
    P.r64a = r64a;
    P.r64b = r64b;
    P.r32a = r32a;
    P.r32b = r32b;
    PairLaunch cfg;
    cfg.rows_per_thread = fp64 ? 1 : 2;
    int ns = pairsum_default_split(P, MODE_EUW, fp64, cfg.rows_per_thread, n_sm);
    if (ns > kNaMaxSplit) ns = kNaMaxSplit;
    cfg.n_split = ns;
    const int ns_used = pairsum_split_count(n_pad, ns);  // the splits the launch uses
    e = launch_pairsum(P, MODE_EUW, fp64, cfg, part, err, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VV10_ERR_CUDA;
    }
    const int nblk = static_cast<int>(n_pad / 256);
    k_na_epilogue<<<nblk, 256, 0, st>>>(n, n_pad, P.beta, part, ns_used, soa, err, vrho, vgamma,
                                        eblk);
    e = launch_sum_blocks(eblk, nblk, energy, st);
    if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) {
        cudaGetLastError();
        return VV10_ERR_CUDA;
    }
    return VV10_OK;
}
