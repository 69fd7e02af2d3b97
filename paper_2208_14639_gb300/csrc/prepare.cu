// K1: per-point precompute (Sec. II.A point quantities) and stable compaction of the
// points that pass the density cutoff, grouped by atom.
//
// Stage 1 (count): per block of kPB caller points, histogram of keys (atom of a kept
//   point, or the "dropped" bucket) and the bounding box of the kept points.
// Stage 2 (scan, one CTA): exclusive scan over the key-major [key][block] histogram; this
//   fixes every kept point's destination (by atom, then by caller order), n_kept, the
//   atom segment starts and the recentring origin for the FP32 records.
// Stage 3 (scatter): each block assigns destinations to its points in caller order.
// Stage 4 (points): omega, kappa and their derivatives in FP64 at every kept point, the
//   SoA arrays and the packed pair records.
// Every stage is deterministic (no floating-point atomics, fixed reduction order).
#include <cmath>

#include "common.cuh"
#include "kernels.hpp"

namespace vv10 {

constexpr int kPB = 1024;       // caller points per count/scatter block
constexpr int kPrepThreads = 256;

int prepare_nblk(int64_t n) { return static_cast<int>((n + kPB - 1) / kPB); }

__device__ __forceinline__ bool finite3(double a, double b, double c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

__device__ __forceinline__ int point_key(int64_t i, const double* rho, const int32_t* atom,
                                         int32_t n_atom, double rho_cut, int n_keys,
                                         bool& keep) {
    const double r = rho[i];
    keep = (r >= rho_cut);
    if (!keep) return n_keys - 1;
    if (!atom) return 0;
    const int a = atom[i];
    return (a >= 0 && a < n_atom) ? a : 0;
}

// One count block (caller points kPB blk ..): key histogram and kept bounding box.
__device__ __forceinline__ void prep_count_block(int64_t n, const double* __restrict__ xyz,
                                                 const double* __restrict__ w,
                                                 const double* __restrict__ rho,
                                                 const double* __restrict__ grad,
                                                 const int32_t* __restrict__ atom, int32_t n_atom,
                                                 double rho_cut, int n_keys, int nblk,
                                                 int32_t* __restrict__ hist,
                                                 double* __restrict__ bbox_part, int* err,
                                                 int64_t blk) {
    extern __shared__ int sh_hist[];
    __shared__ double sh_red[6][kPrepThreads / 32];
    for (int k = threadIdx.x; k < n_keys; k += blockDim.x) sh_hist[k] = 0;
    __syncthreads();
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    const int64_t base = blk * kPB;
    const int64_t end = min(n, base + kPB);
    int bad = 0;
    for (int64_t i = base + threadIdx.x; i < end; i += blockDim.x) {
        const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        if (!finite3(x, y, z) || !isfinite(w[i]) || isnan(rho[i]) ||
            !finite3(grad[3 * i], grad[3 * i + 1], grad[3 * i + 2]))
            bad |= DEVERR_BAD_INPUT;
        if (atom && (atom[i] < 0 || atom[i] >= n_atom)) bad |= DEVERR_BAD_ATOM;
        bool keep;
        const int key = point_key(i, rho, atom, n_atom, rho_cut, n_keys, keep);
        atomicAdd(&sh_hist[key], 1);
        if (keep) {
            mn[0] = fmin(mn[0], x); mn[1] = fmin(mn[1], y); mn[2] = fmin(mn[2], z);
            mx[0] = fmax(mx[0], x); mx[1] = fmax(mx[1], y); mx[2] = fmax(mx[2], z);
        }
    }
    if (bad) atomicOr(err, bad);
    __syncthreads();
    for (int k = threadIdx.x; k < n_keys; k += blockDim.x)
        hist[static_cast<int64_t>(k) * nblk + blk] = sh_hist[k];
    // block min / max of the kept coordinates (exact operations: order independent)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double a = mn[d], b = mx[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) { sh_red[d][wid] = a; sh_red[3 + d][wid] = b; }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = sh_red[threadIdx.x][0];
        for (int q = 1; q < kPrepThreads / 32; ++q)
            v = threadIdx.x < 3 ? fmin(v, sh_red[threadIdx.x][q]) : fmax(v, sh_red[threadIdx.x][q]);
        bbox_part[blk * 6 + threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(kPrepThreads)
k_prep_count(int64_t n, const double* __restrict__ xyz, const double* __restrict__ w,
             const double* __restrict__ rho, const double* __restrict__ grad,
             const int32_t* __restrict__ atom, int32_t n_atom, double rho_cut, int n_keys,
             int nblk, int32_t* __restrict__ hist, double* __restrict__ bbox_part, int* err) {
    prep_count_block(n, xyz, w, rho, grad, atom, n_atom, rho_cut, n_keys, nblk, hist, bbox_part,
                     err, blockIdx.x);
}

__global__ void __launch_bounds__(kPrepThreads)
k_prep_count_batch(const PrepMol* __restrict__ mols, const int64_t* __restrict__ pre, int n_mol,
                   double rho_cut, int* err) {
    int64_t blk;
    const PrepMol& M = mols[batch_block_mol(pre, n_mol, blockIdx.x, blk)];
    prep_count_block(M.n, M.xyz, M.w, M.rho, M.grad, M.atom, M.n_atom, rho_cut, M.n_keys, M.nblk,
                     M.hist, M.bbox_part, err, blk);
}

// One CTA of 1024 threads: exclusive scan of M = n_keys*nblk counts.
__device__ __forceinline__ void prep_scan_block(const int32_t* __restrict__ hist, int64_t M,
                                                int64_t* __restrict__ offs, int n_keys, int nblk,
                                                int32_t n_atom, const double* __restrict__ bbox_part,
                                                double* __restrict__ center,
                                                int64_t* __restrict__ nk_out,
                                                int64_t* __restrict__ seg) {
    __shared__ int64_t sh[1024];
    __shared__ double shb[6];
    const int t = threadIdx.x;
    const int64_t chunk = (M + 1023) / 1024;
    const int64_t b0 = t * chunk, b1 = min(M, b0 + chunk);
    int64_t local = 0;
    for (int64_t k = b0; k < b1; ++k) local += hist[k];
    sh[t] = local;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 1024 chunk totals
    for (int o = 1; o < 1024; o <<= 1) {
        const int64_t v = (t >= o) ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += v;
        __syncthreads();
    }
    int64_t run = sh[t] - local;
    for (int64_t k = b0; k < b1; ++k) {
        offs[k] = run;
        run += hist[k];
    }
    if (t < 6) {
        double v = (t < 3) ? INFINITY : -INFINITY;
        for (int b = 0; b < nblk; ++b)
            v = (t < 3) ? fmin(v, bbox_part[b * 6 + t]) : fmax(v, bbox_part[b * 6 + t]);
        shb[t] = v;
    }
    __syncthreads();  // offs complete, bbox reduced
    const int64_t nk = offs[static_cast<int64_t>(n_keys - 1) * nblk];
    if (t == 0) *nk_out = nk;
    if (t < 3) center[t] = (nk > 0) ? 0.5 * (shb[t] + shb[3 + t]) : 0.0;
    const int32_t n_seg = n_atom > 0 ? n_atom : 1;
    for (int a = t; a < n_seg; a += blockDim.x) seg[a] = offs[static_cast<int64_t>(a) * nblk];
    if (t == 0) seg[n_seg] = nk;
}

__global__ void __launch_bounds__(1024)
k_prep_scan(const int32_t* __restrict__ hist, int64_t M, int64_t* __restrict__ offs, int n_keys,
            int nblk, int32_t n_atom, const double* __restrict__ bbox_part,
            double* __restrict__ center, int64_t* __restrict__ nk_out, int64_t* __restrict__ seg) {
    prep_scan_block(hist, M, offs, n_keys, nblk, n_atom, bbox_part, center, nk_out, seg);
}

// One CTA per molecule; the segment starts go into the slots after its offsets.
__global__ void __launch_bounds__(1024) k_prep_scan_batch(const PrepMol* __restrict__ mols) {
    const PrepMol& P = mols[blockIdx.x];
    const int64_t M = static_cast<int64_t>(P.n_keys) * P.nblk;
    prep_scan_block(P.hist, M, P.offs, P.n_keys, P.nblk, P.n_atom, P.bbox_part, P.center, P.nk_dev,
                    P.offs + M);
}

__device__ __forceinline__ void prep_scatter_block(int64_t n, const double* __restrict__ rho,
                                                   const int32_t* __restrict__ atom, int32_t n_atom,
                                                   double rho_cut, int n_keys, int nblk,
                                                   const int64_t* __restrict__ offs,
                                                   int64_t* __restrict__ orig, int64_t blk) {
    extern __shared__ int64_t sh_cnt[];  // n_keys running destinations
    __shared__ int sh_key[kPB];
    __shared__ int64_t sh_pos[kPB];
    const int64_t base = blk * kPB;
    const int cnt = static_cast<int>(n - base < kPB ? n - base : kPB);
    for (int k = threadIdx.x; k < n_keys; k += blockDim.x)
        sh_cnt[k] = offs[static_cast<int64_t>(k) * nblk + blk];
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        bool keep;
        sh_key[q] = point_key(base + q, rho, atom, n_atom, rho_cut, n_keys, keep);
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // caller order within the block -> stable
        for (int q = 0; q < cnt; ++q) sh_pos[q] = sh_cnt[sh_key[q]]++;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < cnt; q += blockDim.x)
        if (sh_key[q] != n_keys - 1) orig[sh_pos[q]] = base + q;
}

__global__ void __launch_bounds__(kPrepThreads)
k_prep_scatter(int64_t n, const double* __restrict__ rho, const int32_t* __restrict__ atom,
               int32_t n_atom, double rho_cut, int n_keys, int nblk,
               const int64_t* __restrict__ offs, int64_t* __restrict__ orig) {
    prep_scatter_block(n, rho, atom, n_atom, rho_cut, n_keys, nblk, offs, orig, blockIdx.x);
}

// Also copies each molecule's segment starts (block 0 of the molecule).
__global__ void __launch_bounds__(kPrepThreads)
k_prep_scatter_batch(const PrepMol* __restrict__ mols, const int64_t* __restrict__ pre, int n_mol,
                     double rho_cut) {
    int64_t blk;
    const PrepMol& P = mols[batch_block_mol(pre, n_mol, blockIdx.x, blk)];
    if (blk == 0) {
        const int64_t M = static_cast<int64_t>(P.n_keys) * P.nblk;
        const int n_seg = (P.n_atom > 0 ? P.n_atom : 1) + 1;
        for (int a = threadIdx.x; a < n_seg; a += blockDim.x) P.seg[a] = P.offs[M + a];
    }
    prep_scatter_block(P.n, P.rho, P.atom, P.n_atom, rho_cut, P.n_keys, P.nblk, P.offs, P.orig, blk);
}

__device__ __forceinline__ void prep_point(int64_t nk, int64_t nk_pad, const int64_t* __restrict__ orig,
                                           const double* __restrict__ xyz,
                                           const double* __restrict__ w,
                                           const double* __restrict__ rho,
                                           const double* __restrict__ grad,
                                           const int32_t* __restrict__ atom, double b, double C,
                                           const double* __restrict__ center,
                                           int32_t* __restrict__ atom_k, double* __restrict__ soa,
                                           double4* __restrict__ r64a, double4* __restrict__ r64b,
                                           float4* __restrict__ r32a, float4* __restrict__ r32b,
                                           float4* __restrict__ r32p, int64_t p) {
    if (p >= nk_pad) return;
    // pair-packed record slots of this point: pair m = p / 2, component h = p % 2
    float* pk = reinterpret_cast<float*>(r32p) + (p >> 1) * 16 + (p & 1);
    if (p >= nk) {  // padding record: contributes exactly zero to every pair sum
        r64a[p] = make_double4(0.0, 0.0, 0.0, 0.0);
        r64b[p] = make_double4(1.0, 1.0, 0.0, 0.0);
        r32a[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        r32b[p] = make_float4(1.f, 1.f, 0.f, 0.f);
        const float pad[8] = {0.f, 0.f, 0.f, 1.f, 1.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < 8; ++k) pk[2 * k] = pad[k];
        return;
    }
    const int64_t i = orig[p];
    const double r = rho[i];
    const double gx = grad[3 * i], gy = grad[3 * i + 1], gz = grad[3 * i + 2];
    const double gam = gx * gx + gy * gy + gz * gz;
    const double pi = 3.141592653589793238462643383279502884;
    // omega^2 = Q = C gamma^2 / rho^4 + 4 pi rho / 3 and derivatives of Q
    const double ir = 1.0 / r, ir2 = ir * ir, ir4 = ir2 * ir2;
    const double Q = C * gam * gam * ir4 + (4.0 * pi / 3.0) * r;
    const double Qr = -4.0 * C * gam * gam * ir4 * ir + 4.0 * pi / 3.0;
    const double Qg = 2.0 * C * gam * ir4;
    const double Qrr = 20.0 * C * gam * gam * ir4 * ir2;
    const double Qrg = -8.0 * C * gam * ir4 * ir;
    const double Qgg = 2.0 * C * ir4;
    const double om = sqrt(Q), iom = 1.0 / om, iom3 = iom * iom * iom;
    const double om_r = 0.5 * Qr * iom, om_g = 0.5 * Qg * iom;
    const double om_rr = 0.5 * Qrr * iom - 0.25 * Qr * Qr * iom3;
    const double om_rg = 0.5 * Qrg * iom - 0.25 * Qr * Qg * iom3;
    const double om_gg = 0.5 * Qgg * iom - 0.25 * Qg * Qg * iom3;
    // kappa = b (3 pi / 2) (rho / 9 pi)^(1/6)
    const double ka = b * 1.5 * pi * pow(r / (9.0 * pi), 1.0 / 6.0);
    const double ka_r = ka * ir / 6.0, ka_rr = -5.0 * ka * ir2 / 36.0;
    const double wi = w[i];
    double* f = soa;
    f[F_W * nk_pad + p] = wi;
    f[F_RHO * nk_pad + p] = r;
    f[F_GX * nk_pad + p] = gx;
    f[F_GY * nk_pad + p] = gy;
    f[F_GZ * nk_pad + p] = gz;
    f[F_OM * nk_pad + p] = om;
    f[F_KA * nk_pad + p] = ka;
    f[F_OMR * nk_pad + p] = om_r;
    f[F_OMG * nk_pad + p] = om_g;
    f[F_KAR * nk_pad + p] = ka_r;
    f[F_OMRR * nk_pad + p] = om_rr;
    f[F_OMRG * nk_pad + p] = om_rg;
    f[F_OMGG * nk_pad + p] = om_gg;
    f[F_KARR * nk_pad + p] = ka_rr;
    const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    const double cj = -1.5 * wi * r;  // the -3/2 of Phi folded into w rho
    r64a[p] = make_double4(x, y, z, cj);
    r64b[p] = make_double4(om, ka, r * ka_r, r * om_r);
    r32a[p] = make_float4(static_cast<float>(x - center[0]), static_cast<float>(y - center[1]),
                          static_cast<float>(z - center[2]), static_cast<float>(cj));
    r32b[p] = make_float4(static_cast<float>(om), static_cast<float>(ka),
                          static_cast<float>(r * ka_r), static_cast<float>(r * om_r));
    const float4 a = r32a[p];
    const float vals[8] = {-a.x, -a.y, -a.z, static_cast<float>(om), static_cast<float>(ka),
                           -static_cast<float>(r * ka_r), -static_cast<float>(r * om_r),
                           static_cast<float>(cj)};
    for (int k = 0; k < 8; ++k) pk[2 * k] = vals[k];
    atom_k[p] = atom ? atom[i] : 0;
}

__global__ void __launch_bounds__(256)
k_prep_points(int64_t nk, int64_t nk_pad, const int64_t* __restrict__ orig,
              const double* __restrict__ xyz, const double* __restrict__ w,
              const double* __restrict__ rho, const double* __restrict__ grad,
              const int32_t* __restrict__ atom, double b, double C,
              const double* __restrict__ center, int32_t* __restrict__ atom_k,
              double* __restrict__ soa, double4* __restrict__ r64a, double4* __restrict__ r64b,
              float4* __restrict__ r32a, float4* __restrict__ r32b, float4* __restrict__ r32p) {
    prep_point(nk, nk_pad, orig, xyz, w, rho, grad, atom, b, C, center, atom_k, soa, r64a, r64b,
               r32a, r32b, r32p, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(256)
k_prep_points_batch(const PrepMol* __restrict__ mols, const int64_t* __restrict__ pre, int n_mol,
                    double b, double C) {
    int64_t blk;
    const PrepMol& P = mols[batch_block_mol(pre, n_mol, blockIdx.x, blk)];
    prep_point(P.nk, P.nk_pad, P.orig, P.xyz, P.w, P.rho, P.grad, P.atom, b, C, P.center, P.atom_k,
               P.soa, P.r64a, P.r64b, P.r32a, P.r32b, P.r32p, blk * 256 + threadIdx.x);
}

cudaError_t launch_prepare_count(int64_t n, const double* xyz, const double* w, const double* rho,
                                 const double* grad, const int32_t* atom, int32_t n_atom,
                                 double rho_cut, const PrepareScratch& s, int* err,
                                 cudaStream_t st) {
    const int nblk = prepare_nblk(n);
    const int n_keys = (n_atom > 0 ? n_atom : 1) + 1;
    k_prep_count<<<nblk, kPrepThreads, n_keys * sizeof(int), st>>>(
        n, xyz, w, rho, grad, atom, n_atom, rho_cut, n_keys, nblk, s.hist, s.bbox_part, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t M = static_cast<int64_t>(n_keys) * nblk;
    // The scan also writes the atom segment starts, into the n_seg slots after offs.
    k_prep_scan<<<1, 1024, 0, st>>>(s.hist, M, s.offs, n_keys, nblk, n_atom, s.bbox_part,
                                    s.center, s.nk_dev, s.offs + M);
    return cudaGetLastError();
}

cudaError_t launch_prepare_scatter(int64_t n, const double* xyz, const double* w,
                                   const double* rho, const double* grad, const int32_t* atom,
                                   int32_t n_atom, double rho_cut, double b, double C,
                                   const PrepareScratch& s, int64_t nk, int64_t nk_pad,
                                   int64_t* orig, int64_t* seg, int32_t* atom_k, double* soa,
                                   double4* r64a, double4* r64b, float4* r32a, float4* r32b,
                                   float4* r32p, cudaStream_t st) {
    const int nblk = prepare_nblk(n);
    const int n_keys = (n_atom > 0 ? n_atom : 1) + 1;
    const int64_t M = static_cast<int64_t>(n_keys) * nblk;
    const int n_seg = (n_atom > 0 ? n_atom : 1) + 1;
    cudaError_t e = cudaMemcpyAsync(seg, s.offs + M, n_seg * sizeof(int64_t),
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    k_prep_scatter<<<nblk, kPrepThreads, n_keys * sizeof(int64_t), st>>>(
        n, rho, atom, n_atom, rho_cut, n_keys, nblk, s.offs, orig);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nk_pad > 0) {
        const int g = static_cast<int>((nk_pad + 255) / 256);
        k_prep_points<<<g, 256, 0, st>>>(nk, nk_pad, orig, xyz, w, rho, grad, atom, b, C,
                                         s.center, atom_k, soa, r64a, r64b, r32a, r32b, r32p);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_prepare_count_batch(const PrepMol* mols, const int64_t* pre, int n_mol,
                                       int64_t n_blocks, int max_keys, double rho_cut, int* err,
                                       cudaStream_t st) {
    if (n_mol <= 0) return cudaSuccess;
    if (n_blocks > 0) {
        k_prep_count_batch<<<static_cast<unsigned>(n_blocks), kPrepThreads, max_keys * sizeof(int), st>>>(
            mols, pre, n_mol, rho_cut, err);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_prep_scan_batch<<<n_mol, 1024, 0, st>>>(mols);
    return cudaGetLastError();
}

cudaError_t launch_prepare_scatter_batch(const PrepMol* mols, const int64_t* pre_blk,
                                         const int64_t* pre_pts, int n_mol, int64_t n_blocks,
                                         int64_t n_point_blocks, int max_keys, double rho_cut,
                                         double b, double C, cudaStream_t st) {
    if (n_blocks > 0) {
        k_prep_scatter_batch<<<static_cast<unsigned>(n_blocks), kPrepThreads, max_keys * sizeof(int64_t), st>>>(
            mols, pre_blk, n_mol, rho_cut);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_point_blocks > 0) {
        k_prep_points_batch<<<static_cast<unsigned>(n_point_blocks), 256, 0, st>>>(mols, pre_pts,
                                                                                n_mol, b, C);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace vv10
