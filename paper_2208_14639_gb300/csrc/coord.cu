// K4: grid-coordinate derivative terms (Sec. II.A Eq. grad_gr, Sec. II.B Eq. EiBgr).
//
// Point gradient: the MODE_GRAD pair sums G_i = sum_j w_j rho_j Phi_ij D_ij (r_i - r_j) give
// dE/dr_i = -2 w_i rho_i G_i.  Atom terms E^A_gr = sum_{i in A} dE/dr_i: one CTA per atom
// over its contiguous segment (fixed reduction order).
//
// Atom-resolved terms: for every kept row i and atom B != atom(i), sums over j in B of
//   E_i^{Bgr} = -2 sum w_j rho_j Phi D (r_j - r_i)
//   U_i^{Bgr} =  2 sum w_j rho_j Phi [D (1/s + 1/g) + omega_i/g^2 + (omega_i+omega_j)/s^2] (r_j - r_i)
//   W_i^{Bgr} =  2 sum w_j rho_j Phi [R^2 D (1/s + 1/g) + R^2 (omega_i/g^2 + (omega_i+omega_j)/s^2)
//                                     - (1/s + 1/g)] (r_j - r_i)
// and for B = atom(i) minus the sum over the other atoms (translational invariance).
// The E part summed over every atom B (own atom included) is the point-gradient sum G_i,
// so the same pass also writes dE/dr_i = -2 w_i rho_i G_i when asked to.
#include "common.cuh"
#include "kernels.hpp"
#include "pairsum.cuh"

namespace vv10 {

static inline int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

__global__ void k_grad_epilogue(PointsDev P, const double* __restrict__ part, int n_split,
                                double* __restrict__ gk, double* __restrict__ grad_points) {
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= P.nk) return;
    const double c = -2.0 * P.w[p] * P.rho[p];
    const int64_t i = P.orig[p];
    for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int k = 0; k < n_split; ++k) s += part[(static_cast<int64_t>(d) * n_split + k) * P.nk_pad + p];
        const double g = c * s;
        gk[3 * p + d] = g;
        if (grad_points) grad_points[3 * i + d] = g;
    }
}

cudaError_t launch_grad_epilogue(const PointsDev& p, const double* part, int n_split, double* gk,
                                 double* grad_points, cudaStream_t st) {
    if (p.nk == 0) return cudaSuccess;
    k_grad_epilogue<<<static_cast<unsigned>(cdiv64(p.nk, 256)), 256, 0, st>>>(p, part, n_split, gk,
                                                                            grad_points);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256)
k_atom_sums(PointsDev P, const double* __restrict__ gk, double* __restrict__ out) {
    __shared__ double sh[8];
    const int a = blockIdx.x;
    const int64_t s0 = P.seg[a], s1 = P.seg[a + 1];
    for (int d = 0; d < 3; ++d) {
        double v = 0.0;
        for (int64_t p = s0 + threadIdx.x; p < s1; p += blockDim.x) v += gk[3 * p + d];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) out[3 * a + d] = v;
    }
}

cudaError_t launch_atom_sums(const PointsDev& p, const double* gk, double* grad_atoms,
                             cudaStream_t st) {
    if (p.n_atom <= 0) return cudaSuccess;
    k_atom_sums<<<p.n_atom, 256, 0, st>>>(p, gk, grad_atoms);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ atom-resolved
constexpr int kArThreads = 128;
constexpr int kArJT = 256;  // j per shared-memory tile (two records per thread)

// Resident CTAs per SM: 8 (at most 64 registers a thread) for the FP32 kernel, so that its
// grid of one row per thread fits the GPU in about one wave for grids of ~150 k kept points;
// 6 when it also forms the six E/U/W/A/B/C row sums.
template <class T, bool SUMS>
constexpr int ar_min_blocks() { return sizeof(T) == 4 ? (SUMS ? 6 : 8) : (SUMS ? 3 : 4); }

// SUMS: the same pass also forms the row sums of the fused energy + A/B/C mode (the
// pair-sum kernel's MODE_EUWABC) into part[6][nk_pad] (one split), so that a full
// evaluation makes a single pass over the pairs.
template <class T, bool SUMS>
__global__ void __launch_bounds__(kArThreads, ar_min_blocks<T, SUMS>())
k_atom_resolved(PointsDev P, const typename PairRecs<T>::A* __restrict__ ra,
                const typename PairRecs<T>::B* __restrict__ rb, double* __restrict__ out,
                double* __restrict__ gk, double* __restrict__ grad_points,
                double* __restrict__ part) {
    using RA = typename PairRecs<T>::A;
    using RB = typename PairRecs<T>::B;
    __shared__ RA sa[kArJT];
    __shared__ RB sb[kArJT];
    const int tid = threadIdx.x;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kArThreads + tid;
    const bool valid = i < P.nk;
    T xi = 0, yi = 0, zi = 0, oi = 1, ki = 1;
    int ai = -1;
    if (valid) {
        const RA a = ra[i];
        const RB b = rb[i];
        xi = a.x; yi = a.y; zi = a.z; oi = b.x; ki = b.y;
        ai = P.atom[i];
    }
    const int64_t n = P.n, na = P.n_atom;
    const int64_t oi_idx = valid ? P.orig[i] : 0;
    double gsum[3] = {0.0, 0.0, 0.0};  // E part over every atom: the point-gradient sum
    double rs[SUMS ? 6 : 1];           // E/U/W/A/B/C row sums (SUMS)
#pragma unroll
    for (int q = 0; q < (SUMS ? 6 : 1); ++q) rs[q] = 0.0;

    for (int B = 0; B < P.n_atom; ++B) {
        const int64_t s0 = P.seg[B], s1 = P.seg[B + 1];
        double tot[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) tot[q] = 0.0;
        for (int64_t j0 = s0; j0 < s1; j0 += kArJT) {
            __syncthreads();
            for (int t = tid; t < kArJT; t += kArThreads)
                if (j0 + t < s1) {
                    sa[t] = ra[j0 + t];
                    sb[t] = rb[j0 + t];
                }
            __syncthreads();
            const int cnt = static_cast<int>(s1 - j0 < kArJT ? s1 - j0 : kArJT);
            T acc[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) acc[q] = T(0);
            T sacc[SUMS ? 6 : 1];
#pragma unroll
            for (int q = 0; q < (SUMS ? 6 : 1); ++q) sacc[q] = T(0);
            for (int jj = 0; jj < cnt; ++jj) {
                const RA a = sa[jj];
                const RB b = sb[jj];
                const T dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
                const T r2 = dx * dx + dy * dy + dz * dz;
                const T g = oi * r2 + ki;
                const T gp = b.x * r2 + b.y;
                const T s = g + gp;
                const T ggp = g * gp;
                const T inv = recip(ggp * s);
                const T ph = a.w * inv;          // w_j rho_j Phi_ij
                const T sinv = s * inv;          // 1/(g g')
                const T L = ggp * inv;           // 1/s
                const T Gi = gp * sinv;          // 1/g
                const T Gj = g * sinv;           // 1/g'
                const T q = (oi + b.x) * L;      // (omega_i + omega_j)/s
                const T oG = oi * Gi;            // omega_i/g
                const T D = fmadd(b.x, Gj, oG + q);
                const T t1 = L + Gi;
                // omega_i/g^2 + (omega_i + omega_j)/s^2 = oG Gi + q L
                const T X = fmadd(D, t1, fmadd(oG, Gi, q * L));
                const T cE = ph * D;
                const T cU = ph * X;
                const T cW = fmadd(r2, cU, -(ph * t1));
                acc[0] += cE * dx; acc[1] += cE * dy; acc[2] += cE * dz;
                acc[3] += cU * dx; acc[4] += cU * dy; acc[5] += cU * dz;
                acc[6] += cW * dx; acc[7] += cW * dy; acc[8] += cW * dz;
                if constexpr (SUMS) {
                    const T pt = ph * t1;
                    sacc[0] += ph;
                    sacc[1] += pt;
                    sacc[2] = fmadd(pt, r2, sacc[2]);
                    const T v = ph * fmadd(L, t1, Gi * Gi);  // 1/s^2 + 1/(s g) + 1/g^2
                    sacc[3] += v;
                    const T v2 = v * r2;
                    sacc[4] += v2;
                    sacc[5] = fmadd(v2, r2, sacc[5]);
                }
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) tot[q] += static_cast<double>(acc[q]);
            if constexpr (SUMS) {
#pragma unroll
                for (int q = 0; q < 6; ++q) rs[q] += static_cast<double>(sacc[q]);
            }
        }
        gsum[0] += tot[0];
        gsum[1] += tot[1];
        gsum[2] += tot[2];
        // (r_i - r_j) was accumulated: E = +2 acc, U = -2 acc, W = -2 acc
        if (valid && B != ai) {
#pragma unroll
            for (int q = 0; q < 9; ++q)
                out[((static_cast<int64_t>(q / 3) * n + oi_idx) * na + B) * 3 + (q % 3)] =
                    (q < 3 ? 2.0 : -2.0) * tot[q];
        }
    }
    if (valid && ai >= 0 && ai < P.n_atom) {
        // own atom: minus the sum over the other atoms, read back from this thread's writes
        for (int q = 0; q < 9; ++q) {
            double* row = out + (static_cast<int64_t>(q / 3) * n + oi_idx) * na * 3 + (q % 3);
            double rest = 0.0;
            for (int B = 0; B < P.n_atom; ++B)
                if (B != ai) rest += row[3 * B];
            row[3 * ai] = -rest;
        }
    }
    if constexpr (SUMS) {
        if (valid) {
#pragma unroll
            for (int q = 0; q < 6; ++q) part[static_cast<int64_t>(q) * P.nk_pad + i] = rs[q];
        }
    }
    if (valid && gk) {
        const double c = -2.0 * P.w[i] * P.rho[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            gk[3 * i + d] = c * gsum[d];
            if (grad_points) grad_points[3 * oi_idx + d] = c * gsum[d];
        }
    }
}

// ------------------------------------------------------------------ grid-grid Hessian block
// D_i^B (Sec. II.B) for every kept row i and atom B != atom(i):
//   D_i^B = -2 sum_{j in B} w_j rho_j Phi_ij [ 2 (D^2 + (omega_i/g)^2 + (omega_j/g')^2
//           + ((omega_i+omega_j)/s)^2) (r_j - r_i)(r_j - r_i)^T - D I_3 ],
// D = omega_i/g + omega_j/g' + (omega_i+omega_j)/s, and the blocks
//   E^{AB}_{gr,gr} = sum_{i in A} w_i rho_i D_i^B (A != B),  E^{AA} = -sum_{B != A} E^{AB}.
// Kept rows are grouped by atom and cut into chunks of kArThreads rows within one atom; a
// task is (chunk c of atom A, atom B != A), one CTA each, and reduces w_i rho_i D_i^B over
// its rows (fixed order) into part[c][B][6] (the 6 entries of the symmetric 3x3).  FP32
// (or FP64) arithmetic within a j tile, FP64 across tiles.
//
// The pair term is symmetric in i <-> j, so E^{AB} = E^{BA} (and each block is symmetric):
// when only the blocks are asked for, the tasks with B < A are skipped and E^{BA} is read
// from the same partials, which halves the pair evaluations.

// off[a] = chunks of the atoms before a, off[n_atom] = all chunks.
__global__ void k_chunk_offsets(PointsDev P, int64_t* __restrict__ off) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t c = 0;
    for (int a = 0; a < P.n_atom; ++a) {
        off[a] = c;
        c += (P.seg[a + 1] - P.seg[a] + kArThreads - 1) / kArThreads;
    }
    off[P.n_atom] = c;
}

template <class T, bool HALF>
__global__ void __launch_bounds__(kArThreads)
k_coord_hessian(PointsDev P, const typename PairRecs<T>::A* __restrict__ ra,
                const typename PairRecs<T>::B* __restrict__ rb, const int64_t* __restrict__ off,
                double* __restrict__ part, double* __restrict__ Dout) {
    using RA = typename PairRecs<T>::A;
    using RB = typename PairRecs<T>::B;
    __shared__ RA sa[kArJT];
    __shared__ RB sb[kArJT];
    __shared__ double sred[6][kArThreads / 32];
    const int64_t c = blockIdx.x;
    const int B = blockIdx.y;
    if (c >= off[P.n_atom]) return;  // every exit below is uniform over the CTA
    int lo = 0, hi = P.n_atom;       // atom A of chunk c: the last a with off[a] <= c
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= c) lo = mid;
        else hi = mid;
    }
    const int A = lo;
    if (B == A || (HALF && B < A)) return;
    const int64_t s0 = P.seg[B], s1 = P.seg[B + 1];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t i = P.seg[A] + (c - off[A]) * kArThreads + tid;
    const bool valid = i < P.seg[A + 1];
    T xi = 0, yi = 0, zi = 0, oi = 1, ki = 1;
    double ci = 0.0;
    if (valid) {
        const RA a = ra[i];
        const RB b = rb[i];
        xi = a.x; yi = a.y; zi = a.z; oi = b.x; ki = b.y;
        ci = P.w[i] * P.rho[i];
    }
    double tot[7] = {0, 0, 0, 0, 0, 0, 0};  // xx xy xz yy yz zz of the outer products; I term
    for (int64_t j0 = s0; j0 < s1; j0 += kArJT) {
        __syncthreads();
        for (int t = tid; t < kArJT; t += kArThreads)
            if (j0 + t < s1) {
                sa[t] = ra[j0 + t];
                sb[t] = rb[j0 + t];
            }
        __syncthreads();
        const int cnt = static_cast<int>(s1 - j0 < kArJT ? s1 - j0 : kArJT);
        T acc[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        for (int jj = 0; jj < cnt; ++jj) {
            const RA a = sa[jj];
            const RB b = sb[jj];
            const T dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
            const T r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
            const T g = fmadd(oi, r2, ki);
            const T gp = fmadd(b.x, r2, b.y);
            const T s = g + gp;
            const T ggp = g * gp;
            const T inv = recip(ggp * s);
            const T ph = a.w * inv;          // w_j rho_j Phi_ij
            const T sinv = s * inv;          // 1/(g g')
            const T L = ggp * inv;           // 1/s
            const T oG = oi * (gp * sinv);   // omega_i/g
            const T bG = b.x * (g * sinv);   // omega_j/g'
            const T q = (oi + b.x) * L;      // (omega_i + omega_j)/s
            const T D = oG + bG + q;
            // half the squared bracket; the factor 2 is applied to the sums
            const T av = ph * fmadd(D, D, fmadd(oG, oG, fmadd(bG, bG, q * q)));
            const T tx = av * dx, ty = av * dy;
            acc[0] = fmadd(tx, dx, acc[0]);
            acc[1] = fmadd(tx, dy, acc[1]);
            acc[2] = fmadd(tx, dz, acc[2]);
            acc[3] = fmadd(ty, dy, acc[3]);
            acc[4] = fmadd(ty, dz, acc[4]);
            acc[5] = fmadd(av * dz, dz, acc[5]);
            acc[6] = fmadd(ph, D, acc[6]);
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) tot[k] += static_cast<double>(acc[k]);
    }
    // D_i^B = -2 (2 S - S_I I), S the (halved) outer-product sum, S_I the identity term
    double d6[6] = {-2.0 * (2.0 * tot[0] - tot[6]), -4.0 * tot[1], -4.0 * tot[2],
                    -2.0 * (2.0 * tot[3] - tot[6]), -4.0 * tot[4], -2.0 * (2.0 * tot[5] - tot[6])};
    if (!valid) {
#pragma unroll
        for (int k = 0; k < 6; ++k) d6[k] = 0.0;
    } else if (Dout) {
        double* o = Dout + (P.orig[i] * P.n_atom + B) * 9;
        o[0] = d6[0]; o[1] = d6[1]; o[2] = d6[2];
        o[3] = d6[1]; o[4] = d6[3]; o[5] = d6[4];
        o[6] = d6[2]; o[7] = d6[4]; o[8] = d6[5];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double v = warp_sum(ci * d6[k]);
        if (lane == 0) sred[k][wid] = v;
    }
    __syncthreads();
    if (tid < 6) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kArThreads / 32; ++w) v += sred[tid][w];
        part[(c * P.n_atom + B) * 6 + tid] = v;
    }
}

// One CTA per atom A: warp k forms the blocks E^{AB} for B = k, k + 8, ... from the CTA
// partials (lane-strided over the chunks in a fixed order, then a fixed shuffle tree), then
// the diagonal block.  With HALF, E^{AB} for B < A is the sum that the CTA of atom B forms
// for E^{BA} (chunks of B, column A), so the two agree exactly.
constexpr int kChBlkThreads = 256;
template <bool HALF>
__global__ void __launch_bounds__(kChBlkThreads)
k_coord_hessian_blocks(PointsDev P, const int64_t* __restrict__ off,
                       const double* __restrict__ part, double* __restrict__ E) {
    const int A = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t na = P.n_atom;
    for (int B = wid; B < P.n_atom; B += kChBlkThreads / 32) {
        if (B == A) continue;
        const bool mirror = HALF && B < A;
        const int owner = mirror ? B : A, col = mirror ? A : B;
        const int64_t c0 = off[owner], c1 = off[owner + 1];
        double v[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t c = c0 + lane; c < c1; c += 32)
#pragma unroll
            for (int k = 0; k < 6; ++k) v[k] += part[(c * na + col) * 6 + k];
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = warp_sum(v[k]);
        if (lane == 0) {
            double* o = E + (A * na + B) * 9;
            o[0] = v[0]; o[1] = v[1]; o[2] = v[2];
            o[3] = v[1]; o[4] = v[3]; o[5] = v[4];
            o[6] = v[2]; o[7] = v[4]; o[8] = v[5];
        }
    }
    __syncthreads();  // this CTA's writes of row A are visible to the whole CTA
    if (threadIdx.x < 9) {
        double d = 0.0;
        for (int B = 0; B < P.n_atom; ++B)
            if (B != A) d += E[(A * na + B) * 9 + threadIdx.x];
        E[(A * na + A) * 9 + threadIdx.x] = -d;
    }
}

// Upper bound on the row chunks: one per kArThreads rows, plus one partial chunk per atom.
int64_t coord_hessian_chunk_bound(int64_t nk, int32_t n_atom) {
    return cdiv64(nk, kArThreads) + (n_atom > 0 ? n_atom : 0);
}

cudaError_t launch_coord_hessian(const PointsDev& p, bool fp64, int64_t* off, double* part,
                                 double* E, double* Dout, cudaStream_t st) {
    if (p.n_atom <= 0) return cudaSuccess;
    k_chunk_offsets<<<1, 32, 0, st>>>(p, off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const bool half = (Dout == nullptr);
    if (p.nk > 0 && p.n_atom > 1) {
        const dim3 g(static_cast<unsigned>(coord_hessian_chunk_bound(p.nk, p.n_atom)),
                     static_cast<unsigned>(p.n_atom));
        if (fp64) {
            if (half) k_coord_hessian<double, true><<<g, kArThreads, 0, st>>>(p, p.r64a, p.r64b, off, part, Dout);
            else k_coord_hessian<double, false><<<g, kArThreads, 0, st>>>(p, p.r64a, p.r64b, off, part, Dout);
        } else {
            if (half) k_coord_hessian<float, true><<<g, kArThreads, 0, st>>>(p, p.r32a, p.r32b, off, part, Dout);
            else k_coord_hessian<float, false><<<g, kArThreads, 0, st>>>(p, p.r32a, p.r32b, off, part, Dout);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (half) k_coord_hessian_blocks<true><<<p.n_atom, kChBlkThreads, 0, st>>>(p, off, part, E);
    else k_coord_hessian_blocks<false><<<p.n_atom, kChBlkThreads, 0, st>>>(p, off, part, E);
    return cudaGetLastError();
}

cudaError_t launch_atom_resolved(const PointsDev& p, bool fp64, double* out, double* gk,
                                 double* grad_points, double* sums, int* err, cudaStream_t st) {
    if (p.nk == 0 || p.n_atom <= 0) return cudaSuccess;
    const unsigned g = static_cast<unsigned>(cdiv64(p.nk, kArThreads));
    (void)err;
    if (sums) {
        if (fp64) k_atom_resolved<double, true><<<g, kArThreads, 0, st>>>(p, p.r64a, p.r64b, out, gk, grad_points, sums);
        else k_atom_resolved<float, true><<<g, kArThreads, 0, st>>>(p, p.r32a, p.r32b, out, gk, grad_points, sums);
    } else {
        if (fp64) k_atom_resolved<double, false><<<g, kArThreads, 0, st>>>(p, p.r64a, p.r64b, out, gk, grad_points, nullptr);
        else k_atom_resolved<float, false><<<g, kArThreads, 0, st>>>(p, p.r32a, p.r32b, out, gk, grad_points, nullptr);
    }
    return cudaGetLastError();
}

}  // namespace vv10
