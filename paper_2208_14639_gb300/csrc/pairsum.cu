// K2 / K4: flash-style double grid sums over kept points i (rows) and j (columns).
//
// One CTA owns NT*RPT rows i held in registers and streams a contiguous range of
// j-records through shared memory in tiles of kJTile, double-buffered, each tile fetched
// by two 1-D bulk asynchronous copies (TMA engine) completing on an mbarrier.  Every
// thread evaluates the closed-form pair kernel for its rows against every j of the tile
// (shared-memory broadcast reads).  The j range may be split over gridDim.y CTAs; each
// split writes FP64 partial sums that an epilogue reduces in a fixed order.
//
// Modes (the three quantities each mode accumulates per row i):
//   MODE_EUW  E_i = sum_j w_j rho_j Phi_ij, and sum_j w_j rho_j Phi_ij (1/s + 1/g) {1, R^2}
//             (U_i and W_i of Sec. II.A up to their sign)
//   MODE_ABC  sum_j w_j rho_j Phi_ij (1/s^2 + 1/(s g) + 1/g^2) {1, R^2, R^4}
//             (A_i, B_i, C_i of Sec. II.B up to the factor 2)
//   MODE_GRAD sum_j w_j rho_j Phi_ij D_ij (r_i - r_j), D_ij the bracket of Eq. grad_gr
//   MODE_EUWABC the six sums of MODE_EUW and MODE_ABC from one pass (partials [6][..])
//   MODE_EUWABCG those six and the three of MODE_GRAD from one pass (partials [9][..])
// with g = omega_i R^2 + kappa_i, g' = omega_j R^2 + kappa_j, s = g + g' and all of
// 1/g, 1/g', 1/s, Phi obtained from the single reciprocal inv = 1/(g g' s).
//
// FP32 variant: recentred FP32 coordinates, FP32 pair arithmetic, FP32 sums within a
// tile, promoted to FP64 once per tile.  FP64 variant: everything in FP64.
#include <cmath>

#include "common.cuh"
#include "kernels.hpp"
#include "pairsum.cuh"

namespace vv10 {

template <class T, int MODE, int RPT, int NT>
__global__ void __launch_bounds__(NT)
k_pairsum(const typename Recs<T>::A* __restrict__ ra, const typename Recs<T>::B* __restrict__ rb,
          int64_t nk, int64_t nk_pad, int64_t j_per_split, double* __restrict__ part,
          int* __restrict__ err, int stall) {
    using RA = typename Recs<T>::A;
    using RB = typename Recs<T>::B;
    __shared__ __align__(128) RA sa[2][kJTile];
    __shared__ __align__(128) RB sb[2][kJTile];
    __shared__ __align__(8) uint64_t bar[2];

    const int tid = threadIdx.x;
    const int n_split = gridDim.y;
    const int split = blockIdx.y;
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * (NT * RPT);
    const int64_t jb = static_cast<int64_t>(split) * j_per_split;
    const int64_t je = min(nk_pad, jb + j_per_split);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // Test hook: a stalled CTA never issues its copies, so its first wait runs out.
    const bool stalled = stall && blockIdx.x == 0 && blockIdx.y == 0;
    uint32_t gtile = 0;
    double dacc[RPT][pair_mode_nq(MODE)];
    pairsum_range<T, MODE, RPT, NT>(sa, sb, bar, gtile, ra, rb, nk, i0, jb, je, dacc, err, stalled);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int64_t i = i0 + r * NT + tid;
        if (i < nk) {
#pragma unroll
            for (int q = 0; q < pair_mode_nq(MODE); ++q)
                part[(static_cast<int64_t>(q) * n_split + split) * nk_pad + i] = dacc[r][q];
        }
    }
}

static inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Normalise a requested split count so that every split holds whole tiles.
static inline void split_geometry(int64_t nk_pad, int req, int64_t& j_per_split, int& n_split) {
    const int64_t ntile = nk_pad / kJTile;
    if (req < 1) req = 1;
    if (req > ntile) req = static_cast<int>(ntile > 0 ? ntile : 1);
    const int64_t tps = cdiv(ntile, req);
    j_per_split = tps * kJTile;
    n_split = static_cast<int>(ntile > 0 ? cdiv(ntile, tps) : 1);
}

template <class T, int MODE, int RPT, int NT>
static int blocks_per_sm_t() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pairsum<T, MODE, RPT, NT>, NT, 0) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n > 0 ? n : 1;
}

template <int MODE>
static int blocks_per_sm_mode(bool fp64, int rpt) {
    if (fp64) return rpt >= 2 ? blocks_per_sm_t<double, MODE, 2, 128>() : blocks_per_sm_t<double, MODE, 1, 128>();
    if (rpt >= 4) return blocks_per_sm_t<float, MODE, 4, 256>();
    return rpt == 2 ? blocks_per_sm_t<float, MODE, 2, 256>() : blocks_per_sm_t<float, MODE, 1, 256>();
}

static int pairsum_blocks_per_sm(int mode, bool fp64, int rpt) {
    switch (mode) {
        case MODE_EUW: return blocks_per_sm_mode<MODE_EUW>(fp64, rpt);
        case MODE_ABC: return blocks_per_sm_mode<MODE_ABC>(fp64, rpt);
        case MODE_EUWABC: return blocks_per_sm_mode<MODE_EUWABC>(fp64, rpt);
        case MODE_EUWABCG: return blocks_per_sm_mode<MODE_EUWABCG>(fp64, rpt);
        default: return blocks_per_sm_mode<MODE_GRAD>(fp64, rpt);
    }
}

// j-splits for a launch: the grid (row tiles x splits) is sized to fill the resident CTA
// slots in as close to whole waves as possible (a partial last wave leaves SMs idle while
// it runs); among choices within 1 % of the best, the fewest splits.
int pairsum_default_split(const PointsDev& p, int mode, bool fp64, int rpt, int n_sm) {
    const int NT = fp64 ? 128 : 256;
    const int64_t n_itile = cdiv(p.nk, static_cast<int64_t>(NT) * rpt);
    const double slots = static_cast<double>(n_sm) * pairsum_blocks_per_sm(mode, fp64, rpt);
    int best = 1;
    double best_eff = -1.0;
    for (int req = 1; req <= 16; ++req) {
        int64_t jps;
        int ns;
        split_geometry(p.nk_pad, req, jps, ns);
        const double w = static_cast<double>(n_itile * ns) / slots;
        const double eff = w / std::ceil(w);
        if (eff > best_eff + 0.01) {
            best_eff = eff;
            best = ns;
        }
    }
    return best;
}

template <class T, int MODE, int RPT, int NT>
static cudaError_t launch_t(const PointsDev& p, const typename Recs<T>::A* ra,
                            const typename Recs<T>::B* rb, int req_split, int stall,
                            double* part, int* err, cudaStream_t st) {
    int64_t jps;
    int ns;
    split_geometry(p.nk_pad, req_split, jps, ns);
    dim3 grid(static_cast<unsigned>(cdiv(p.nk, static_cast<int64_t>(NT) * RPT)),
              static_cast<unsigned>(ns));
    k_pairsum<T, MODE, RPT, NT><<<grid, NT, 0, st>>>(ra, rb, p.nk, p.nk_pad, jps, part, err,
                                                     stall);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_mode(const PointsDev& p, bool fp64, const PairLaunch& cfg, double* part,
                               int* err, cudaStream_t st) {
    if (fp64) {
        if (cfg.rows_per_thread >= 2)
            return launch_t<double, MODE, 2, 128>(p, p.r64a, p.r64b, cfg.n_split, cfg.stall, part, err, st);
        return launch_t<double, MODE, 1, 128>(p, p.r64a, p.r64b, cfg.n_split, cfg.stall, part, err, st);
    }
    if (cfg.rows_per_thread >= 4)
        return launch_t<float, MODE, 4, 256>(p, p.r32a, p.r32b, cfg.n_split, cfg.stall, part, err, st);
    if (cfg.rows_per_thread == 2)
        return launch_t<float, MODE, 2, 256>(p, p.r32a, p.r32b, cfg.n_split, cfg.stall, part, err, st);
    return launch_t<float, MODE, 1, 256>(p, p.r32a, p.r32b, cfg.n_split, cfg.stall, part, err, st);
}

int pairsum_split_count(int64_t nk_pad, int req) {
    int64_t jps;
    int ns;
    split_geometry(nk_pad, req, jps, ns);
    return ns;
}

cudaError_t launch_pairsum(const PointsDev& p, int mode, bool fp64, const PairLaunch& cfg,
                           double* part, int* err, cudaStream_t st) {
    if (p.nk == 0) return cudaSuccess;
    switch (mode) {
        case MODE_EUW: return launch_mode<MODE_EUW>(p, fp64, cfg, part, err, st);
        case MODE_ABC: return launch_mode<MODE_ABC>(p, fp64, cfg, part, err, st);
        case MODE_EUWABC: return launch_mode<MODE_EUWABC>(p, fp64, cfg, part, err, st);
        case MODE_EUWABCG: return launch_mode<MODE_EUWABCG>(p, fp64, cfg, part, err, st);
        default: return launch_mode<MODE_GRAD>(p, fp64, cfg, part, err, st);
    }
}

// ------------------------------------------------------------------ epilogues
constexpr int kEpThreads = 256;
int ep_epilogue_blocks(int64_t nk) { return static_cast<int>(cdiv(nk > 0 ? nk : 1, kEpThreads)); }

__device__ __forceinline__ double sum_splits(const double* part, int q, int n_split,
                                             int64_t nk_pad, int64_t p) {
    double s = 0.0;
    for (int k = 0; k < n_split; ++k) s += part[(static_cast<int64_t>(q) * n_split + k) * nk_pad + p];
    return s;
}

// One block of the energy/potential epilogue: kept points 256 blk .. (block sums into
// eblk[blk]).
__device__ __forceinline__ void ep_epilogue_block(const PointsDev& P, const double* __restrict__ part,
                                                  int n_split, double* __restrict__ E,
                                                  double* __restrict__ U, double* __restrict__ W,
                                                  double* __restrict__ vrho,
                                                  double* __restrict__ vgamma,
                                                  double* __restrict__ eblk, int* err, int64_t blk) {
    __shared__ double sh[kEpThreads / 32];
    const int64_t p = blk * kEpThreads + threadIdx.x;
    double ei = 0.0;
    if (p < P.nk) {
        const double e = sum_splits(part, 0, n_split, P.nk_pad, p);
        const double u = -sum_splits(part, 1, n_split, P.nk_pad, p);
        const double wv = -sum_splits(part, 2, n_split, P.nk_pad, p);
        E[p] = e;
        U[p] = u;
        W[p] = wv;
        const double r = P.rho[p];
        const double fr = P.beta + e + r * (P.ka_r[p] * u + P.om_r[p] * wv);  // f^rho
        const double fg = r * P.om_g[p] * wv;                                  // f^gamma
        const int64_t i = P.orig[p];
        if (vrho) vrho[i] = fr;
        if (vgamma) vgamma[i] = fg;
        if (!isfinite(fr) || !isfinite(fg)) atomicOr(err, DEVERR_NONFINITE);
        ei = P.w[p] * r * (P.beta + 0.5 * e);
    }
    const double s = block_sum(ei, sh);
    if (threadIdx.x == 0) eblk[blk] = s;
}

__global__ void __launch_bounds__(kEpThreads)
k_ep_epilogue(PointsDev P, const double* __restrict__ part, int n_split, double* __restrict__ E,
              double* __restrict__ U, double* __restrict__ W, double* __restrict__ vrho,
              double* __restrict__ vgamma, double* __restrict__ eblk, int* err) {
    ep_epilogue_block(P, part, n_split, E, U, W, vrho, vgamma, eblk, err, blockIdx.x);
}

__global__ void __launch_bounds__(kEpThreads)
k_ep_epilogue_batch(const EpiMol* __restrict__ mols, const int64_t* __restrict__ pre, int n_mol,
                    double* __restrict__ vrho, double* __restrict__ vgamma, int* err) {
    int64_t blk;
    const EpiMol& M = mols[batch_block_mol(pre, n_mol, blockIdx.x, blk)];
    ep_epilogue_block(M.P, M.part, M.n_split, M.sums, M.sums + M.cap, M.sums + 2 * M.cap,
                      vrho ? vrho + M.off : nullptr, vgamma ? vgamma + M.off : nullptr, M.eblk,
                      err, blk);
}

cudaError_t launch_ep_epilogue_batch(const EpiMol* mols, const int64_t* pre, int n_mol, int64_t n_blocks,
                                     double* vrho, double* vgamma, int* err, cudaStream_t st) {
    if (n_blocks <= 0) return cudaSuccess;
    k_ep_epilogue_batch<<<static_cast<unsigned>(n_blocks), kEpThreads, 0, st>>>(mols, pre, n_mol,
                                                                                vrho, vgamma, err);
    return cudaGetLastError();
}

cudaError_t launch_ep_epilogue(const PointsDev& p, const double* part, int n_split, double* E,
                               double* U, double* W, double* vrho, double* vgamma,
                               double* eblk, int* err, cudaStream_t st) {
    k_ep_epilogue<<<ep_epilogue_blocks(p.nk), kEpThreads, 0, st>>>(p, part, n_split, E, U, W,
                                                                    vrho, vgamma, eblk, err);
    return cudaGetLastError();
}

// Compensated (Neumaier per thread, TwoSum tree across threads) sum of block partials.
__device__ __forceinline__ void sum_blocks_body(const double* __restrict__ v, int n,
                                                double* __restrict__ out) {
    __shared__ double ss[256], sc[256];
    double s = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) {
        const double x = v[k];
        const double t = s + x;
        c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            double hi, lo;
            two_sum(ss[threadIdx.x], ss[threadIdx.x + o], hi, lo);
            ss[threadIdx.x] = hi;
            sc[threadIdx.x] += sc[threadIdx.x + o] + lo;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = ss[0] + sc[0];
}

__global__ void __launch_bounds__(256) k_sum_blocks(const double* __restrict__ v, int n,
                                                    double* __restrict__ out) {
    sum_blocks_body(v, n, out);
}

// One block per molecule: its energy from its block partials.
__global__ void __launch_bounds__(256) k_sum_blocks_batch(const EpiMol* __restrict__ mols,
                                                          double* __restrict__ energies) {
    const EpiMol& M = mols[blockIdx.x];
    sum_blocks_body(M.eblk, M.nblk, energies + blockIdx.x);
}

cudaError_t launch_sum_blocks_batch(const EpiMol* mols, int n_mol, double* energies,
                                    cudaStream_t st) {
    if (n_mol <= 0) return cudaSuccess;
    k_sum_blocks_batch<<<n_mol, 256, 0, st>>>(mols, energies);
    return cudaGetLastError();
}

cudaError_t launch_sum_blocks(const double* eblk, int nblk, double* out, cudaStream_t st) {
    k_sum_blocks<<<1, 256, 0, st>>>(eblk, nblk, out);
    return cudaGetLastError();
}

__device__ __forceinline__ void abc_epilogue_row(const PointsDev& P, const double* __restrict__ part,
                                                 int n_split, double* __restrict__ A,
                                                 double* __restrict__ B, double* __restrict__ C,
                                                 int64_t p) {
    if (p >= P.nk) return;
    A[p] = 2.0 * sum_splits(part, 0, n_split, P.nk_pad, p);
    B[p] = 2.0 * sum_splits(part, 1, n_split, P.nk_pad, p);
    C[p] = 2.0 * sum_splits(part, 2, n_split, P.nk_pad, p);
}

__global__ void k_abc_epilogue(PointsDev P, const double* __restrict__ part, int n_split,
                               double* __restrict__ A, double* __restrict__ B,
                               double* __restrict__ C) {
    abc_epilogue_row(P, part, n_split, A, B, C, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
}

// A/B/C from quantities 3..5 of each molecule's EUWABC partials.
__global__ void __launch_bounds__(kEpThreads)
k_abc_epilogue_batch(const EpiMol* __restrict__ mols, const int64_t* __restrict__ pre, int n_mol) {
    int64_t blk;
    const EpiMol& M = mols[batch_block_mol(pre, n_mol, blockIdx.x, blk)];
    abc_epilogue_row(M.P, M.part + 3 * static_cast<int64_t>(M.n_split) * M.P.nk_pad, M.n_split,
                     M.sums + 3 * M.cap, M.sums + 4 * M.cap, M.sums + 5 * M.cap,
                     blk * kEpThreads + threadIdx.x);
}

cudaError_t launch_abc_epilogue_batch(const EpiMol* mols, const int64_t* pre, int n_mol, int64_t n_blocks,
                                      cudaStream_t st) {
    if (n_blocks <= 0) return cudaSuccess;
    k_abc_epilogue_batch<<<static_cast<unsigned>(n_blocks), kEpThreads, 0, st>>>(mols, pre, n_mol);
    return cudaGetLastError();
}

cudaError_t launch_abc_epilogue(const PointsDev& p, const double* part, int n_split, double* A,
                                double* B, double* C, cudaStream_t st) {
    if (p.nk == 0) return cudaSuccess;
    k_abc_epilogue<<<ep_epilogue_blocks(p.nk), kEpThreads, 0, st>>>(p, part, n_split, A, B, C);
    return cudaGetLastError();
}

__global__ void k_weight_grad(PointsDev P, const double* __restrict__ E, double* __restrict__ out) {
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= P.nk) return;
    out[P.orig[p]] = P.rho[p] * (P.beta + E[p]);  // dE/dw_i = rho_i (beta + E_i)
}

cudaError_t launch_weight_grad(const PointsDev& p, const double* E, double* dEdw,
                               cudaStream_t st) {
    if (p.nk == 0) return cudaSuccess;
    k_weight_grad<<<ep_epilogue_blocks(p.nk), kEpThreads, 0, st>>>(p, E, dEdw);
    return cudaGetLastError();
}

}  // namespace vv10
