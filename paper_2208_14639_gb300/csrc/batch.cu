// K5: one persistent launch of the pair sums over many molecules.
//
// The work is a table of tasks (molecule, row tile, j-split) ordered largest molecule
// first.  Each CTA repeatedly takes the next task from a global counter (an atomic
// work queue: no CTA ever waits for another), evaluates it with the same tile loop as
// the single-system kernel and writes that task's FP64 partial sums into its molecule's
// partial buffer.  The per-molecule epilogues then reduce the splits in a fixed order.
#include "common.cuh"
#include "kernels.hpp"
#include "pairsum.cuh"

namespace vv10 {

template <class T, int MODE, int RPT, int NT>
__global__ void __launch_bounds__(NT)
k_pairsum_batch(const PairMol* __restrict__ mols, const PairTask* __restrict__ tasks,
                int n_tasks, int* __restrict__ counter, int* __restrict__ err) {
    using RA = typename Recs<T>::A;
    using RB = typename Recs<T>::B;
    __shared__ __align__(128) RA sa[2][kJTile];
    __shared__ __align__(128) RB sb[2][kJTile];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int task_id;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    uint32_t gtile = 0;  // tiles this CTA has streamed (selects buffer and phase)
    for (;;) {
        if (tid == 0) task_id = atomicAdd(counter, 1);
        __syncthreads();
        const int q = task_id;
        __syncthreads();  // everyone has read task_id before thread 0 overwrites it
        if (q >= n_tasks) break;
        const PairTask tk = tasks[q];
        const PairMol m = mols[tk.mol];
        const RA* ra = static_cast<const RA*>(sizeof(T) == 8 ? m.ra64 : m.ra32);
        const RB* rb = static_cast<const RB*>(sizeof(T) == 8 ? m.rb64 : m.rb32);
        const int64_t i0 = static_cast<int64_t>(tk.row_tile) * (NT * RPT);
        const int64_t jb = static_cast<int64_t>(tk.split) * m.j_per_split;
        const int64_t je = min(m.nk_pad, jb + m.j_per_split);
        double dacc[RPT][pair_mode_nq(MODE)];
        const bool ok = pairsum_range<T, MODE, RPT, NT>(sa, sb, bar, gtile, ra, rb, m.nk, i0, jb, je,
                                                        dacc, err, false);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int64_t i = i0 + r * NT + tid;
            if (i < m.nk) {
#pragma unroll
                for (int c = 0; c < pair_mode_nq(MODE); ++c)
                    m.part[(static_cast<int64_t>(c) * m.n_split + tk.split) * m.nk_pad + i] = dacc[r][c];
            }
        }
        if (!ok) break;  // a wait gave up: leave the rest of the queue (error already flagged)
    }
}

template <class T, int MODE, int RPT, int NT>
static cudaError_t launch_batch_t(const PairMol* mols, const PairTask* tasks, int n_tasks,
                                  int* counter, int n_sm, int* err, cudaStream_t st) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_pairsum_batch<T, MODE, RPT, NT>, NT, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int grid = n_sm * per_sm;
    if (grid > n_tasks) grid = n_tasks;
    if (grid < 1) return cudaSuccess;
    k_pairsum_batch<T, MODE, RPT, NT><<<grid, NT, 0, st>>>(mols, tasks, n_tasks, counter, err);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_batch_mode(const PairMol* mols, const PairTask* tasks, int n_tasks,
                                     int* counter, bool fp64, int rpt, int n_sm, int* err,
                                     cudaStream_t st) {
    if (fp64) {
        if (rpt >= 2) return launch_batch_t<double, MODE, 2, 128>(mols, tasks, n_tasks, counter, n_sm, err, st);
        return launch_batch_t<double, MODE, 1, 128>(mols, tasks, n_tasks, counter, n_sm, err, st);
    }
    if (rpt >= 4) return launch_batch_t<float, MODE, 4, 256>(mols, tasks, n_tasks, counter, n_sm, err, st);
    if (rpt == 2) return launch_batch_t<float, MODE, 2, 256>(mols, tasks, n_tasks, counter, n_sm, err, st);
    return launch_batch_t<float, MODE, 1, 256>(mols, tasks, n_tasks, counter, n_sm, err, st);
}

cudaError_t launch_pairsum_batch(const PairMol* mols, const PairTask* tasks, int n_tasks,
                                 int* counter, int mode, bool fp64, int rows_per_thread, int n_sm,
                                 int* err, cudaStream_t st) {
    if (n_tasks <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    switch (mode) {
        case MODE_EUW: return launch_batch_mode<MODE_EUW>(mols, tasks, n_tasks, counter, fp64, rows_per_thread, n_sm, err, st);
        case MODE_ABC: return launch_batch_mode<MODE_ABC>(mols, tasks, n_tasks, counter, fp64, rows_per_thread, n_sm, err, st);
        case MODE_EUWABC: return launch_batch_mode<MODE_EUWABC>(mols, tasks, n_tasks, counter, fp64, rows_per_thread, n_sm, err, st);
        default: return launch_batch_mode<MODE_GRAD>(mols, tasks, n_tasks, counter, fp64, rows_per_thread, n_sm, err, st);
    }
}

int pairsum_rows_per_cta(bool fp64, int rows_per_thread) { return (fp64 ? 128 : 256) * rows_per_thread; }

}  // namespace vv10
