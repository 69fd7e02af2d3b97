// K3 on tensor cores: the pair part of Eq. frhot (Sec. II.B) as a product of generated
// kernel tiles with the trial matrix, split-TF32 (hi*hi + hi*lo + lo*hi) on tcgen05.
//
// Work unit ("tile"): 128 rows i (TMEM lanes) x one output kind (0: f^{rho,t} with
// kernel tiles T1 | T2, 1: f^{gamma,t} / sigma_i with T3 | T4) x all P trials (N of the
// MMA, padded to a multiple of 32, <= 192) x every j.  A persistent CTA walks its tiles;
// per stage of 16 j:
//   * 16 generator warps (4 per TMEM lane quadrant, 4 j each) evaluate the two kernel
//     tiles for their row in FP32, split them into TF32 hi/lo and store the four 128x16
//     operand tiles into tensor memory (tcgen05.st);
//   * the producer warp fetches the stage's j-records (1-D bulk copy) and the four
//     16 x P trial tiles u_hi, u_lo, y_hi, y_lo (2-D TMA, 64-byte swizzle) into a ring;
//   * one thread issues 12 MMAs per output kind (2 k-steps x 6 products) into a TMEM
//     accumulator (double-buffered), the first of each stage overwriting it, and commits
//     the stage once;
//   * the generator warps drain the finished stage's accumulator into FP32 registers
//     (round-to-nearest adds), release the stage's ring slot, and every `flush` stages
//     add the registers into the FP64 partial output in global memory (each tile's rows
//     are owned by one CTA: no atomics).
// The tensor core accumulates with truncation, so each TMEM accumulation run is kept to
// one stage, with the hi*lo and lo*hi products first and the four hi*hi products last
// (bits are lost at the scale of the stage sum only in those four adds); the register and
// FP64 levels bound the rest of the rounding.
#include <cstring>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.hpp"
#include "tc.cuh"

namespace vv10 {

constexpr int kTcKj = 16;                        // j per stage
constexpr int kTcGenWarps = 16;                  // generator / drain warps (4 per lane quadrant)
constexpr int kTcProducerWarp = kTcGenWarps;     // TMA producer
constexpr int kTcMmaWarp = kTcGenWarps + 1;      // MMA issuer + TMEM owner
constexpr int kTcThreads = (kTcGenWarps + 2) * 32;
constexpr int kTcRing = 4;                       // stages of trial tiles in flight
constexpr int kTcMaxPpad = 192;
constexpr uint32_t kTmemCols = 512;
// TMEM columns: accumulator buffer b at kDCol * b, A-operand staging buffer b (4 tiles x 16
// columns) at kACol0 + 64 * b.
constexpr uint32_t kDCol = 192;
constexpr uint32_t kACol0 = 384;

struct TcSmemLayout {
    uint32_t ring_bytes;  // per ring slot: 4 trial tiles
    uint32_t tile_bytes;  // one 16 x Ppad trial tile (64 B rows)
    uint32_t rec_off;     // j-records region
    uint32_t bar_off;     // barriers
    uint32_t total;
};
__host__ __device__ inline TcSmemLayout tc_layout(int ppad) {
    TcSmemLayout L;
    L.tile_bytes = static_cast<uint32_t>(ppad) * 64u;
    L.ring_bytes = 4u * L.tile_bytes;
    L.rec_off = kTcRing * L.ring_bytes;
    L.bar_off = L.rec_off + kTcRing * 512u;
    L.total = L.bar_off + 256u + 1024u;  // barriers + slack for 1024-B alignment
    return L;
}

// One system (molecule) of a tensor-core launch.
struct TcMol {
    const float4* r32a;     // row records (x, y, z, c) and (omega, kappa, p, q)
    const float4* r32b;
    const float4* r32p;     // pair-packed column records
    const CUtensorMap* maps;  // u_hi, u_lo, y_hi, y_lo maps in global memory (batch), or null
    double* acc;            // [2][acc_P][nk_pad] FP64 partial output, zero on entry
    int64_t nk, nk_pad, acc_P;
    int32_t Pn, t0;         // trials of this launch and the first one's row in the split arrays
};
// One work unit: 128 rows of molecule `mol`, output kind (ignored when both kinds share a tile).
struct TcTask {
    int32_t mol, row_tile, kind, pad;
};
struct TcArgs {
    TcMol single;           // the system of a single-system launch
    const TcMol* mols;      // batch: molecule table (null for a single system)
    const TcTask* tasks;    // batch: task table, largest molecules first (null: implicit)
    int64_t n_tasks;
    int flush;              // stages per FP64 flush
    int* err;
};

template <int NK>
__device__ __forceinline__ TcTask tc_task(const TcArgs& a, int64_t q) {
    if (a.tasks) return a.tasks[q];
    TcTask t;
    t.mol = 0;
    t.row_tile = static_cast<int32_t>(NK == 2 ? q : (q >> 1));
    t.kind = NK == 2 ? 0 : static_cast<int32_t>(q & 1);
    t.pad = 0;
    return t;
}

__device__ __forceinline__ void tmap_acquire(const CUtensorMap* m) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     reinterpret_cast<uint64_t>(m))
                 : "memory");
}

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, int* err,
                                              volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kSpinCycles) {
            atomicOr(err, DEVERR_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// Kernel tiles for two j at once (packed FP32x2 arithmetic) from a pair-packed record
// v0..v3 = {-x,-y}, {-z,om}, {ka,-p}, {-q,c} (two lanes each), against row i.
// With inv = 1/(g g' s), L = 1/s, G_i = 1/g, G_j = 1/g', M = 2/s^2 + 2/(g g'),
// nA_i = -rho_i a_i, nA_j = -rho_j a_j and rp = R^2 inv, the values produced are
//   T1c = inv (1 + nA_i (L+G_i) + nA_j (L+G_j) + nA_i nA_j M)   = T1 / (-3/2)
//   T2c = rp (nA_i M + L + G_j)                                   = T2 / (+3/2)
//   T3c = rp (nA_j M + L + G_i)                                   = T3 / (+3/2)
//   T4c = rp R^2 M                                                = T4 / (-3/2)
// The trial split carries u -> -3/2 u and y -> +3/2 y, so the rho accumulator receives
// sum T1 u + T2 y and the gamma accumulator receives -(sum T3 u + T4 y) (its flush
// negates).  The hardware reciprocal (relative error below 2^-22) suffices for operands
// carried to ~22 bits.  NK = 2: all four tiles; NK = 1: the two of output `kind`.
struct RowC {
    float2 x, y, z, om, ka, np, nq;  // row i values, both lanes equal; np = -p_i, nq = -q_i
};
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

template <int NK>
__device__ __forceinline__ void pair_tiles2(int kind, const RowC& r, const float4 v0,
                                            const float4 v1, const float4 v2, const float4 v3,
                                            float2 (&t)[2 * NK]) {
    const float2 one = make_float2(1.0f, 1.0f), two = make_float2(2.0f, 2.0f);
    const float2 dx = __fadd2_rn(r.x, lo2(v0));
    const float2 dy = __fadd2_rn(r.y, hi2(v0));
    const float2 dz = __fadd2_rn(r.z, lo2(v1));
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    const float2 g = __ffma2_rn(r.om, r2, r.ka);
    const float2 gp = __ffma2_rn(hi2(v1), r2, lo2(v2));
    const float2 s = __fadd2_rn(g, gp);
    const float2 ggp = __fmul2_rn(g, gp);
    const float2 den = __fmul2_rn(ggp, s);
    float2 inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv.x) : "f"(den.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv.y) : "f"(den.y));
    const float2 L = __fmul2_rn(ggp, inv);
    const float2 Gi = __fmul2_rn(__fmul2_rn(gp, s), inv);
    const float2 Gj = __fmul2_rn(__fmul2_rn(g, s), inv);
    const float2 M = __fmul2_rn(two, __ffma2_rn(L, L, __fmul2_rn(Gi, Gj)));
    const float2 nAi = __ffma2_rn(r.nq, r2, r.np);
    const float2 nAj = __ffma2_rn(lo2(v3), r2, hi2(v2));
    const float2 rp = __fmul2_rn(r2, inv);
    const float2 LGi = __fadd2_rn(L, Gi), LGj = __fadd2_rn(L, Gj);
    if (NK == 2 || kind == 0) {
        float2 br = __ffma2_rn(nAi, LGi, one);
        br = __ffma2_rn(nAj, LGj, br);
        br = __ffma2_rn(__fmul2_rn(nAi, nAj), M, br);
        t[0] = __fmul2_rn(inv, br);                       // T1c
        t[1] = __fmul2_rn(rp, __ffma2_rn(nAi, M, LGj));   // T2c
    }
    if (NK == 2 || kind == 1) {
        t[2 * NK - 2] = __fmul2_rn(rp, __ffma2_rn(nAj, M, LGi));  // T3c
        t[2 * NK - 1] = __fmul2_rn(__fmul2_rn(rp, r2), M);        // T4c
    }
}

// FP32 -> TF32 with round-to-nearest, ties away from zero, on the bit pattern (finite x):
// add half a TF32 ulp to the magnitude and clear the 13 low mantissa bits.
__device__ __forceinline__ uint32_t tf32_rna_bits(float x) {
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

// TMEM column map.  NK = 1 (Ppad <= 192): accumulator buffer b at 192 b, operand buffer
// b (4 tiles x 16 columns) at 384 + 64 b.  NK = 2 (Ppad <= 64): accumulator (kind k,
// buffer b) at 64 (2k + b), operand buffer b (8 tiles x 16 columns) at 256 + 128 b.
template <int NK>
__device__ __forceinline__ uint32_t d_col(int kind, int b) {
    return NK == 1 ? 192u * b : 64u * (2 * kind + b);
}
template <int NK>
__device__ __forceinline__ uint32_t a_col(int b) {
    return NK == 1 ? 384u + 64u * b : 256u + 128u * b;
}

template <int PQ, int NK>  // PQ accumulator columns per generator thread (= Ppad / 4)
__global__ void __launch_bounds__(kTcThreads, 1)
k_hess_tc(const __grid_constant__ CUtensorMap tm_uh, const __grid_constant__ CUtensorMap tm_ul,
          const __grid_constant__ CUtensorMap tm_yh, const __grid_constant__ CUtensorMap tm_yl,
          TcArgs args) {
    constexpr int PPAD = 4 * PQ;
    static_assert(NK == 1 || PPAD <= 64, "two kinds per tile need Ppad <= 64");
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-B aligned base (the 64-B swizzle pattern repeats every 512 B)
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const TcSmemLayout L = tc_layout(PPAD);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* b_full = bars;                   // [kTcRing]
    uint64_t* b_empty = bars + kTcRing;        // [kTcRing]
    uint64_t* a_full = bars + 2 * kTcRing;     // [2]
    uint64_t* mma_done = bars + 2 * kTcRing + 2;  // [2]
    uint64_t* fin = bars + 2 * kTcRing + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kTcRing + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * kTcRing + 6);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // a task = 128 rows of one molecule x (both kinds if NK == 2, else one kind)
    const int64_t n_tiles = args.n_tasks;

    if (threadIdx.x == 0) {
        for (int b = 0; b < kTcRing; ++b) {
            mbar_init(&b_full[b], 1);
            mbar_init(&b_empty[b], kTcGenWarps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&a_full[b], kTcGenWarps);
            mbar_init(&mma_done[b], 1);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kTcMmaWarp) tc::tmem_alloc(tmem_slot, kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == kTcProducerWarp) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int slot = 0;
            uint32_t ph = 0;   // phase bit of the ring slot's current use
            int64_t issued = 0;
            bool ok = true;
            int cur_mol = -1;
            const CUtensorMap* mp[4] = {&tm_uh, &tm_ul, &tm_yh, &tm_yl};
            for (int64_t q = blockIdx.x; q < n_tiles && ok; q += gridDim.x) {
                const TcTask tk = tc_task<NK>(args, q);
                const TcMol M = args.mols ? args.mols[tk.mol] : args.single;
                if (tk.mol != cur_mol) {  // a new molecule's tensor maps
                    cur_mol = tk.mol;
                    for (int k = 0; k < 4; ++k) {
                        if (M.maps) {
                            mp[k] = M.maps + k;
                            tmap_acquire(mp[k]);
                        }
                        tc::prefetch_tmap(mp[k]);
                    }
                }
                const int n_stage = static_cast<int>(M.nk_pad / kTcKj);
                for (int s = 0; s < n_stage; ++s) {
                    if (!wait_or_abort(&b_empty[slot], ph ^ 1u, args.err, abort_flag)) {
                        ok = false;
                        break;
                    }
                    uint8_t* base = smem + slot * L.ring_bytes;
                    uint8_t* rec = smem + L.rec_off + slot * 512;
                    const int j0 = s * kTcKj;
                    mbar_expect_tx(&b_full[slot], L.ring_bytes + 512u);
                    bulk_g2s(rec, M.r32p + 2 * j0, 512u, &b_full[slot]);
                    tc::tma_load_2d(base + 0 * L.tile_bytes, mp[0], j0, M.t0, &b_full[slot]);
                    tc::tma_load_2d(base + 1 * L.tile_bytes, mp[1], j0, M.t0, &b_full[slot]);
                    tc::tma_load_2d(base + 2 * L.tile_bytes, mp[2], j0, M.t0, &b_full[slot]);
                    tc::tma_load_2d(base + 3 * L.tile_bytes, mp[3], j0, M.t0, &b_full[slot]);
                    ++issued;
                    if (++slot == kTcRing) {
                        slot = 0;
                        ph ^= 1u;
                    }
                }
            }
            // copies in flight must land before the CTA exits
            for (int64_t k = (issued > kTcRing ? issued - kTcRing : 0); k < issued; ++k)
                mbar_wait(&b_full[k % kTcRing], static_cast<uint32_t>((k / kTcRing) & 1), args.err);
        }
    } else if (warp == kTcMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(128, PPAD);
            int slot = 0, ab = 0;
            uint32_t ph = 0, aph = 0;
            bool ok = true, issued_any = false;
            for (int64_t q = blockIdx.x; q < n_tiles && ok; q += gridDim.x) {
                const TcTask tk = tc_task<NK>(args, q);
                const int kind0 = tk.kind;
                const int64_t nkp = args.mols ? args.mols[tk.mol].nk_pad : args.single.nk_pad;
                const int n_stage = static_cast<int>(nkp / kTcKj);
                for (int s = 0; s < n_stage; ++s) {
                    if (!wait_or_abort(&a_full[ab], aph, args.err, abort_flag) ||
                        !wait_or_abort(&b_full[slot], ph, args.err, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t base = smem_u32(smem + slot * L.ring_bytes);
                    const uint32_t a = tmem + a_col<NK>(ab);
#pragma unroll
                    for (int k = 0; k < NK; ++k) {
                        const uint32_t d = tmem + d_col<NK>(NK == 2 ? k : kind0, ab);
                        const uint32_t at = a + 64u * k;  // this kind's 4 operand tiles
                        // K-step kk: 8 tf32 along K inside the 64-B rows of the trial tiles
                        const uint64_t duh0 = tc::sdesc_kmajor_sw64(base + 0 * L.tile_bytes);
                        const uint64_t dul0 = tc::sdesc_kmajor_sw64(base + 1 * L.tile_bytes);
                        const uint64_t dyh0 = tc::sdesc_kmajor_sw64(base + 2 * L.tile_bytes);
                        const uint64_t dyl0 = tc::sdesc_kmajor_sw64(base + 3 * L.tile_bytes);
                        constexpr uint64_t kStep = 32u >> 4;  // +32 B in the descriptor's address field
                        // The small products (hi*lo, lo*hi) go first, while the accumulator is
                        // still small, and the four hi*hi products last: the truncating
                        // accumulation then loses bits at the scale of the stage sum only four
                        // times per stage.
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t ah = at + 0 + 8 * kk, al = at + 16 + 8 * kk;
                            const uint32_t bh = at + 32 + 8 * kk, bl = at + 48 + 8 * kk;
                            tc::mma_tf32_ts(d, ah, dul0 + kStep * kk, idesc, kk);  // the first overwrites
                            tc::mma_tf32_ts(d, al, duh0 + kStep * kk, idesc, 1);
                            tc::mma_tf32_ts(d, bh, dyl0 + kStep * kk, idesc, 1);
                            tc::mma_tf32_ts(d, bl, dyh0 + kStep * kk, idesc, 1);
                        }
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            tc::mma_tf32_ts(d, at + 0 + 8 * kk, duh0 + kStep * kk, idesc, 1);
                            tc::mma_tf32_ts(d, at + 32 + 8 * kk, dyh0 + kStep * kk, idesc, 1);
                        }
                    }
                    issued_any = true;
                    tc::commit(&mma_done[ab]);  // the ring slot is released by the generators
                    if (++slot == kTcRing) {
                        slot = 0;
                        ph ^= 1u;
                    }
                    ab ^= 1;
                    if (ab == 0) aph ^= 1u;
                }
            }
            if (issued_any) {  // every MMA finished before TMEM is released
                tc::commit(fin);
                mbar_wait(fin, 0, args.err);
            }
        }
    } else {
        // ------------------------------------------------------------ generators
        const int quad = warp & 3, part = warp >> 2;
        const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
        float acc[NK][PQ];
#pragma unroll
        for (int k = 0; k < NK; ++k)
#pragma unroll
            for (int c = 0; c < PQ; ++c) acc[k][c] = 0.0f;
        bool ok = true;

        // Drain a finished accumulator (all kinds of this tile) into the FP32 registers, in
        // chunks of at most 32 columns so that the staging registers stay few.
        auto drain = [&](int db, uint32_t dphase, int kind0) -> bool {
            const bool got = wait_or_abort(&mma_done[db], dphase, args.err, abort_flag);
            if (!__all_sync(0xffffffffu, got)) return false;  // warp-uniform exit
            tc::fence_after();
            constexpr int kCols = NK * PQ;  // this thread's accumulator columns
            constexpr int kChunk = kCols < 32 ? kCols : 32;
#pragma unroll
            for (int c0 = 0; c0 < kCols; c0 += kChunk) {
                uint32_t r[kChunk];
#pragma unroll
                for (int c = 0; c < kChunk; c += 8) {
                    const int col = c0 + c, k = col / PQ, cc = col % PQ;
                    if (col < kCols) {
                        uint32_t (&rc)[8] = *reinterpret_cast<uint32_t(*)[8]>(&r[c]);
                        tc::ld_x8(tmem + lane_off + d_col<NK>(NK == 2 ? k : kind0, db) + part * PQ + cc, rc);
                    }
                }
                tc::wait_ld();
#pragma unroll
                for (int c = 0; c < kChunk; c += 2) {
                    const int col = c0 + c, k = col / PQ, cc = col % PQ;
                    if (col < kCols) {
                        const float2 v = __fadd2_rn(make_float2(acc[k][cc], acc[k][cc + 1]),
                                                    make_float2(__uint_as_float(r[c]), __uint_as_float(r[c + 1])));
                        acc[k][cc] = v.x;
                        acc[k][cc + 1] = v.y;
                    }
                }
            }
            tc::fence_before();
            return true;
        };
        // descriptor fields are read where they are used (not held across the stage loop)
        auto flush = [&](int mol, int kind0, int64_t i) {
            const TcMol* mp = args.mols ? args.mols + mol : nullptr;
            const int64_t nk = mp ? mp->nk : args.single.nk;
            const int64_t nk_pad = mp ? mp->nk_pad : args.single.nk_pad;
            const int64_t acc_P = mp ? mp->acc_P : args.single.acc_P;
            const int32_t Pn = mp ? mp->Pn : args.single.Pn;
            const int32_t t0 = mp ? mp->t0 : args.single.t0;
            double* acc_base = mp ? mp->acc : args.single.acc;
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const int kind = NK == 2 ? k : kind0;
#pragma unroll
                for (int c = 0; c < PQ; ++c) {
                    const int t = part * PQ + c;
                    if (i < nk && t < Pn) {
                        double* o = acc_base + ((static_cast<int64_t>(kind) * acc_P + t0 + t) * nk_pad + i);
                        const double v = static_cast<double>(acc[k][c]);
                        // the gamma accumulator holds -(T3 u + T4 y); streaming loads and
                        // stores keep the partial output from evicting the trial tiles
                        __stcs(o, __ldcs(o) + ((kind == 0) ? v : -v));
                    }
                    acc[k][c] = 0.0f;
                }
            }
        };

        int slot = 0, ab = 0;
        uint32_t ph = 0, aph = 0;
        int pslot = 0;         // ring slot of the previous stage
        int dbuf = 0;          // accumulator buffer of the previous stage
        uint32_t dph = 0;      // and its phase bit
        for (int64_t q = blockIdx.x; q < n_tiles && ok; q += gridDim.x) {
            const TcTask tk = tc_task<NK>(args, q);
            const TcMol* mp = args.mols ? args.mols + tk.mol : nullptr;
            const int n_stage = static_cast<int>((mp ? mp->nk_pad : args.single.nk_pad) / kTcKj);
            const int kind0 = tk.kind;
            const int64_t i = static_cast<int64_t>(tk.row_tile) * 128 + quad * 32 + lane;
            float xi = 0.f, yi = 0.f, zi = 0.f, oi = 1.f, ki = 1.f, pi_ = 0.f, qi = 0.f;
            if (i < (mp ? mp->nk : args.single.nk)) {
                const float4 a = (mp ? mp->r32a : args.single.r32a)[i];
                const float4 b = (mp ? mp->r32b : args.single.r32b)[i];
                xi = a.x; yi = a.y; zi = a.z; oi = b.x; ki = b.y; pi_ = b.z; qi = b.w;
            }
            const RowC rc{make_float2(xi, xi), make_float2(yi, yi), make_float2(zi, zi),
                          make_float2(oi, oi), make_float2(ki, ki), make_float2(-pi_, -pi_),
                          make_float2(-qi, -qi)};
            int until_flush = args.flush;
            for (int s = 0; s < n_stage; ++s) {
                // operand buffer ab is free once the MMAs of the stage two back are done
                bool got = wait_or_abort(&b_full[slot], ph, args.err, abort_flag);
                got = got && wait_or_abort(&mma_done[ab], aph ^ 1u, args.err, abort_flag);
                if (!__all_sync(0xffffffffu, got)) {  // warp-uniform exit
                    ok = false;
                    break;
                }
                tc::fence_after();  // the MMAs that read this operand buffer are complete
                const float4* rec = reinterpret_cast<const float4*>(smem + L.rec_off + slot * 512);
                {
                    // this warp's 4 j = pair-packed records 2 part and 2 part + 1
                    uint32_t hi[2 * NK][4], lo[2 * NK][4];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float4* v = rec + 4 * (2 * part + h);
                        float2 t[2 * NK];
                        pair_tiles2<NK>(kind0, rc, v[0], v[1], v[2], v[3], t);
#pragma unroll
                        for (int m = 0; m < 2 * NK; ++m) {
                            const uint32_t h0 = tf32_rna_bits(t[m].x), h1 = tf32_rna_bits(t[m].y);
                            const float2 l = __ffma2_rn(make_float2(__uint_as_float(h0), __uint_as_float(h1)),
                                                        make_float2(-1.0f, -1.0f), t[m]);
                            hi[m][2 * h] = h0;
                            hi[m][2 * h + 1] = h1;
                            lo[m][2 * h] = __float_as_uint(l.x);
                            lo[m][2 * h + 1] = __float_as_uint(l.y);
                        }
                    }
                    // operand tiles of kind k: [hi(Ta), lo(Ta), hi(Tb), lo(Tb)], 16 columns each
                    const uint32_t a = tmem + lane_off + a_col<NK>(ab) + part * 4;
#pragma unroll
                    for (int k = 0; k < NK; ++k) {
                        tc::st_x4(a + 64u * k + 0, hi[2 * k]);
                        tc::st_x4(a + 64u * k + 16, lo[2 * k]);
                        tc::st_x4(a + 64u * k + 32, hi[2 * k + 1]);
                        tc::st_x4(a + 64u * k + 48, lo[2 * k + 1]);
                    }
                }
                tc::wait_st();
                tc::fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&a_full[ab]);  // hand the operands to the MMA issuer
                // drain the previous stage while this stage's MMAs run
                if (s > 0) {
                    if (!drain(dbuf, dph, kind0)) {
                        ok = false;
                        break;
                    }
                    // its MMAs are done, and so is this warp's use of its records: the ring
                    // slot of the previous stage can be refilled
                    if (lane == 0) mbar_arrive(&b_empty[pslot]);
                    if (--until_flush == 0) {
                        flush(tk.mol, kind0, i);
                        until_flush = args.flush;
                    }
                }
                dbuf = ab;
                dph = aph;
                pslot = slot;
                if (++slot == kTcRing) {
                    slot = 0;
                    ph ^= 1u;
                }
                ab ^= 1;
                if (ab == 0) aph ^= 1u;
            }
            if (!ok) break;
            if (!drain(dbuf, dph, kind0)) {
                ok = false;
                break;
            }
            if (lane == 0) mbar_arrive(&b_empty[pslot]);
            flush(tk.mol, kind0, i);
        }
        tc::wait_st();  // nothing of ours is in flight to TMEM on any exit path
        tc::wait_ld();
    }

    tc::fence_before();
    __syncthreads();
    if (warp == kTcMmaWarp) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// ---------------------------------------------------------------- host side

__global__ void k_trial_split(const double* __restrict__ u, const double* __restrict__ y,
                              int32_t P, int64_t nk_pad, float* __restrict__ uh,
                              float* __restrict__ ul, float* __restrict__ yh,
                              float* __restrict__ yl) {
    const int t = blockIdx.y;
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= nk_pad) return;
    const int64_t o = static_cast<int64_t>(t) * nk_pad + p;
    float a = 0.f, b = 0.f;
    if (t < P) {  // the kernel tiles omit the -3/2 of Phi and the sign of T2: see pair_tiles2
        a = static_cast<float>(-1.5 * u[o]);
        b = static_cast<float>(1.5 * y[o]);
    }
    const float ah = __uint_as_float(tc::to_tf32(a)), bh = __uint_as_float(tc::to_tf32(b));
    uh[o] = ah;
    ul[o] = a - ah;
    yh[o] = bh;
    yl[o] = b - bh;
}

cudaError_t launch_trial_split(const double* u, const double* y, int32_t P, int32_t Prows,
                               int64_t nk_pad, bool bf16, float* uh, float* ul, float* yh,
                               float* yl, cudaStream_t st) {
    (void)bf16;
    dim3 grid(static_cast<unsigned>((nk_pad + 255) / 256), static_cast<unsigned>(Prows));
    k_trial_split<<<grid, 256, 0, st>>>(u, y, P, nk_pad, uh, ul, yh, yl);
    return cudaGetLastError();
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D map over a [rows][nk_pad] FP32 array, box = 16 j x ppad trials, 64-B swizzle.
static bool make_map(CUtensorMap* m, const float* base, int64_t nk_pad, int64_t rows, int ppad) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(nk_pad), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(nk_pad) * sizeof(float)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kTcKj), static_cast<cuuint32_t>(ppad)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool tc_make_map_f32(void* out, const float* base, int64_t nk_pad, int64_t rows, int ppad) {
    return make_map(static_cast<CUtensorMap*>(out), base, nk_pad, rows, ppad);
}

int hess_tc_ppad(int32_t P) {
    const int p = ((P + 31) / 32) * 32;
    return p < 32 ? 32 : p;
}

template <int PQ, int NK>
static cudaError_t launch_tc_t(const CUtensorMap* maps, const TcArgs& a, int n_sm, cudaStream_t st) {
    const TcSmemLayout L = tc_layout(4 * PQ);
    cudaError_t e = cudaFuncSetAttribute(k_hess_tc<PQ, NK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L.total));
    if (e != cudaSuccess) return e;
    const int grid = static_cast<int>(a.n_tasks < n_sm ? a.n_tasks : n_sm);
    if (grid <= 0) return cudaSuccess;
    k_hess_tc<PQ, NK><<<grid, kTcThreads, L.total, st>>>(maps[0], maps[1], maps[2], maps[3], a);
    return cudaGetLastError();
}

// Both kinds share a tile whenever both accumulators fit in TMEM (Ppad <= 64).
int hess_tc_kinds_per_tile(int ppad) { return ppad <= 64 ? 2 : 1; }

static cudaError_t launch_tc_dispatch(int ppad, const CUtensorMap* maps, const TcArgs& a, int n_sm,
                                      cudaStream_t st) {
    switch (ppad / 4) {
        case 8: return launch_tc_t<8, 2>(maps, a, n_sm, st);
        case 16: return launch_tc_t<16, 2>(maps, a, n_sm, st);
        case 24: return launch_tc_t<24, 1>(maps, a, n_sm, st);
        case 32: return launch_tc_t<32, 1>(maps, a, n_sm, st);
        case 40: return launch_tc_t<40, 1>(maps, a, n_sm, st);
        case 48: return launch_tc_t<48, 1>(maps, a, n_sm, st);
        default: return cudaErrorInvalidValue;
    }
}

// Contract the trials [t0, t0 + Pn) (Pn <= 192) of one system; split arrays have `rows` rows.
cudaError_t launch_hess_tc(const PointsDev& p, int32_t Pn, int32_t t0, int64_t acc_P,
                           const float* uh, const float* ul, const float* yh, const float* yl,
                           int64_t rows, int n_sm, int flush, double* acc, int* err,
                           cudaStream_t st) {
    if (p.nk == 0) return cudaSuccess;
    const int ppad = hess_tc_ppad(Pn);
    if (ppad > kTcMaxPpad) return cudaErrorInvalidValue;
    CUtensorMap maps[4];
    const float* src[4] = {uh, ul, yh, yl};
    for (int k = 0; k < 4; ++k)
        if (!make_map(&maps[k], src[k], p.nk_pad, rows, ppad)) return cudaErrorInvalidValue;
    TcArgs a;
    a.single = TcMol{p.r32a, p.r32b, p.r32p, nullptr, acc, p.nk, p.nk_pad, acc_P, Pn, t0};
    a.mols = nullptr;
    a.tasks = nullptr;
    a.n_tasks = (hess_tc_kinds_per_tile(ppad) == 2 ? 1 : 2) * ((p.nk + 127) / 128);
    a.flush = flush > 0 ? flush : 512;
    a.err = err;
    return launch_tc_dispatch(ppad, maps, a, n_sm, st);
}

// Tensor maps of one molecule of a batched contraction (4 consecutive CUtensorMap).
bool hess_tc_make_maps(void* out4, const float* uh, const float* ul, const float* yh,
                       const float* yl, int64_t nk_pad, int64_t rows, int ppad) {
    CUtensorMap* m = static_cast<CUtensorMap*>(out4);
    const float* src[4] = {uh, ul, yh, yl};
    for (int k = 0; k < 4; ++k)
        if (!make_map(&m[k], src[k], nk_pad, rows, ppad)) return false;
    return true;
}

// Batched contraction: every task of the table shares `ppad`; molecules and tensor maps
// live in device memory (written before the launch).
cudaError_t launch_hess_tc_batch(const void* mols, const void* tasks, int64_t n_tasks, int ppad,
                                 int n_sm, int flush, int* err, cudaStream_t st) {
    if (n_tasks <= 0) return cudaSuccess;
    CUtensorMap unused[4];
    memset(unused, 0, sizeof(unused));
    TcArgs a;
    memset(&a.single, 0, sizeof(a.single));
    a.mols = static_cast<const TcMol*>(mols);
    a.tasks = static_cast<const TcTask*>(tasks);
    a.n_tasks = n_tasks;
    a.flush = flush > 0 ? flush : 512;
    a.err = err;
    return launch_tc_dispatch(ppad, unused, a, n_sm, st);
}

size_t hess_tc_mol_bytes() { return sizeof(TcMol); }
size_t hess_tc_task_bytes() { return sizeof(TcTask); }

void hess_tc_fill_mol(void* dst, const float4* r32a, const float4* r32b, const float4* r32p,
                      const void* maps_dev, double* acc, int64_t nk, int64_t nk_pad, int64_t acc_P,
                      int32_t Pn, int32_t t0) {
    TcMol m{r32a, r32b, r32p, static_cast<const CUtensorMap*>(maps_dev), acc, nk, nk_pad, acc_P, Pn, t0};
    memcpy(dst, &m, sizeof(m));
}

void hess_tc_fill_task(void* dst, int32_t mol, int32_t row_tile, int32_t kind) {
    TcTask t{mol, row_tile, kind, 0};
    memcpy(dst, &t, sizeof(t));
}

}  // namespace vv10
