// K3 on tensor cores with FP16 operands: the pair part of Eq. frhot (Sec. II.B) as a product
// of generated kernel tiles with the trial matrix, split FP16 (hi*hi + hi*lo + lo*hi) on
// tcgen05 kind::f16 with FP32 accumulation (VV10_MIXED_F16X3).
//
// FP16 carries 11 significant bits, like TF32, but only 5 exponent bits, so every operand is
// brought into its range by an exact power of two:
//  * trials (B operand): one factor s_t per trial column t maps the column's largest |u'|,
//    |c_y y'| into [2^14, 2^15) (u' = -3/2 u, y' = 3/2 y as for the TF32 kernel); c_y is one
//    global power of two that balances y against u, and the kernel tiles that multiply y
//    are divided by c_y instead;
//  * kernel tiles (A operand): one factor r per row i and stage (32 j) maps the largest |T|
//    of the row's two tiles in the stage into [2^14, 2^15).
// A stage's accumulator then holds r_i s_t sum_j A_ij B_jt: the drain multiplies by 1/r_i
// before its round-to-nearest FP32 register sum, the flush to FP64 by 1/s_t.  A value far
// below its scale becomes subnormal and keeps an absolute error of at most 2^-25 of the scale
// (2^-40 of the largest element sharing it); every other value is carried to ~22 bits as in
// the TF32 split.  Per stage and output kind the MMA issues 12 instructions of K = 16 (four
// K-steps: u and y of each 16-j half of the 128-byte trial rows; three products each), half
// the instruction count of the TF32 split for the same j.
//
// Work unit: 128 rows i (TMEM lanes) x output kind (both kinds when Ppad <= 64) x the trials
// of the launch (MMA N = Ppad).  The j range is cut into chunks whose trial tiles fit in L2;
// the persistent CTAs walk the chunks in order and, inside a chunk, each CTA its fixed units
// u = blockIdx.x + k gridDim.x, adding its FP32 register sums into the FP64 partial output at
// the end of every unit-chunk.  All CTAs therefore stream the same chunk's trial tiles at
// about the same time (they stay in L2 at any N), and every output row is updated by one
// CTA only, in a fixed order (no atomics).
//
// 16 warps per CTA (4 per TMEM lane quadrant, 8 j each), every one of which, per stage:
// evaluates its part of the two (or four) kernel tiles, exchanges the row maxima of the
// stage with the quadrant's other warps through shared memory, scales, splits and stores
// its operand columns into TMEM, then drains the previous stage's accumulator.  Two single
// threads carry the other roles inside that loop, so that each warp keeps 128 registers
// (four warps per SM sub-partition): lane 0 of warp 0 issues the stage's MMAs once every
// warp's operands are in place, lane 0 of warp 1 keeps the ring of copies (j records by
// 1-D bulk copy, the hi and lo trial tiles by 2-D tensor copies) kF16Ring - 1 stages ahead.
// Every wait is bounded (kSpinCycles); a wait that gives up sets the TIMEOUT bit and an
// abort flag that ends the other waits.
#include <cstring>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.hpp"
#include "tc.cuh"

namespace vv10 {

constexpr int kF16Kj = 32;                      // j per stage
constexpr int kF16Warps = 16;                   // every warp generates and drains
constexpr int kF16ProducerWarp = 1;             // lane 0 also issues the copies
constexpr int kF16MmaWarp = 0;                  // lane 0 also issues the MMAs; owns TMEM
constexpr int kF16Threads = kF16Warps * 32;
constexpr int kF16Ring = 4;                     // stages of trial tiles in flight
constexpr int kF16MaxPpad = 192;
constexpr uint32_t kF16TmemCols = 512;
constexpr size_t kF16ChunkBytes = 24u << 20;    // trial-tile bytes of one j chunk (L2-resident)

struct F16Layout {
    uint32_t tile_bytes;  // one Ppad x 64-half trial tile (128-byte rows: 16 u, 16 y, 16 u, 16 y)
    uint32_t slot_bytes;  // hi and lo tiles of one stage
    uint32_t rec_off;     // j records, 1024 B per stage
    uint32_t xm_off;      // row-maximum exchange [2][4 quads][NK][32 lanes][4 parts] floats
    uint32_t prod_off;    // the producer thread's state
    uint32_t bar_off;
    uint32_t total;
};
__host__ __device__ inline F16Layout f16_layout(int ppad, int nk) {
    F16Layout L;
    L.tile_bytes = static_cast<uint32_t>(ppad) * 128u;
    L.slot_bytes = 2u * L.tile_bytes;
    L.rec_off = kF16Ring * L.slot_bytes;
    L.xm_off = L.rec_off + kF16Ring * 1024u;
    L.prod_off = L.xm_off + 2u * 4u * static_cast<uint32_t>(nk) * 32u * 16u;
    L.bar_off = L.prod_off + 128u;
    L.total = L.bar_off + 512u + 1024u;  // barriers + slack for the 1024-B alignment
    return L;
}

// One system (molecule) of a launch: its records, trial tiles, factors and output.
struct F16Mol {
    const float4* r32a;        // row records (x, y, z, c) and (omega, kappa, p, q)
    const float4* r32b;
    const float4* r32p;        // pair-packed column records
    const CUtensorMap* maps;   // batch: its hi and lo tile maps (device memory); single: unused
    double* acc;               // [2][acc_P][nk_pad] FP64 partial output, zero on entry
    const double* col_isc;     // [acc_P] 1/s_t per trial column
    const float* params;       // [0] = 1/c_y
    int64_t nk, nk_pad, acc_P;
    int32_t Pn, t0;            // trials of this launch and the first one's row
};
// One unit of a batched launch: 128 rows of molecule `mol` x output kind.
struct F16Task {
    int32_t mol, row_tile, kind, pad;
};
struct F16Args {
    F16Mol single;             // the system of a single-system launch
    const F16Mol* mols;        // batch: molecule table (null for a single system)
    const F16Task* tasks;      // batch: units, largest molecules first
    int* counter;              // batch: next unit to take (zero on entry)
    int64_t n_units;           // single: row tiles x kinds per tile's pass; batch: tasks
    int32_t n_stage, chunk;    // single: stages in all, stages per j chunk
    int32_t flush;             // stages per FP64 flush inside a unit-chunk
    int* err;
};

__device__ __forceinline__ void tmap_acquire(const CUtensorMap* m) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     reinterpret_cast<uint64_t>(m))
                 : "memory");
}

__device__ __forceinline__ bool f16_wait(uint64_t* bar, uint32_t parity, int* err,
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

// The FP32 kernel tiles of two j at once against row i, from a pair-packed record
// v0..v3 = {-x,-y}, {-z,om}, {ka,-p}, {-q,c} (two lanes each).  With inv = 1/(g g' s),
// L = 1/s, G_i = 1/g, G_j = 1/g', M = 2/s^2 + 2/(g g'), nA = -rho a and rp = R^2 inv:
//   T1c = inv (1 + nA_i (L+G_i) + nA_j (L+G_j) + nA_i nA_j M)   = T1 / (-3/2)
//   T2c = rp (nA_i M + L + G_j)                                   = T2 / (+3/2)
//   T3c = rp (nA_j M + L + G_i)                                   = T3 / (+3/2)
//   T4c = rp R^2 M                                                = T4 / (-3/2)
// (the factors -3/2, +3/2 travel with the trials).  NK = 2: t = {T1c, T2c, T3c, T4c};
// NK = 1: the two tiles of output `kind`.
struct RowF {
    float x, y, z, om, ka, np, nq;  // row i values; np = -p_i, nq = -q_i
};
__device__ __forceinline__ float2 f16_dup(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 f16_lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 f16_hi2(float4 v) { return make_float2(v.z, v.w); }

template <int NK>
__device__ __forceinline__ void f16_tiles2(int kind, const RowF& r, const float4 v0,
                                           const float4 v1, const float4 v2, const float4 v3,
                                           float2 (&t)[2 * NK]) {
    const float2 one = make_float2(1.0f, 1.0f), two = make_float2(2.0f, 2.0f);
    const float2 dx = __fadd2_rn(f16_dup(r.x), f16_lo2(v0));
    const float2 dy = __fadd2_rn(f16_dup(r.y), f16_hi2(v0));
    const float2 dz = __fadd2_rn(f16_dup(r.z), f16_lo2(v1));
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    const float2 g = __ffma2_rn(f16_dup(r.om), r2, f16_dup(r.ka));
    const float2 gp = __ffma2_rn(f16_hi2(v1), r2, f16_lo2(v2));
    const float2 s = __fadd2_rn(g, gp);
    const float2 ggp = __fmul2_rn(g, gp);
    const float2 den = __fmul2_rn(ggp, s);
    float2 inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv.x) : "f"(den.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv.y) : "f"(den.y));
    const float2 L = __fmul2_rn(ggp, inv);
    const float2 sinv = __fmul2_rn(s, inv);  // 1/(g g')
    const float2 Gi = __fmul2_rn(gp, sinv);
    const float2 Gj = __fmul2_rn(g, sinv);
    const float2 M = __fmul2_rn(two, __ffma2_rn(L, L, sinv));
    const float2 nAi = __ffma2_rn(f16_dup(r.nq), r2, f16_dup(r.np));
    const float2 nAj = __ffma2_rn(f16_lo2(v3), r2, f16_hi2(v2));
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

// Power-of-two factor that maps a maximum m >= 0 into [2^14, 2^15), and its inverse (both
// normal FP32 numbers: the exponent is clamped to [-126, 126]).
__device__ __forceinline__ void f16_scale(float m, float& sc, float& isc) {
    const int eb = static_cast<int>((__float_as_uint(m) >> 23) & 0xFFu);
    int se = 141 - eb;
    se = se > 126 ? 126 : (se < -126 ? -126 : se);
    sc = __uint_as_float(static_cast<uint32_t>(se + 127) << 23);
    isc = __uint_as_float(static_cast<uint32_t>(127 - se) << 23);
}

// Two scaled values -> packed FP16 hi and lo words (lower j in the low half).
__device__ __forceinline__ void f16_split2(float2 x, float sc, uint32_t& hi, uint32_t& lo) {
    x = __fmul2_rn(x, make_float2(sc, sc));
    const __half2 h = __floats2half2_rn(x.x, x.y);
    const float2 hf = __half22float2(h);
    const float2 r = __ffma2_rn(hf, make_float2(-1.0f, -1.0f), x);  // x - hi, exact
    const __half2 l = __floats2half2_rn(r.x, r.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ float f16_absmax4(float2 a, float2 b) {
    return fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(b.x), fabsf(b.y)));
}

// TMEM column map.  NK = 1 (Ppad <= 192): accumulator buffer b at Ppad b, operand buffer b
// (4 tiles x 16 columns) at 2 Ppad + 64 b.  NK = 2 (Ppad <= 64): accumulator (kind k, buffer
// b) at Ppad (2k + b), operand buffer b (2 kinds x 4 tiles x 16 columns) at 4 Ppad + 128 b.
// An operand tile holds the stage's 32 j as 16 columns of two FP16 each.
template <int NK, int PPAD>
__device__ __forceinline__ uint32_t f16_dcol(int kind, int b) {
    return NK == 1 ? static_cast<uint32_t>(PPAD * b) : static_cast<uint32_t>(PPAD * (2 * kind + b));
}
template <int NK, int PPAD>
__device__ __forceinline__ uint32_t f16_acol(int b) {
    return NK == 1 ? static_cast<uint32_t>(2 * PPAD + 64 * b) : static_cast<uint32_t>(4 * PPAD + 128 * b);
}

// Stage metadata the producer writes next to every stage it loads (the walk's single source
// of truth: the other roles follow it).
enum : int32_t { F16_FIRST = 1, F16_LAST = 2, F16_END = 4 };
struct F16Meta {
    int32_t mol, row_tile, kind, flags;
};

// The producer's position in the walk.  Single system: (j chunk c, unit u, stage s), units
// u = blockIdx.x + k gridDim.x inside every chunk.  Batch: (task q, stage s), tasks taken
// from an atomic counter, largest molecules first.
struct F16Cursor {
    int c, s, s0, s1;
    int64_t u;
    int32_t mol, row_tile, kind;
    bool done;
};
// The producer thread's state (shared memory).
struct F16Prod {
    F16Cursor k;
    int64_t issued;
    int32_t slot, mol;
    uint32_t ph, end;
};

// Batch: the next task from the CTAs' shared counter (false once every task is taken).
__device__ __forceinline__ bool f16_next_task(F16Cursor& k, const F16Args& a) {
    const int64_t q = atomicAdd(a.counter, 1);
    if (q >= a.n_units) return false;
    const F16Task t = a.tasks[q];
    k.u = q;
    k.mol = t.mol;
    k.row_tile = t.row_tile;
    k.kind = t.kind;
    k.s0 = 0;
    k.s1 = static_cast<int>(a.mols[t.mol].nk_pad / kF16Kj);  // tasks exist for kept points only
    k.s = 0;
    return true;
}
template <int NK>
__device__ __forceinline__ void f16_cursor_init(F16Cursor& k, const F16Args& a) {
    k.c = 0;
    k.mol = 0;
    if (a.mols) {
        k.done = !f16_next_task(k, a);
        return;
    }
    k.u = blockIdx.x;
    k.row_tile = static_cast<int32_t>(NK == 2 ? k.u : (k.u >> 1));
    k.kind = NK == 2 ? 0 : static_cast<int32_t>(k.u & 1);
    k.s0 = 0;
    k.s1 = min(a.n_stage, a.chunk);
    k.s = 0;
    k.done = (k.u >= a.n_units) || (a.n_stage <= 0);
}
template <int NK>
__device__ __forceinline__ void f16_cursor_next(F16Cursor& k, const F16Args& a) {
    if (++k.s < k.s1) return;
    if (a.mols) {
        k.done = !f16_next_task(k, a);
        return;
    }
    k.u += gridDim.x;
    if (k.u >= a.n_units) {
        k.u = blockIdx.x;
        ++k.c;
        k.s0 = k.c * a.chunk;
        if (k.s0 >= a.n_stage) {
            k.done = true;
            return;
        }
        k.s1 = min(a.n_stage, k.s0 + a.chunk);
    }
    k.row_tile = static_cast<int32_t>(NK == 2 ? k.u : (k.u >> 1));
    k.kind = NK == 2 ? 0 : static_cast<int32_t>(k.u & 1);
    k.s = k.s0;
}

template <int PQ, int NK>  // PQ accumulator columns per thread and kind (= Ppad / 4)
__global__ void __launch_bounds__(kF16Threads, 1)
k_hess_f16(const __grid_constant__ CUtensorMap tm_bh, const __grid_constant__ CUtensorMap tm_bl,
           F16Args args) {
    constexpr int PPAD = 4 * PQ;
    static_assert(NK == 1 || PPAD <= 64, "two kinds per tile need Ppad <= 64");
    static_assert(NK == 2 || 2 * PPAD + 128 <= static_cast<int>(kF16TmemCols), "TMEM columns");
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const F16Layout L = f16_layout(PPAD, NK);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* b_full = bars;                          // [kF16Ring]
    uint64_t* b_empty = bars + kF16Ring;              // [kF16Ring]
    uint64_t* a_full = bars + 2 * kF16Ring;           // [2]
    uint64_t* mma_done = bars + 2 * kF16Ring + 2;     // [2]
    uint64_t* xbar = bars + 2 * kF16Ring + 4;         // [2 slots][4 quads]
    uint64_t* fin = bars + 2 * kF16Ring + 12;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kF16Ring + 13);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * kF16Ring + 14);
    F16Meta* meta = reinterpret_cast<F16Meta*>(bars + 2 * kF16Ring + 16);  // [kF16Ring]
    float* xm = reinterpret_cast<float*>(smem + L.xm_off);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quad = warp & 3, part = warp >> 2;
    const bool is_producer = (warp == kF16ProducerWarp && lane == 0);
    const bool is_mma = (warp == kF16MmaWarp && lane == 0);

    if (threadIdx.x == 0) {
        for (int b = 0; b < kF16Ring; ++b) {
            mbar_init(&b_full[b], 1);
            mbar_init(&b_empty[b], kF16Warps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&a_full[b], kF16Warps);
            mbar_init(&mma_done[b], 1);
        }
        for (int b = 0; b < 8; ++b) mbar_init(&xbar[b], 4);  // one arrival per warp of a quad
        mbar_init(fin, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kF16MmaWarp) tc::tmem_alloc(tmem_slot, kF16TmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    // ---------------------------------------------------------------- producer (one thread)
    // keeps the ring kF16Ring - 1 stages ahead of the walk; every stage's copies complete on
    // its b_full barrier together with the producer's arrival, which releases the metadata.
    // Its state lives in shared memory (only one thread touches it), not in every thread's
    // registers.
    F16Prod* pr = reinterpret_cast<F16Prod*>(smem + L.prod_off);
    bool ok = true;
    auto produce = [&]() -> bool {
        F16Prod& P = *pr;
        if (P.end) return true;
        if (!f16_wait(&b_empty[P.slot], P.ph ^ 1u, args.err, abort_flag)) return false;
        if (P.k.done) {  // the end of the walk takes one slot, with no copies
            meta[P.slot] = F16Meta{0, 0, 0, F16_END};
            mbar_arrive(&b_full[P.slot]);
            P.end = 1;
            return true;
        }
        const F16Mol& M = args.mols ? args.mols[P.k.mol] : args.single;
        const CUtensorMap* mh = &tm_bh;
        const CUtensorMap* ml = &tm_bl;
        if (args.mols) {
            mh = M.maps;
            ml = M.maps + 1;
            if (P.k.mol != P.mol) {  // a new molecule's tensor maps
                P.mol = P.k.mol;
                tmap_acquire(mh);
                tmap_acquire(ml);
                tc::prefetch_tmap(mh);
                tc::prefetch_tmap(ml);
            }
        }
        const int s = P.k.s;
        meta[P.slot] = F16Meta{P.k.mol, P.k.row_tile, P.k.kind,
                               (s == P.k.s0 ? F16_FIRST : 0) | (s == P.k.s1 - 1 ? F16_LAST : 0)};
        uint8_t* base = smem + P.slot * L.slot_bytes;
        uint8_t* rec = smem + L.rec_off + P.slot * 1024;
        mbar_expect_tx(&b_full[P.slot], L.slot_bytes + 1024u);
        bulk_g2s(rec, M.r32p + 2 * kF16Kj * static_cast<int64_t>(s), 1024u, &b_full[P.slot]);
        // the chunk's trial tiles are re-read by every unit: keep them in L2 before other lines
        const uint64_t pol = tc::l2_evict_last();
        tc::tma_load_2d_hint(base, mh, 64 * s, M.t0, &b_full[P.slot], pol);
        tc::tma_load_2d_hint(base + L.tile_bytes, ml, 64 * s, M.t0, &b_full[P.slot], pol);
        ++P.issued;
        if (++P.slot == kF16Ring) {
            P.slot = 0;
            P.ph ^= 1u;
        }
        f16_cursor_next<NK>(P.k, args);
        return true;
    };
    if (is_producer) {
        F16Prod& P = *pr;
        P.slot = 0;
        P.ph = 0;
        P.end = 0;
        P.mol = -1;
        P.issued = 0;
        f16_cursor_init<NK>(P.k, args);
        if (!args.mols) {
            tc::prefetch_tmap(&tm_bh);
            tc::prefetch_tmap(&tm_bl);
        }
        for (int k = 0; k < kF16Ring - 1 && ok; ++k) ok = produce();
        if (!ok) *abort_flag = 1;
    }

    const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
    const uint32_t idesc = tc::idesc_f16(128, PPAD);
    float acc[NK][PQ];
#pragma unroll
    for (int k = 0; k < NK; ++k)
#pragma unroll
        for (int c = 0; c < PQ; ++c) acc[k][c] = 0.0f;

    // Drain a finished accumulator (every kind of the unit) into the FP32 registers, each
    // value times the inverse row factor of its stage.
    auto drain = [&](int db, uint32_t dphase, int kind0, const float (&iscp)[NK]) -> bool {
        const bool got = f16_wait(&mma_done[db], dphase, args.err, abort_flag);
        if (!__all_sync(0xffffffffu, got)) return false;  // warp-uniform exit
        tc::fence_after();
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const uint32_t col = tmem + lane_off + f16_dcol<NK, PPAD>(NK == 2 ? k : kind0, db) + part * PQ;
            constexpr int kChunk = PQ % 16 == 0 ? 16 : 8;
#pragma unroll
            for (int c0 = 0; c0 < PQ; c0 += kChunk) {
                uint32_t r[kChunk];
#pragma unroll
                for (int c = 0; c < kChunk; c += 8)
                    tc::ld_x8(col + c0 + c, *reinterpret_cast<uint32_t(*)[8]>(&r[c]));
                tc::wait_ld();
#pragma unroll
                for (int c = 0; c < kChunk; c += 2) {
                    const float2 v = __ffma2_rn(make_float2(__uint_as_float(r[c]), __uint_as_float(r[c + 1])),
                                                make_float2(iscp[k], iscp[k]),
                                                make_float2(acc[k][c0 + c], acc[k][c0 + c + 1]));
                    acc[k][c0 + c] = v.x;
                    acc[k][c0 + c + 1] = v.y;
                }
            }
        }
        tc::fence_before();
        return true;
    };
    // Add the registers into the molecule's FP64 partial output (times 1/s_t; the gamma
    // accumulator holds -(T3 u + T4 y)) and clear them.
    auto flush = [&](int mol, int kind0, int64_t i) {
        const F16Mol& M = args.mols ? args.mols[mol] : args.single;
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const int kind = NK == 2 ? k : kind0;
#pragma unroll
            for (int c = 0; c < PQ; ++c) {
                const int t = part * PQ + c;
                if (i < M.nk && t < M.Pn) {
                    const int64_t tg = static_cast<int64_t>(M.t0) + t;
                    double* o = M.acc + ((static_cast<int64_t>(kind) * M.acc_P + tg) * M.nk_pad + i);
                    const double v = static_cast<double>(acc[k][c]) * M.col_isc[tg];
                    // streaming loads and stores: the partial output must not evict the
                    // chunk's trial tiles from L2
                    __stcs(o, __ldcs(o) + ((kind == 0) ? v : -v));
                }
                acc[k][c] = 0.0f;
            }
        }
    };

    int slot = 0, ab = 0;
    uint32_t ph = 0, aph = 0;
    int pslot = 0, dbuf = 0;
    uint32_t dph = 0;
    uint32_t gs = 0;  // stages walked by this CTA (exchange slot and phase)
    bool mma_any = false;
    float isc_prev[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) isc_prev[k] = 1.0f;
    // the current unit: molecule, output kind, row, row data, 1/c_y
    int mol = 0, kind0 = 0, until_flush = args.flush;
    int64_t i = 0;
    float inv_cy = 1.f;
    RowF rc{0.f, 0.f, 0.f, 1.f, 1.f, 0.f, 0.f};
    ok = __all_sync(0xffffffffu, !*abort_flag);
    while (ok) {
        // the operand buffer ab is free once the MMAs of the stage two back are done
        bool got = f16_wait(&b_full[slot], ph, args.err, abort_flag);
        got = got && f16_wait(&mma_done[ab], aph ^ 1u, args.err, abort_flag);
        if (!__all_sync(0xffffffffu, got)) break;
        tc::fence_after();
        const F16Meta m = meta[slot];
        if (m.flags & F16_END) break;
        if (m.flags & F16_FIRST) {  // a new unit: its rows and molecule
            mol = m.mol;
            kind0 = NK == 2 ? 0 : m.kind;
            const F16Mol& M = args.mols ? args.mols[mol] : args.single;
            i = static_cast<int64_t>(m.row_tile) * 128 + quad * 32 + lane;
            float xi = 0.f, yi = 0.f, zi = 0.f, oi = 1.f, ki = 1.f, pi_ = 0.f, qi = 0.f;
            if (i < M.nk) {
                const float4 a4 = M.r32a[i];
                const float4 b4 = M.r32b[i];
                xi = a4.x; yi = a4.y; zi = a4.z; oi = b4.x; ki = b4.y; pi_ = b4.z; qi = b4.w;
            }
            rc = RowF{xi, yi, zi, oi, ki, -pi_, -qi};
            inv_cy = M.params[0];
            until_flush = args.flush;
        }
        // this warp's 8 j: pair-packed records 4 part .. 4 part + 3
        const float4* rec = reinterpret_cast<const float4*>(smem + L.rec_off + slot * 1024);
        float2 t[4][2 * NK];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float4* v = rec + 4 * (4 * part + h);
            f16_tiles2<NK>(kind0, rc, v[0], v[1], v[2], v[3], t[h]);
#pragma unroll
            for (int k = 0; k < NK; ++k)  // the tiles that multiply y carry 1/c_y
                t[h][2 * k + 1] = __fmul2_rn(t[h][2 * k + 1], make_float2(inv_cy, inv_cy));
        }
        // the row's largest |T| over the stage: this thread's 8 j, then the quad's 4 parts
        const int xs = static_cast<int>(gs & 1u);
        float* xrow = xm + (static_cast<size_t>((xs * 4 + quad) * NK) * 32 + lane) * 4;
#pragma unroll
        for (int k = 0; k < NK; ++k)
            xrow[k * 32 * 4 + part] = fmaxf(fmaxf(f16_absmax4(t[0][2 * k], t[1][2 * k]),
                                                  f16_absmax4(t[2][2 * k], t[3][2 * k])),
                                            fmaxf(f16_absmax4(t[0][2 * k + 1], t[1][2 * k + 1]),
                                                  f16_absmax4(t[2][2 * k + 1], t[3][2 * k + 1])));
        __syncwarp();  // the warp's 32 stores are ordered before lane 0's release
        if (lane == 0) mbar_arrive(&xbar[xs * 4 + quad]);
        got = f16_wait(&xbar[xs * 4 + quad], (gs >> 1) & 1u, args.err, abort_flag);
        if (!__all_sync(0xffffffffu, got)) break;
        float sc[NK], isc[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const float4 q = *reinterpret_cast<const float4*>(xrow + k * 32 * 4);
            f16_scale(fmaxf(fmaxf(q.x, q.y), fmaxf(q.z, q.w)), sc[k], isc[k]);
        }
        // scaled FP16 hi / lo operand tiles of kind k: [hi Ta | lo Ta | hi Tb | lo Tb], 16
        // columns each; this warp's 8 j are columns 4 part .. 4 part + 3
        const uint32_t a = tmem + lane_off + f16_acol<NK, PPAD>(ab) + 4 * part;
#pragma unroll
        for (int k = 0; k < NK; ++k) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) f16_split2(t[h][2 * k + b], sc[k], hw[h], lw[h]);
                tc::st_x4(a + 64u * k + 32u * b, hw);
                tc::st_x4(a + 64u * k + 32u * b + 16u, lw);
            }
        }
        tc::wait_st();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[ab]);  // this warp's operands are in place
        // ---- MMA issue (one thread): this stage, once every warp's operands are in place
        if (is_mma) {
            bool go = f16_wait(&a_full[ab], aph, args.err, abort_flag);
            if (go) {
                tc::fence_after();
                const uint32_t base = smem_u32(smem + slot * L.slot_bytes);
                const uint64_t bh = tc::sdesc_kmajor_sw128(base);
                const uint64_t bl = tc::sdesc_kmajor_sw128(base + L.tile_bytes);
                // trial rows: [u (16 j) | y (16 j)] for the stage's two halves, 32 B each; a
                // K-step moves the descriptor's address field by 32 B (2 units)
#pragma unroll
                for (int k = 0; k < NK; ++k) {
                    const uint32_t d = tmem + f16_dcol<NK, PPAD>(NK == 2 ? k : kind0, ab);
                    const uint32_t aa = tmem + f16_acol<NK, PPAD>(ab) + 64u * k;
                    // operand tiles: Ta hi | Ta lo | Tb hi | Tb lo, 16 columns each (8 per
                    // 16-j half).  The small products first (the accumulator truncates its
                    // adds), the four hi*hi last.
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const uint64_t ku = 4u * hh, ky = 4u * hh + 2u;
                        tc::mma_f16_ts(d, aa + 0 + 8 * hh, bl + ku, idesc, hh);   // Ta_hi u_lo
                        tc::mma_f16_ts(d, aa + 16 + 8 * hh, bh + ku, idesc, 1u);  // Ta_lo u_hi
                        tc::mma_f16_ts(d, aa + 32 + 8 * hh, bl + ky, idesc, 1u);  // Tb_hi y_lo
                        tc::mma_f16_ts(d, aa + 48 + 8 * hh, bh + ky, idesc, 1u);  // Tb_lo y_hi
                    }
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const uint64_t ku = 4u * hh, ky = 4u * hh + 2u;
                        tc::mma_f16_ts(d, aa + 0 + 8 * hh, bh + ku, idesc, 1u);   // Ta_hi u_hi
                        tc::mma_f16_ts(d, aa + 32 + 8 * hh, bh + ky, idesc, 1u);  // Tb_hi y_hi
                    }
                }
                tc::commit(&mma_done[ab]);  // the ring slot is released after the drains
                mma_any = true;
            }
        }
        if (!__all_sync(0xffffffffu, !*abort_flag)) break;
        // ---- drain the previous stage of this unit while this stage's MMAs run; then one
        // more copy (one per drained stage: the slot it fills was drained a stage earlier)
        if (!(m.flags & F16_FIRST)) {
            if (!drain(dbuf, dph, kind0, isc_prev)) break;
            if (lane == 0) mbar_arrive(&b_empty[pslot]);
            if (--until_flush == 0) {
                flush(mol, kind0, i);
                until_flush = args.flush;
            }
            if (is_producer && !produce()) *abort_flag = 1;
            if (!__all_sync(0xffffffffu, !*abort_flag)) break;
        }
#pragma unroll
        for (int k = 0; k < NK; ++k) isc_prev[k] = isc[k];
        dbuf = ab;
        dph = aph;
        pslot = slot;
        if (++slot == kF16Ring) {
            slot = 0;
            ph ^= 1u;
        }
        ab ^= 1;
        if (ab == 0) aph ^= 1u;
        ++gs;
        if (m.flags & F16_LAST) {  // the unit's last stage: drain it and write the rows out
            if (!drain(dbuf, dph, kind0, isc_prev)) break;
            if (lane == 0) mbar_arrive(&b_empty[pslot]);
            if (is_producer && !produce()) *abort_flag = 1;
            flush(mol, kind0, i);
            if (!__all_sync(0xffffffffu, !*abort_flag)) break;
        }
    }
    tc::wait_st();  // nothing of ours is in flight to TMEM on any exit path
    tc::wait_ld();
    if (is_producer) {  // copies in flight must land before the CTA exits
        // (after the end marker, its slot's previous stage was drained before it was written,
        // and that slot's parity has moved on: wait for the other ring slots only)
        const int64_t issued = pr->issued;
        const int64_t back = pr->end ? kF16Ring - 1 : kF16Ring;
        for (int64_t k = (issued > back ? issued - back : 0); k < issued; ++k)
            mbar_wait(&b_full[k % kF16Ring], static_cast<uint32_t>((k / kF16Ring) & 1), args.err);
    }
    if (is_mma && mma_any) {  // every MMA finished before TMEM is released
        tc::commit(fin);
        mbar_wait(fin, 0, args.err);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == kF16MmaWarp) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kF16TmemCols);
    }
}

// ---------------------------------------------------------------- trial split

// Per trial column, the largest |u'| and |y'| (u' = -3/2 u, y' = 3/2 y, in FP32) as bit
// patterns (non-negative floats order like unsigned integers); colmax zeroed before.
__global__ void __launch_bounds__(256)
k_f16_colmax(const double* __restrict__ u, const double* __restrict__ y, int64_t nk_pad,
             unsigned int* __restrict__ colmax, int32_t P) {
    const int t = blockIdx.y;
    const double* ut = u + static_cast<int64_t>(t) * nk_pad;
    const double* yt = y + static_cast<int64_t>(t) * nk_pad;
    float mu = 0.f, my = 0.f;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < nk_pad;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        mu = fmaxf(mu, fabsf(static_cast<float>(-1.5 * ut[j])));
        my = fmaxf(my, fabsf(static_cast<float>(1.5 * yt[j])));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&colmax[t], __float_as_uint(mu));
        atomicMax(&colmax[P + t], __float_as_uint(my));
    }
}

// c_y (a power of two near max|u'| / max|y'| over all trials, clamped to 2^[-24, 24]) and the
// column factors s_t (the column's max(|u'|, c_y |y'|) mapped into [2^14, 2^15)).
// params[0] = 1/c_y, params[1] = c_y; scale[t] = s_t; col_isc[t] = 1/s_t.
__device__ __forceinline__ void f16_scales_block(const unsigned int* __restrict__ colmax, int32_t P,
                                                 float* __restrict__ params,
                                                 float* __restrict__ scale,
                                                 double* __restrict__ col_isc) {
    __shared__ float su[8], sy[8];
    __shared__ float s_cy;
    float mu = 0.f, my = 0.f;
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        mu = fmaxf(mu, __uint_as_float(colmax[t]));
        my = fmaxf(my, __uint_as_float(colmax[P + t]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    if ((threadIdx.x & 31) == 0) {
        su[threadIdx.x >> 5] = mu;
        sy[threadIdx.x >> 5] = my;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (blockDim.x >> 5); ++w) {
            mu = fmaxf(mu, su[w]);
            my = fmaxf(my, sy[w]);
        }
        int e = 0;
        if (mu > 0.f && my > 0.f && isfinite(mu) && isfinite(my)) {
            e = static_cast<int>((__float_as_uint(mu) >> 23) & 0xFFu) -
                static_cast<int>((__float_as_uint(my) >> 23) & 0xFFu);
            e = e > 24 ? 24 : (e < -24 ? -24 : e);
        }
        s_cy = ldexpf(1.0f, e);
        params[0] = ldexpf(1.0f, -e);
        params[1] = s_cy;
    }
    __syncthreads();
    const float cy = s_cy;
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        float sc, isc;
        f16_scale(fmaxf(__uint_as_float(colmax[t]), cy * __uint_as_float(colmax[P + t])), sc, isc);
        scale[t] = sc;
        col_isc[t] = static_cast<double>(isc);
    }
}

__global__ void __launch_bounds__(256)
k_f16_scales(const unsigned int* __restrict__ colmax, int32_t P, float* __restrict__ params,
             float* __restrict__ scale, double* __restrict__ col_isc) {
    f16_scales_block(colmax, P, params, scale, col_isc);
}

// FP16 hi / lo trial tiles: row t, stage s holds 32 halves, u' s_t for the stage's 16 j
// then c_y y' s_t; rows t >= P are zero.
// Row t, point j of the FP16 hi / lo trial tiles from u, y (zero where t or j is padding).
__device__ __forceinline__ void f16_split_point(double u, double y, bool real, int t, int64_t j,
                                                int64_t nk_pad, const float* __restrict__ params,
                                                const float* __restrict__ scale,
                                                __half* __restrict__ bh, __half* __restrict__ bl) {
    float a = 0.f, b = 0.f;
    if (real) {
        const float st = scale[t];
        a = static_cast<float>(-1.5 * u) * st;            // exact power-of-two scalings
        b = static_cast<float>(1.5 * y) * (params[1] * st);
    }
    const __half ah = __float2half_rn(a), bhh = __float2half_rn(b);
    const __half al = __float2half_rn(a - __half2float(ah)), bll = __float2half_rn(b - __half2float(bhh));
    const int64_t off = static_cast<int64_t>(t) * (2 * nk_pad) + (j >> 4) * 32 + (j & 15);
    bh[off] = ah;
    bh[off + 16] = bhh;
    bl[off] = al;
    bl[off + 16] = bll;
}

__global__ void __launch_bounds__(256)
k_f16_split(const double* __restrict__ u, const double* __restrict__ y, int32_t P,
            int64_t nk_pad, const float* __restrict__ params, const float* __restrict__ scale,
            __half* __restrict__ bh, __half* __restrict__ bl) {
    const int t = blockIdx.y;
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= nk_pad) return;
    const int64_t o = static_cast<int64_t>(t) * nk_pad + j;
    f16_split_point(t < P ? u[o] : 0.0, t < P ? y[o] : 0.0, t < P, t, j, nk_pad, params, scale, bh, bl);
}

// ---- the batch: every molecule's trial values, column maxima, factors and FP16 tiles in three
// launches (the molecule table's f16 area: colmax [2 n_t] words (zeroed by the caller) |
// params at o_par | scale [n_t] floats at o_sc | col_isc [n_t] doubles at o_isc).
struct F16Small {
    unsigned int* colmax;
    float* params;
    float* scale;
    double* col_isc;
};
__device__ __forceinline__ F16Small f16_small(const EpiMol& M) {
    char* sm = static_cast<char*>(M.f16small);
    const size_t o_par = ((sizeof(unsigned int) * 2 * M.n_t + 255) / 256) * 256;
    const size_t o_sc = o_par + 256;
    const size_t o_isc = o_sc + ((sizeof(float) * M.n_t + 255) / 256) * 256;
    return F16Small{reinterpret_cast<unsigned int*>(sm), reinterpret_cast<float*>(sm + o_par),
                    reinterpret_cast<float*>(sm + o_sc), reinterpret_cast<double*>(sm + o_isc)};
}

// Block k of molecule m: trial t = k / nb, kept points 256 (k mod nb) .., nb = nk_pad / 256:
// rho^t and gamma^t at the kept points, and the trial's largest |u'|, |y'|.
__global__ void __launch_bounds__(256)
k_f16_trial_max_batch(const EpiMol* __restrict__ mols, const int64_t* __restrict__ pre, int n_mol,
                      const double* __restrict__ rho_t, const double* __restrict__ grad_rho_t) {
    int64_t blk;
    const EpiMol& M = mols[batch_block_mol(pre, n_mol, blockIdx.x, blk)];
    const int64_t nb = M.P.nk_pad / 256;
    const int t = static_cast<int>(blk / nb);
    const int64_t p = (blk - t * nb) * 256 + threadIdx.x;
    float mu = 0.f, my = 0.f;
    if (p < M.P.nk) {
        double u, y, rt, gt;
        trial_values(M.P, rho_t + M.toff, grad_rho_t + 3 * M.toff, t, p, u, y, rt, gt);
        M.rt[static_cast<int64_t>(t) * M.P.nk + p] = rt;
        M.gt[static_cast<int64_t>(t) * M.P.nk + p] = gt;
        mu = fabsf(static_cast<float>(-1.5 * u));
        my = fabsf(static_cast<float>(1.5 * y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    if ((threadIdx.x & 31) == 0) {
        const F16Small f = f16_small(M);
        atomicMax(&f.colmax[t], __float_as_uint(mu));
        atomicMax(&f.colmax[M.n_t + t], __float_as_uint(my));
    }
}

__global__ void __launch_bounds__(256) k_f16_scales_batch(const EpiMol* __restrict__ mols) {
    const EpiMol& M = mols[blockIdx.x];
    if (M.P.nk == 0 || M.n_t == 0) return;
    const F16Small f = f16_small(M);
    f16_scales_block(f.colmax, M.n_t, f.params, f.scale, f.col_isc);
}

// Block k of molecule m: row t = k / nb of its FP16 tiles (rows >= n_t zero), points
// 256 (k mod nb) ..; hi tiles at M.split, lo tiles M.split_step halves further.
__global__ void __launch_bounds__(256)
k_f16_split_batch(const EpiMol* __restrict__ mols, const int64_t* __restrict__ pre, int n_mol,
                  const double* __restrict__ rho_t, const double* __restrict__ grad_rho_t) {
    int64_t blk;
    const EpiMol& M = mols[batch_block_mol(pre, n_mol, blockIdx.x, blk)];
    const int64_t nb = M.P.nk_pad / 256;
    const int t = static_cast<int>(blk / nb);
    const int64_t p = (blk - t * nb) * 256 + threadIdx.x;
    const bool real = t < M.n_t && p < M.P.nk;
    double u = 0.0, y = 0.0;
    if (real) {
        double rt, gt;
        trial_values(M.P, rho_t + M.toff, grad_rho_t + 3 * M.toff, t, p, u, y, rt, gt);
    }
    const F16Small f = f16_small(M);
    __half* bh = reinterpret_cast<__half*>(M.split);
    f16_split_point(u, y, real, t, p, M.P.nk_pad, f.params, f.scale, bh, bh + M.split_step);
}

cudaError_t launch_f16_trial_batch(const EpiMol* mols, const int64_t* pre_max,
                                   const int64_t* pre_split, int n_mol, int64_t n_max_blocks,
                                   int64_t n_split_blocks, const double* rho_t,
                                   const double* grad_rho_t, cudaStream_t st) {
    if (n_max_blocks > 0)
        k_f16_trial_max_batch<<<static_cast<unsigned>(n_max_blocks), 256, 0, st>>>(mols, pre_max, n_mol,
                                                                                 rho_t, grad_rho_t);
    k_f16_scales_batch<<<n_mol, 256, 0, st>>>(mols);
    if (n_split_blocks > 0)
        k_f16_split_batch<<<static_cast<unsigned>(n_split_blocks), 256, 0, st>>>(mols, pre_split, n_mol,
                                                                               rho_t, grad_rho_t);
    return cudaGetLastError();
}

cudaError_t launch_f16_trial_split(const double* u, const double* y, int32_t P, int32_t rows,
                                   int64_t nk_pad, unsigned int* colmax, float* params,
                                   float* scale, double* col_isc, void* bh, void* bl,
                                   cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(colmax, 0, sizeof(unsigned int) * 2 * static_cast<size_t>(P), st);
    if (e != cudaSuccess) return e;
    const int64_t nb = (nk_pad + 255) / 256;
    dim3 g1(static_cast<unsigned>(nb < 16 ? nb : 16), static_cast<unsigned>(P));
    k_f16_colmax<<<g1, 256, 0, st>>>(u, y, nk_pad, colmax, P);
    k_f16_scales<<<1, 256, 0, st>>>(colmax, P, params, scale, col_isc);
    dim3 g2(static_cast<unsigned>(nb), static_cast<unsigned>(rows));
    k_f16_split<<<g2, 256, 0, st>>>(u, y, P, nk_pad, params, scale, static_cast<__half*>(bh),
                                    static_cast<__half*>(bl));
    return cudaGetLastError();
}

// ---------------------------------------------------------------- host side

static PFN_cuTensorMapEncodeTiled_v12000 f16_encode_fn() {
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

// 2-D map over a [rows][2 nk_pad] FP16 array, box = 64 halves (one stage: 16 u, 16 y, 16 u,
// 16 y) x ppad trials, 128-B swizzle.
static bool f16_make_map(CUtensorMap* m, const void* base, int64_t nk_pad, int64_t rows, int ppad) {
    auto fn = f16_encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(2 * nk_pad), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(2 * nk_pad) * sizeof(__half)};
    cuuint32_t box[2] = {64u, static_cast<cuuint32_t>(ppad)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int PQ, int NK>
static cudaError_t launch_f16_t(const CUtensorMap* maps, const F16Args& a, int n_sm, cudaStream_t st) {
    const F16Layout L = f16_layout(4 * PQ, NK);
    cudaError_t e = cudaFuncSetAttribute(k_hess_f16<PQ, NK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L.total));
    if (e != cudaSuccess) return e;
    const int grid = static_cast<int>(a.n_units < n_sm ? a.n_units : n_sm);
    if (grid <= 0) return cudaSuccess;
    k_hess_f16<PQ, NK><<<grid, kF16Threads, L.total, st>>>(maps[0], maps[1], a);
    return cudaGetLastError();
}

static cudaError_t launch_f16_dispatch(int ppad, const CUtensorMap* maps, const F16Args& a, int n_sm,
                                       cudaStream_t st) {
    switch (ppad / 4) {
        case 8: return launch_f16_t<8, 2>(maps, a, n_sm, st);
        case 16: return launch_f16_t<16, 2>(maps, a, n_sm, st);
        case 24: return launch_f16_t<24, 1>(maps, a, n_sm, st);
        case 32: return launch_f16_t<32, 1>(maps, a, n_sm, st);
        case 40: return launch_f16_t<40, 1>(maps, a, n_sm, st);
        case 48: return launch_f16_t<48, 1>(maps, a, n_sm, st);
        default: return cudaErrorInvalidValue;
    }
}

int hess_f16_kinds_per_tile(int ppad) { return ppad <= 64 ? 2 : 1; }
size_t hess_f16_default_chunk_bytes() { return kF16ChunkBytes; }

// Contract the trials [t0, t0 + Pn) (Pn <= 192) of one system; the split arrays have `rows`
// rows; col_isc and params as written by launch_f16_trial_split.
cudaError_t launch_hess_f16(const PointsDev& p, int32_t Pn, int32_t t0, int64_t acc_P,
                            const void* bh, const void* bl, int64_t rows, const double* col_isc,
                            const float* params, int n_sm, int flush, size_t chunk_bytes,
                            double* acc, int* err, cudaStream_t st) {
    if (p.nk == 0) return cudaSuccess;
    const int ppad = hess_tc_ppad(Pn);
    if (ppad > kF16MaxPpad || t0 + ppad > rows) return cudaErrorInvalidValue;
    CUtensorMap maps[2];
    if (!f16_make_map(&maps[0], bh, p.nk_pad, rows, ppad) || !f16_make_map(&maps[1], bl, p.nk_pad, rows, ppad))
        return cudaErrorInvalidValue;
    const int nk_t = hess_f16_kinds_per_tile(ppad);
    F16Args a;
    memset(&a, 0, sizeof(a));
    a.single = F16Mol{p.r32a, p.r32b, p.r32p, nullptr, acc, col_isc, params, p.nk, p.nk_pad, acc_P, Pn, t0};
    a.n_units = (nk_t == 2 ? 1 : 2) * ((p.nk + 127) / 128);
    a.n_stage = static_cast<int32_t>(p.nk_pad / kF16Kj);
    const size_t stage_bytes = 2u * static_cast<size_t>(ppad) * 128u + 1024u;
    int64_t chunk = static_cast<int64_t>((chunk_bytes > 0 ? chunk_bytes : kF16ChunkBytes) / stage_bytes);
    if (chunk < 64) chunk = 64;
    a.chunk = static_cast<int32_t>(chunk < a.n_stage ? chunk : a.n_stage);
    a.flush = flush > 0 ? flush : 512;
    a.err = err;
    return launch_f16_dispatch(ppad, maps, a, n_sm, st);
}

// ---------------------------------------------------------------- batched launches

size_t hess_f16_mol_bytes() { return sizeof(F16Mol); }
size_t hess_f16_task_bytes() { return sizeof(F16Task); }

// Tensor maps of one molecule (hi, lo: 2 consecutive CUtensorMap).
bool hess_f16_make_maps(void* out2, const void* bh, const void* bl, int64_t nk_pad, int64_t rows,
                        int ppad) {
    CUtensorMap* m = static_cast<CUtensorMap*>(out2);
    return f16_make_map(&m[0], bh, nk_pad, rows, ppad) && f16_make_map(&m[1], bl, nk_pad, rows, ppad);
}

void hess_f16_fill_mol(void* dst, const float4* r32a, const float4* r32b, const float4* r32p,
                       const void* maps_dev, double* acc, const double* col_isc,
                       const float* params, int64_t nk, int64_t nk_pad, int64_t acc_P, int32_t Pn,
                       int32_t t0) {
    const F16Mol m{r32a, r32b, r32p, static_cast<const CUtensorMap*>(maps_dev), acc, col_isc, params,
                   nk, nk_pad, acc_P, Pn, t0};
    memcpy(dst, &m, sizeof(m));
}

void hess_f16_fill_task(void* dst, int32_t mol, int32_t row_tile, int32_t kind) {
    const F16Task t{mol, row_tile, kind, 0};
    memcpy(dst, &t, sizeof(t));
}

// Batched contraction: every task of the table shares `ppad`; molecules, tasks and tensor
// maps live in device memory (written before the launch); counter: one int, zeroed here.
cudaError_t launch_hess_f16_batch(const void* mols, const void* tasks, int64_t n_tasks, int ppad,
                                  int* counter, int n_sm, int flush, int* err, cudaStream_t st) {
    if (n_tasks <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    CUtensorMap unused[2];
    memset(unused, 0, sizeof(unused));
    F16Args a;
    memset(&a, 0, sizeof(a));
    a.mols = static_cast<const F16Mol*>(mols);
    a.tasks = static_cast<const F16Task*>(tasks);
    a.counter = counter;
    a.n_units = n_tasks;
    a.flush = flush > 0 ? flush : 512;
    a.err = err;
    return launch_f16_dispatch(ppad, unused, a, n_sm, st);
}

}  // namespace vv10
