// K3 with FP64 accuracy on the tensor cores (VV10_FP64_TC): the pair part of Eq. frhot
// (Sec. II.B) as a product of kernel tiles with the trial matrix, both cut into seven 8-bit
// integer slices (an Ozaki-style split) whose products tcgen05 kind::f16 sums exactly.
//
// Tiles in double-FP32.  GB300 runs FP64 at 1/64 of the FP32 rate, so the kernel tiles are
// generated as unevaluated pairs of FP32 numbers (hi + lo, about 46 correct bits) with the
// error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2): TwoSum for additions,
// the FMA product error for multiplications, Newton's iteration for the reciprocal.  The
// coordinates are held as FP32 pairs too, and their differences are formed exactly (TwoSum
// of the high parts), so near pairs lose nothing to cancellation.
//
// Slices.  A value scaled by a power of two into |x| < 2^7 is written as
//   x = s0 + s1 2^-8 + s2 2^-16 + s3 2^-24 + s4 2^-32 + s5 2^-40 + s6 2^-48 + e,
// every s an integer of at most 8 bits (|s3|, |s6| <= 192), exactly representable in FP16.
// Kernel tiles take one factor per row and 16-j stage (the row's largest |T| in the stage into
// [2^6, 2^7)); trials one per column and 16-j stage (the largest of |u'| and c_y |y'| in the
// block, with one global y balance c_y), so that a small value far below its row's or
// column's maximum keeps its own precision.  The product of slices p and q carries the weight
// 2^-8(p+q); the 28 pairs with p + q <= 6 are formed, the rest are below 2^-56 of the stage's
// scale.  Each level l = p + q has its own TMEM accumulator, and a level's sum over one stage
// is a sum of at most 7 x 32 products of integers below 2^14.6: below 2^22.4, so FP32 holds it
// exactly, whatever order and truncation the tensor core uses.  The drain combines the seven
// levels of a stage into an unevaluated FP32 pair, multiplies it by the row and column
// factors' inverses (powers of two) and adds it into a double-FP32 register sum per output;
// the flush adds that sum in FP64 to the partial output.
//
// Work unit: 128 rows x one output kind x the trials of the launch (MMA N = Ppad = 32; TMEM
// holds 7 x 32 accumulator and 7 x 16 operand columns).  The j range is walked in L2-sized
// chunks as in the split-FP16 kernel (each CTA its fixed units in every chunk).  16 warps (4
// per TMEM lane quadrant, 4 j each): generate the two tiles of the row, exchange the stage's
// row maxima, wait for the previous stage's MMAs and drain them, slice and store the operands
// into TMEM; lane 0 of warp 0 issues the 56 MMAs of a stage, lane 0 of warp 1 keeps the copy
// ring kO64Ring - 1 stages ahead.  Every wait is bounded (kSpinCycles).
#include <cstring>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.hpp"
#include "tc.cuh"

namespace vv10 {

constexpr int kO64Kj = 16;          // j per stage (one K = 16 MMA step per tile)
constexpr int kO64Warps = 16;
constexpr int kO64Threads = kO64Warps * 32;
constexpr int kO64Ring = 4;         // stages of copies in flight
constexpr int kO64Slices = 7;
constexpr int kO64Levels = 7;       // p + q = 0 .. 6
constexpr int kO64Ppad = 32;        // trials per launch (MMA N)
constexpr int kO64PQ = kO64Ppad / 4;
constexpr uint32_t kO64TmemCols = 512;
constexpr size_t kO64ChunkBytes = 48u << 20;
constexpr uint32_t kO64RecBytes = 64;  // one column record (FP32 pairs)

struct O64Layout {
    uint32_t tile_bytes;  // one Ppad x 32-half slice tile (64-byte rows: 16 u', 16 c_y y')
    uint32_t slot_bytes;  // the seven slice tiles of one stage
    uint32_t civ_off;     // the stage's column-factor inverses [Ppad] floats, per ring slot
    uint32_t rec_off;     // the stage's 16 column records, per ring slot
    uint32_t xm_off;      // row-maximum exchange [2][4 quads][32 lanes][4 parts] floats
    uint32_t prod_off;    // the producer thread's state
    uint32_t bar_off;
    uint32_t total;
};
__host__ __device__ constexpr O64Layout o64_layout() {
    O64Layout L{};
    L.tile_bytes = kO64Ppad * 64u;
    L.slot_bytes = kO64Slices * L.tile_bytes;
    L.civ_off = kO64Ring * L.slot_bytes;
    L.rec_off = L.civ_off + kO64Ring * kO64Ppad * 4u;
    L.xm_off = L.rec_off + kO64Ring * kO64Kj * kO64RecBytes;
    L.prod_off = L.xm_off + 2u * 4u * 32u * 4u * 4u;
    L.bar_off = L.prod_off + 128u;
    L.total = L.bar_off + 512u + 1024u;
    return L;
}

// Records of two consecutive points j0 = 2m, j1 = 2m + 1: every quantity v as an FP32 pair
// (hi = fl32(v), lo = fl32(v - hi)), stored as {hi0, hi1, lo0, lo1} so that the two points' his
// and los are ready-made operands of packed FP32x2 instructions: x, y, z, omega, kappa,
// p = rho kappa_rho, q = rho omega_rho (and one unused float4).
struct __align__(16) O64Rec {
    float4 v[8];
};
static_assert(sizeof(O64Rec) == 2 * kO64RecBytes, "record size");
enum : int { R_X = 0, R_Y, R_Z, R_OM, R_KA, R_P, R_Q };

struct O64Args {
    const O64Rec* rec;       // [nk_pad / 2] pair records of the kept points
    double* acc;             // [2][acc_P][nk_pad] FP64 partial output, zero on entry
    const float* civ;        // [n_stage][Ppad] column-factor inverses of this launch's group
    const double* params;    // [0] = 1/c_y
    int64_t nk, nk_pad, acc_P;
    int32_t Pn, t0;
    int64_t n_units;         // row tiles x 2 output kinds
    int32_t n_stage, chunk;
    int32_t flush;
    int* err;
};

struct O64Cursor {
    int c, s, s0, s1;
    int64_t u;
    bool done;
};
struct O64Prod {
    O64Cursor k;
    int64_t issued;
    int32_t slot;
    uint32_t ph, end;
};
enum : int32_t { O64_FIRST = 1, O64_LAST = 2, O64_END = 4 };
struct O64Meta {
    int32_t row_tile, kind, flags, pad;
};

__device__ __forceinline__ void o64_cursor_init(O64Cursor& k, const O64Args& a) {
    k.c = 0;
    k.u = blockIdx.x;
    k.s0 = 0;
    k.s1 = min(a.n_stage, a.chunk);
    k.s = 0;
    k.done = (k.u >= a.n_units) || (a.n_stage <= 0);
}
__device__ __forceinline__ void o64_cursor_next(O64Cursor& k, const O64Args& a) {
    if (++k.s < k.s1) return;
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
    k.s = k.s0;
}

__device__ __forceinline__ bool o64_wait(uint64_t* bar, uint32_t parity, int* err,
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

// ---------------------------------------------------------------- double-FP32 arithmetic

struct DF {
    float h, l;
};
// Knuth's TwoSum: a + b = s + e exactly.
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = a + b;
    const float bp = s - a;
    return DF{s, (a - (s - bp)) + (b - bp)};
}
// Dekker's FastTwoSum (|a| >= |b| or a = 0): a + b = s + e exactly.
__device__ __forceinline__ DF df_fast(float a, float b) {
    const float s = a + b;
    return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
    DF s = df_two_sum(x.h, y.h);
    return df_fast(s.h, s.l + (x.l + y.l));
}
__device__ __forceinline__ DF df_sub(DF x, DF y) { return df_add(x, DF{-y.h, -y.l}); }
__device__ __forceinline__ DF df_mul(DF x, DF y) {
    const float p = x.h * y.h;
    float e = fmaf(x.h, y.h, -p);  // the product's rounding error, exactly
    e = fmaf(x.h, y.l, e);
    e = fmaf(x.l, y.h, e);
    return df_fast(p, e);
}
__device__ __forceinline__ DF df_sqr(DF x) {
    const float p = x.h * x.h;
    float e = fmaf(x.h, x.h, -p);
    e = fmaf(x.h + x.h, x.l, e);
    return df_fast(p, e);
}
// 1/x: an FP32 reciprocal refined by one Newton step, then one Newton step in double-FP32.
__device__ __forceinline__ DF df_rcp(DF x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.h));
    r = fmaf(r, fmaf(-x.h, r, 1.0f), r);
    const float p = x.h * r;
    const float pe = fmaf(x.h, r, -p);  // x.h r = p + pe
    float res = (1.0f - p) - pe;        // 1 - p is exact (p is within 2^-22 of 1)
    res = fmaf(-x.l, r, res);
    return df_fast(r, r * res);
}
__device__ __forceinline__ DF df_neg(DF x) { return DF{-x.h, -x.l}; }
__device__ __forceinline__ DF df_scale(DF x, float f) { return DF{x.h * f, x.l * f}; }  // f = 2^k

// The same operations on two independent values at once (packed FP32x2 instructions: one
// issue slot for two lanes, each lane rounded to nearest as the scalar forms).
struct DF2 {
    float2 h, l;
};
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ DF2 df2_two_sum(float2 a, float2 b) {
    const float2 s = add2(a, b);
    const float2 bp = sub2(s, a);
    return DF2{s, add2(sub2(a, sub2(s, bp)), sub2(b, bp))};
}
__device__ __forceinline__ DF2 df2_fast(float2 a, float2 b) {
    const float2 s = add2(a, b);
    return DF2{s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ DF2 df2_add(DF2 x, DF2 y) {
    const DF2 s = df2_two_sum(x.h, y.h);
    return df2_fast(s.h, add2(s.l, add2(x.l, y.l)));
}
__device__ __forceinline__ DF2 df2_mul(DF2 x, DF2 y) {
    const float2 p = mul2(x.h, y.h);
    float2 e = fma2(x.h, y.h, mul2(p, f2(-1.0f)));  // the product's rounding error, exactly
    e = fma2(x.h, y.l, e);
    e = fma2(x.l, y.h, e);
    return df2_fast(p, e);
}
__device__ __forceinline__ DF2 df2_sqr(DF2 x) {
    const float2 p = mul2(x.h, x.h);
    float2 e = fma2(x.h, x.h, mul2(p, f2(-1.0f)));
    e = fma2(add2(x.h, x.h), x.l, e);
    return df2_fast(p, e);
}
__device__ __forceinline__ DF2 df2_rcp(DF2 x) {
    float2 r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(x.h.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(x.h.y));
    const float2 nxh = mul2(x.h, f2(-1.0f));
    r = fma2(r, fma2(nxh, r, f2(1.0f)), r);
    const float2 p = mul2(x.h, r);
    const float2 pe = fma2(x.h, r, mul2(p, f2(-1.0f)));  // x.h r = p + pe
    float2 res = sub2(sub2(f2(1.0f), p), pe);            // 1 - p is exact
    res = fma2(mul2(x.l, f2(-1.0f)), r, res);
    return df2_fast(r, mul2(r, res));
}
__device__ __forceinline__ DF2 df2_neg(DF2 x) { return DF2{mul2(x.h, f2(-1.0f)), mul2(x.l, f2(-1.0f))}; }
__device__ __forceinline__ DF2 df2_dup(DF x) { return DF2{f2(x.h), f2(x.l)}; }
__device__ __forceinline__ DF2 df2_rec(const float4& v) {
    return DF2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}

// Exact difference of two coordinates held as FP32 pairs, rounded to a pair.
__device__ __forceinline__ DF df_diff(float ah, float al, float bh, float bl) {
    const DF s = df_two_sum(ah, -bh);
    return df_fast(s.h, s.l + (al - bl));
}

// Row data: x, y, z, omega, kappa and -p, -q of row i.
struct RowDF {
    float xh, xl, yh, yl, zh, zl;
    DF om, ka, np, nq;
};

// The two kernel tiles of output `kind` for row r against the two columns of pair record c
// (lane 0: j0, lane 1: j1; the quantities and signs of the FP32 generator of the split
// kernels): kind 0 -> (T1c, T2c), kind 1 -> (T3c, T4c).
__device__ __forceinline__ void o64_tiles2(int kind, const RowDF& r, const O64Rec& c, DF2& ta, DF2& tb) {
    // exact coordinate differences (TwoSum of the high parts), rounded to pairs
    auto diff = [&](float ah, float al, const float4& b) {
        const DF2 t = df2_two_sum(f2(ah), mul2(make_float2(b.x, b.y), f2(-1.0f)));
        return df2_fast(t.h, add2(t.l, sub2(f2(al), make_float2(b.z, b.w))));
    };
    const DF2 dx = diff(r.xh, r.xl, c.v[R_X]);
    const DF2 dy = diff(r.yh, r.yl, c.v[R_Y]);
    const DF2 dz = diff(r.zh, r.zl, c.v[R_Z]);
    const DF2 r2 = df2_add(df2_add(df2_sqr(dx), df2_sqr(dy)), df2_sqr(dz));
    const DF2 g = df2_add(df2_mul(df2_dup(r.om), r2), df2_dup(r.ka));
    const DF2 gp = df2_add(df2_mul(df2_rec(c.v[R_OM]), r2), df2_rec(c.v[R_KA]));
    const DF2 s = df2_add(g, gp);
    const DF2 ggp = df2_mul(g, gp);
    const DF2 inv = df2_rcp(df2_mul(ggp, s));
    const DF2 L = df2_mul(ggp, inv);
    const DF2 sinv = df2_mul(s, inv);  // 1/(g g')
    DF2 M = df2_add(df2_sqr(L), sinv);
    M = DF2{add2(M.h, M.h), add2(M.l, M.l)};
    const DF2 nAi = df2_add(df2_mul(df2_dup(r.nq), r2), df2_dup(r.np));
    const DF2 nAj = df2_neg(df2_add(df2_mul(df2_rec(c.v[R_Q]), r2), df2_rec(c.v[R_P])));
    const DF2 rp = df2_mul(r2, inv);
    if (kind == 0) {
        const DF2 LGi = df2_add(L, df2_mul(gp, sinv)), LGj = df2_add(L, df2_mul(g, sinv));
        DF2 br = df2_add(DF2{f2(1.0f), f2(0.0f)}, df2_mul(nAi, LGi));
        br = df2_add(br, df2_mul(nAj, LGj));
        br = df2_add(br, df2_mul(df2_mul(nAi, nAj), M));
        ta = df2_mul(inv, br);                                   // T1c
        tb = df2_mul(rp, df2_add(df2_mul(nAi, M), LGj));         // T2c
    } else {
        const DF2 LGi = df2_add(L, df2_mul(gp, sinv));
        ta = df2_mul(rp, df2_add(df2_mul(nAj, M), LGi));         // T3c
        tb = df2_mul(df2_mul(rp, r2), M);                        // T4c
    }
}

// Power of two that maps a maximum m >= 0 into [2^6, 2^7), and its inverse, both normal FP32
// numbers (the factor's exponent is clamped to [-120, 120]; a zero maximum takes 2^120).
__device__ __forceinline__ void o64_scale_f(float m, float& sc, float& isc) {
    const int eb = static_cast<int>((__float_as_uint(m) >> 23) & 0xFFu);
    int se = 6 - (eb - 127);
    se = se > 120 ? 120 : (se < -120 ? -120 : se);
    sc = __int_as_float((127 + se) << 23);
    isc = __int_as_float((127 - se) << 23);
}

// The seven integer slices of x = hi + lo (|x| < 2^7, |lo| <= ulp(hi) / 2), weights 2^0, 2^-8,
// ..., 2^-48, in FP32 arithmetic: three from hi, whose remainder (weight 2^-16) joins lo
// through an error-free sum w + e; three from w; the last from what is left and e.
__device__ __forceinline__ void o64_slices(float hi, float lo, float (&s)[kO64Slices]) {
    s[0] = rintf(hi);
    const float r0 = (hi - s[0]) * 256.0f;              // exact
    s[1] = rintf(r0);
    const float r1 = (r0 - s[1]) * 256.0f;              // exact
    s[2] = rintf(r1);
    const DF w = df_two_sum((r1 - s[2]) * 0.0000152587890625f, lo);
    const float u3 = w.h * 16777216.0f;                 // 2^24: |u3| <= 192
    s[3] = rintf(u3);
    const float u4 = (u3 - s[3]) * 256.0f;              // exact
    s[4] = rintf(u4);
    const float u5 = (u4 - s[4]) * 256.0f;              // exact
    s[5] = rintf(u5);
    s[6] = rintf(fmaf(w.l, 281474976710656.0f, (u5 - s[5]) * 256.0f));  // w.l 2^48
}

// TMEM columns: level l accumulator at 32 l (l = 0..6); operand slices at 224: slice p, tile
// b (0: Ta, 1: Tb) at 224 + 16 p + 8 b, 8 columns (16 j, two FP16 each).
__device__ __forceinline__ uint32_t o64_dcol(int l) { return static_cast<uint32_t>(kO64Ppad * l); }
__device__ __forceinline__ uint32_t o64_acol(int p, int b) {
    return static_cast<uint32_t>(kO64Levels * kO64Ppad + 16 * p + 8 * b);
}
static_assert(kO64Levels * kO64Ppad + 16 * kO64Slices <= static_cast<int>(kO64TmemCols), "TMEM");

__global__ void __launch_bounds__(kO64Threads, 1)
k_hess_o64(const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1,
           const __grid_constant__ CUtensorMap tm2, const __grid_constant__ CUtensorMap tm3,
           const __grid_constant__ CUtensorMap tm4, const __grid_constant__ CUtensorMap tm5,
           const __grid_constant__ CUtensorMap tm6, O64Args args) {
    constexpr int PQ = kO64PQ;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    constexpr O64Layout L = o64_layout();
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* b_full = bars;                    // [kO64Ring]
    uint64_t* b_empty = bars + kO64Ring;        // [kO64Ring]
    uint64_t* a_full = bars + 2 * kO64Ring;     // operands in TMEM
    uint64_t* mma_done = bars + 2 * kO64Ring + 1;
    uint64_t* xbar = bars + 2 * kO64Ring + 2;   // [2 slots][4 quads]
    uint64_t* fin = bars + 2 * kO64Ring + 10;   // every MMA of the CTA done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kO64Ring + 11);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * kO64Ring + 12);
    O64Meta* meta = reinterpret_cast<O64Meta*>(bars + 2 * kO64Ring + 13);  // [kO64Ring]
    float* xm = reinterpret_cast<float*>(smem + L.xm_off);
    const CUtensorMap* maps[kO64Slices] = {&tm0, &tm1, &tm2, &tm3, &tm4, &tm5, &tm6};

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quad = warp & 3, part = warp >> 2;
    const bool is_producer = (warp == 1 && lane == 0);
    const bool is_mma = (warp == 0 && lane == 0);

    if (threadIdx.x == 0) {
        for (int b = 0; b < kO64Ring; ++b) {
            mbar_init(&b_full[b], 1);
            mbar_init(&b_empty[b], kO64Warps);
        }
        mbar_init(a_full, kO64Warps);
        mbar_init(mma_done, 1);
        mbar_init(fin, 1);
        for (int b = 0; b < 8; ++b) mbar_init(&xbar[b], 4);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, kO64TmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    // ---------------------------------------------------------------- producer (one thread)
    O64Prod* pr = reinterpret_cast<O64Prod*>(smem + L.prod_off);
    bool ok = true;
    auto produce = [&]() -> bool {
        O64Prod& P = *pr;
        if (P.end) return true;
        if (!o64_wait(&b_empty[P.slot], P.ph ^ 1u, args.err, abort_flag)) return false;
        if (P.k.done) {
            meta[P.slot] = O64Meta{0, 0, O64_END, 0};
            mbar_arrive(&b_full[P.slot]);
            P.end = 1;
            return true;
        }
        const int s = P.k.s;
        meta[P.slot] = O64Meta{static_cast<int32_t>(P.k.u >> 1), static_cast<int32_t>(P.k.u & 1),
                               (s == P.k.s0 ? O64_FIRST : 0) | (s == P.k.s1 - 1 ? O64_LAST : 0), 0};
        constexpr uint32_t rec_bytes = kO64Kj * kO64RecBytes, civ_bytes = kO64Ppad * 4u;
        mbar_expect_tx(&b_full[P.slot], L.slot_bytes + rec_bytes + civ_bytes);
        bulk_g2s(smem + L.rec_off + P.slot * rec_bytes, args.rec + static_cast<int64_t>(kO64Kj / 2) * s,
                 rec_bytes, &b_full[P.slot]);  // the stage's kO64Kj / 2 pair records
        bulk_g2s(smem + L.civ_off + P.slot * civ_bytes, args.civ + static_cast<int64_t>(kO64Ppad) * s,
                 civ_bytes, &b_full[P.slot]);
        uint8_t* base = smem + P.slot * L.slot_bytes;
        for (int q = 0; q < kO64Slices; ++q)
            tc::tma_load_2d(base + q * L.tile_bytes, maps[q], 32 * s, args.t0, &b_full[P.slot]);
        ++P.issued;
        if (++P.slot == kO64Ring) {
            P.slot = 0;
            P.ph ^= 1u;
        }
        o64_cursor_next(P.k, args);
        return true;
    };
    if (is_producer) {
        O64Prod& P = *pr;
        P.slot = 0;
        P.ph = 0;
        P.end = 0;
        P.issued = 0;
        o64_cursor_init(P.k, args);
        for (int q = 0; q < kO64Slices; ++q) tc::prefetch_tmap(maps[q]);
        for (int k = 0; k < kO64Ring - 1 && ok; ++k) ok = produce();
        if (!ok) *abort_flag = 1;
    }

    const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
    const uint32_t idesc = tc::idesc_f16(128, kO64Ppad);
    const float inv_cy = static_cast<float>(args.params[0]);  // a power of two
    float ahi[PQ], alo[PQ];  // double-FP32 sums of this thread's columns
#pragma unroll
    for (int c = 0; c < PQ; ++c) ahi[c] = alo[c] = 0.0f;

    // Drain the previous stage: the seven levels of each column combined, times the row and
    // column factors' inverses, added into (ahi, alo).
    auto drain = [&](uint32_t dphase, float riv, const float* civ) -> bool {
        const bool got = o64_wait(mma_done, dphase, args.err, abort_flag);
        if (!__all_sync(0xffffffffu, got)) return false;
        tc::fence_after();
#pragma unroll
        for (int c0 = 0; c0 < PQ; c0 += 4) {
            uint32_t r[kO64Levels][4];
#pragma unroll
            for (int l = 0; l < kO64Levels; ++l)
                tc::ld_x4(tmem + lane_off + o64_dcol(l) + part * PQ + c0, r[l]);
            tc::wait_ld();
            const float4 cv = *reinterpret_cast<const float4*>(civ + part * PQ + c0);
            const float cf[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                // v = L0 + L1 2^-8 + ... + L6 2^-48 (each L an exact integer below 2^22.4),
                // as an unevaluated FP32 pair; the first three sums error-free
                DF v = df_two_sum(__uint_as_float(r[0][c]), __uint_as_float(r[1][c]) * 0.00390625f);
                const DF w = df_two_sum(v.h, __uint_as_float(r[2][c]) * 0.0000152587890625f);
                v.h = w.h;
                v.l += w.l + (__uint_as_float(r[3][c]) * 5.9604644775390625e-8f +
                              (__uint_as_float(r[4][c]) * 2.3283064365386963e-10f +
                               (__uint_as_float(r[5][c]) * 9.094947017729282e-13f +
                                __uint_as_float(r[6][c]) * 3.552713678800501e-15f)));
                const float f = riv * cf[c];  // a power of two
                const DF a = df_add(DF{ahi[c0 + c], alo[c0 + c]}, DF{v.h * f, v.l * f});
                ahi[c0 + c] = a.h;
                alo[c0 + c] = a.l;
            }
        }
        tc::fence_before();
        return true;
    };
    auto flush = [&](int kind, int64_t i) {
#pragma unroll
        for (int c = 0; c < PQ; ++c) {
            const int t = part * PQ + c;
            if (i < args.nk && t < args.Pn) {
                const int64_t tg = static_cast<int64_t>(args.t0) + t;
                double* o = args.acc + ((static_cast<int64_t>(kind) * args.acc_P + tg) * args.nk_pad + i);
                const double v = static_cast<double>(ahi[c]) + static_cast<double>(alo[c]);
                __stcs(o, __ldcs(o) + ((kind == 0) ? v : -v));  // streaming: keep the tiles in L2
            }
            ahi[c] = alo[c] = 0.0f;
        }
    };

    int slot = 0;
    uint32_t ph = 0, mph = 0;  // ring phase; phase of the (single) operand / MMA barrier pair
    uint32_t gs = 0;
    bool pending = false;      // a stage's MMAs not drained yet
    bool mma_any = false;      // this thread issued MMAs
    float riv_prev = 1.0f;     // the pending stage's inverse row factor
    int pslot = 0;             // and its ring slot
    int kind0 = 0, until_flush = args.flush;
    int64_t i = 0;
    RowDF rc{};
    ok = __all_sync(0xffffffffu, !*abort_flag);
    while (ok) {
        bool got = o64_wait(&b_full[slot], ph, args.err, abort_flag);
        if (!__all_sync(0xffffffffu, got)) break;
        const O64Meta m = meta[slot];
        if (m.flags & O64_END) break;
        if (m.flags & O64_FIRST) {
            kind0 = m.kind;
            i = static_cast<int64_t>(m.row_tile) * 128 + quad * 32 + lane;
            const int64_t ir = i < args.nk ? i : args.nk_pad - 1;  // a padding record
            const O64Rec& R = args.rec[ir >> 1];
            const bool odd = (ir & 1) != 0;
            auto hl = [&](int q) {
                const float4 v = R.v[q];
                return DF{odd ? v.y : v.x, odd ? v.w : v.z};
            };
            const DF x = hl(R_X), y = hl(R_Y), z = hl(R_Z);
            rc.xh = x.h; rc.xl = x.l; rc.yh = y.h; rc.yl = y.l; rc.zh = z.h; rc.zl = z.l;
            rc.om = hl(R_OM);
            rc.ka = hl(R_KA);
            const DF p = hl(R_P), q = hl(R_Q);
            rc.np = DF{-p.h, -p.l};
            rc.nq = DF{-q.h, -q.l};
            until_flush = args.flush;
        }
        // tiles of this warp's 4 j (pair records 2 part, 2 part + 1), two j per packed lane pair
        const O64Rec* rs = reinterpret_cast<const O64Rec*>(smem + L.rec_off + slot * kO64Kj * kO64RecBytes);
        DF ta[4], tb[4];
        float mx = 0.0f;
#pragma unroll
        for (int hp = 0; hp < 2; ++hp) {
            DF2 a2, b2;
            o64_tiles2(kind0, rc, rs[2 * part + hp], a2, b2);
            b2 = DF2{mul2(b2.h, f2(inv_cy)), mul2(b2.l, f2(inv_cy))};  // the tile that multiplies y carries 1/c_y
            ta[2 * hp] = DF{a2.h.x, a2.l.x};
            ta[2 * hp + 1] = DF{a2.h.y, a2.l.y};
            tb[2 * hp] = DF{b2.h.x, b2.l.x};
            tb[2 * hp + 1] = DF{b2.h.y, b2.l.y};
        }
#pragma unroll
        for (int h = 0; h < 4; ++h) mx = fmaxf(mx, fmaxf(fabsf(ta[h].h), fabsf(tb[h].h)));
        // the row's largest |T| over the stage: the quad's 4 parts
        const int xs = static_cast<int>(gs & 1u);
        float* xrow = xm + (static_cast<size_t>(xs * 4 + quad) * 32 + lane) * 4;
        xrow[part] = mx;
        __syncwarp();
        if (lane == 0) mbar_arrive(&xbar[xs * 4 + quad]);
        got = o64_wait(&xbar[xs * 4 + quad], (gs >> 1) & 1u, args.err, abort_flag);
        if (!__all_sync(0xffffffffu, got)) break;
        float sc, riv;
        {
            const float4 q = *reinterpret_cast<const float4*>(xrow);
            o64_scale_f(fmaxf(fmaxf(q.x, q.y), fmaxf(q.z, q.w)), sc, riv);
        }
        // the previous stage's MMAs must be done (single operand and accumulator buffers):
        // drain them before the operands are overwritten
        if (pending) {
            if (!drain(mph ^ 1u, riv_prev,
                       reinterpret_cast<const float*>(smem + L.civ_off + pslot * kO64Ppad * 4)))
                break;
            if (lane == 0) mbar_arrive(&b_empty[pslot]);
            if (--until_flush == 0) {
                flush(kind0, i);
                until_flush = args.flush;
            }
            if (is_producer && !pr->end && !produce()) *abort_flag = 1;
            pending = false;
        }
        // slices of the scaled tiles: this warp's 4 j are columns 2 part, 2 part + 1 of each
        // 8-column operand
        const uint32_t a = tmem + lane_off + 2 * part;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const DF* t = b == 0 ? ta : tb;
            float s0[kO64Slices], s1[kO64Slices], s2[kO64Slices], s3[kO64Slices];
            o64_slices(t[0].h * sc, t[0].l * sc, s0);
            o64_slices(t[1].h * sc, t[1].l * sc, s1);
            o64_slices(t[2].h * sc, t[2].l * sc, s2);
            o64_slices(t[3].h * sc, t[3].l * sc, s3);
#pragma unroll
            for (int p = 0; p < kO64Slices; ++p) {
                const __half2 x = __floats2half2_rn(s0[p], s1[p]);
                const __half2 y = __floats2half2_rn(s2[p], s3[p]);
                tc::st_x2(a + o64_acol(p, b), *reinterpret_cast<const uint32_t*>(&x),
                          *reinterpret_cast<const uint32_t*>(&y));
            }
        }
        tc::wait_st();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(a_full);
        if (is_mma) {
            if (o64_wait(a_full, mph, args.err, abort_flag)) {
                tc::fence_after();
                const uint32_t base = smem_u32(smem + slot * L.slot_bytes);
                // level l = p + q: slices p of the tiles (TMEM) x slices q of the trials (smem);
                // trial rows: [u' (16 j) | c_y y' (16 j)], 32 B each (2 descriptor units)
#pragma unroll
                for (int l = 0; l < kO64Levels; ++l) {
                    const uint32_t d = tmem + o64_dcol(l);
#pragma unroll
                    for (int p = 0; p <= l; ++p) {
                        const uint64_t bd = tc::sdesc_kmajor_sw64(base + (l - p) * L.tile_bytes);
                        tc::mma_f16_ts(d, tmem + o64_acol(p, 0), bd, idesc, p == 0 ? 0u : 1u);
                        tc::mma_f16_ts(d, tmem + o64_acol(p, 1), bd + 2u, idesc, 1u);
                    }
                }
                tc::commit(mma_done);
                mma_any = true;
            }
        }
        if (!__all_sync(0xffffffffu, !*abort_flag)) break;
        pending = true;
        riv_prev = riv;
        pslot = slot;
        mph ^= 1u;
        if (++slot == kO64Ring) {
            slot = 0;
            ph ^= 1u;
        }
        ++gs;
        if (m.flags & O64_LAST) {  // the unit's last stage: drain it and write the rows out
            if (!drain(mph ^ 1u, riv_prev,
                       reinterpret_cast<const float*>(smem + L.civ_off + pslot * kO64Ppad * 4)))
                break;
            if (lane == 0) mbar_arrive(&b_empty[pslot]);
            if (is_producer && !pr->end && !produce()) *abort_flag = 1;
            pending = false;
            flush(kind0, i);
            if (!__all_sync(0xffffffffu, !*abort_flag)) break;
        }
    }
    tc::wait_st();
    tc::wait_ld();
    if (is_producer) {  // copies in flight must land before the CTA exits
        // (after the end marker, its slot's previous stage was drained before it was written,
        // and that slot's parity has moved on: wait for the other ring slots only)
        const int64_t issued = pr->issued;
        const int64_t back = pr->end ? kO64Ring - 1 : kO64Ring;
        for (int64_t k = (issued > back ? issued - back : 0); k < issued; ++k)
            mbar_wait(&b_full[k % kO64Ring], static_cast<uint32_t>((k / kO64Ring) & 1), args.err);
    }
    if (is_mma && mma_any) {  // every MMA finished before TMEM is released
        tc::commit(fin);
        mbar_wait(fin, 0, args.err);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kO64TmemCols);
    }
}

// ---------------------------------------------------------------- records and trial slices

__device__ __forceinline__ float2 o64_split(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - static_cast<double>(h)));
}

// Pair records of the kept points (padding points keep the prepared padding values): point j
// writes lane j & 1 of pair record j / 2.
__global__ void __launch_bounds__(256)
k_o64_records(const double4* __restrict__ r64a, const double4* __restrict__ r64b, int64_t nk_pad,
              O64Rec* __restrict__ rec) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= nk_pad) return;
    const double4 a = r64a[j], b = r64b[j];
    const double vals[7] = {a.x, a.y, a.z, b.x, b.y, b.z, b.w};  // x y z omega kappa p q
    float* r = reinterpret_cast<float*>(rec + (j >> 1)) + (j & 1);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const float2 v = o64_split(vals[q]);
        r[4 * q] = v.x;      // hi of this lane
        r[4 * q + 2] = v.y;  // lo of this lane
    }
    if ((j & 1) == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) r[28 + k] = 0.0f;
    }
}

// Largest |u'| and |y'| over all trials (u' = -3/2 u, y' = 3/2 y) as FP64 bit patterns
// (non-negative doubles order like unsigned integers); colmax[0..1] zeroed before.
__global__ void __launch_bounds__(256)
k_o64_colmax(const double* __restrict__ u, const double* __restrict__ y, int64_t nk_pad,
             unsigned long long* __restrict__ colmax) {
    const int t = blockIdx.y;
    const double* ut = u + static_cast<int64_t>(t) * nk_pad;
    const double* yt = y + static_cast<int64_t>(t) * nk_pad;
    double mu = 0.0, my = 0.0;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < nk_pad;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        mu = fmax(mu, fabs(1.5 * ut[j]));
        my = fmax(my, fabs(1.5 * yt[j]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mu = fmax(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&colmax[0], static_cast<unsigned long long>(__double_as_longlong(mu)));
        atomicMax(&colmax[1], static_cast<unsigned long long>(__double_as_longlong(my)));
    }
}

// c_y: a power of two near max|u'| / max|y'| (clamped to 2^[-60, 60]); params[0] = 1/c_y,
// params[1] = c_y.
__global__ void k_o64_balance(const unsigned long long* __restrict__ colmax,
                              double* __restrict__ params) {
    const double mu = __longlong_as_double(static_cast<long long>(colmax[0]));
    const double my = __longlong_as_double(static_cast<long long>(colmax[1]));
    long long e = 0;
    if (mu > 0.0 && my > 0.0 && isfinite(mu) && isfinite(my)) {
        e = ((__double_as_longlong(mu) >> 52) & 0x7FF) - ((__double_as_longlong(my) >> 52) & 0x7FF);
        e = e > 60 ? 60 : (e < -60 ? -60 : e);
    }
    params[0] = ldexp(1.0, static_cast<int>(-e));
    params[1] = ldexp(1.0, static_cast<int>(e));
}

// The seven FP16 slice arrays [rows][2 nk_pad] (per 16-j block: 16 u' then 16 c_y y', scaled by
// the block's column factor; slices exact in FP64) and the factors' inverses
// civ[group][n_stage][32] for trial groups [g pg, g pg + pg): one half-warp per (trial, 16-j
// block).  Rows t >= P are zero.
__global__ void __launch_bounds__(256)
k_o64_split(const double* __restrict__ u, const double* __restrict__ y, int32_t P, int32_t pg,
            int64_t nk_pad, const double* __restrict__ params, __half* __restrict__ out,
            int64_t slice_stride, float* __restrict__ civ) {
    const int t = blockIdx.y;
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;  // < nk_pad
    double a = 0.0, b = 0.0;
    if (t < P) {
        const int64_t o = static_cast<int64_t>(t) * nk_pad + j;
        a = -1.5 * u[o];
        b = 1.5 * y[o] * params[1];
    }
    // the block maximum in FP32 (rounding can only carry it up to the next power of two,
    // which keeps the scaled values below 2^7)
    float m = static_cast<float>(fmax(fabs(a), fabs(b)));
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    float sc, isc;
    o64_scale_f(m, sc, isc);
    double ra = a * sc, rb = b * sc;
    const int64_t off = static_cast<int64_t>(t) * (2 * nk_pad) + (j >> 4) * 32 + (j & 15);
#pragma unroll
    for (int q = 0; q < kO64Slices; ++q) {
        const double sa = rint(ra), sb = rint(rb);
        out[q * slice_stride + off] = __float2half_rn(static_cast<float>(sa));  // integers, exact
        out[q * slice_stride + off + 16] = __float2half_rn(static_cast<float>(sb));
        ra = (ra - sa) * 256.0;
        rb = (rb - sb) * 256.0;
    }
    if (t < P && (j & 15) == 0) {
        const int g = t / pg, c = t - g * pg;
        const int64_t n_stage = nk_pad / kO64Kj;
        civ[(static_cast<int64_t>(g) * n_stage + (j >> 4)) * kO64Ppad + c] = isc;
    }
}

// ---------------------------------------------------------------- host side

static PFN_cuTensorMapEncodeTiled_v12000 o64_encode_fn() {
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

// [rows][2 nk_pad] halves; box 32 halves (one stage: 16 u', 16 c_y y') x 32 rows, 64-byte swizzle.
static bool o64_make_map(CUtensorMap* m, const void* base, int64_t nk_pad, int64_t rows) {
    auto fn = o64_encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(2 * nk_pad), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(2 * nk_pad) * sizeof(__half)};
    cuuint32_t box[2] = {32u, static_cast<cuuint32_t>(kO64Ppad)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int hess_o64_max_group() { return kO64Ppad; }
int hess_o64_slices() { return kO64Slices; }
int64_t hess_o64_civ_floats(int32_t P, int32_t pg, int64_t nk_pad) {
    return static_cast<int64_t>((P + pg - 1) / pg) * (nk_pad / kO64Kj) * kO64Ppad;
}

cudaError_t launch_o64_prep(const PointsDev& p, const double* u, const double* y, int32_t P,
                            int32_t rows, int32_t pg, void* rec, unsigned long long* colmax,
                            double* params, void* slices, int64_t slice_stride, float* civ,
                            cudaStream_t st) {
    const int64_t nk_pad = p.nk_pad;
    if (nk_pad % 256 != 0 || pg < 1 || pg > kO64Ppad) return cudaErrorInvalidValue;
    const int ng = (P + pg - 1) / pg;
    const int64_t nb = nk_pad / 256;
    k_o64_records<<<static_cast<unsigned>(nb), 256, 0, st>>>(p.r64a, p.r64b, nk_pad,
                                                              static_cast<O64Rec*>(rec));  // nk_pad / 2 pair records
    cudaError_t e = cudaMemsetAsync(colmax, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    // zero factors for the padding columns of every group
    e = cudaMemsetAsync(civ, 0, sizeof(float) * static_cast<size_t>(ng) * (nk_pad / kO64Kj) * kO64Ppad, st);
    if (e != cudaSuccess) return e;
    dim3 g1(static_cast<unsigned>(nb < 16 ? nb : 16), static_cast<unsigned>(P));
    k_o64_colmax<<<g1, 256, 0, st>>>(u, y, nk_pad, colmax);
    k_o64_balance<<<1, 1, 0, st>>>(colmax, params);
    dim3 g2(static_cast<unsigned>(nb), static_cast<unsigned>(rows));
    k_o64_split<<<g2, 256, 0, st>>>(u, y, P, pg, nk_pad, params, static_cast<__half*>(slices),
                                    slice_stride, civ);
    return cudaGetLastError();
}

cudaError_t launch_hess_o64(const PointsDev& p, int32_t Pn, int32_t t0, int64_t acc_P,
                            const void* rec, const void* slices, int64_t slice_stride,
                            int64_t rows, const float* civ, const double* params, int n_sm,
                            int flush, double* acc, int* err, cudaStream_t st) {
    if (p.nk == 0) return cudaSuccess;
    if (Pn < 1 || Pn > kO64Ppad || t0 + kO64Ppad > rows || p.nk_pad % 256 != 0)
        return cudaErrorInvalidValue;
    CUtensorMap maps[kO64Slices];
    for (int q = 0; q < kO64Slices; ++q)
        if (!o64_make_map(&maps[q], static_cast<const __half*>(slices) + q * slice_stride, p.nk_pad, rows))
            return cudaErrorInvalidValue;
    O64Args a;
    memset(&a, 0, sizeof(a));
    a.rec = static_cast<const O64Rec*>(rec);
    a.acc = acc;
    a.civ = civ;
    a.params = params;
    a.nk = p.nk;
    a.nk_pad = p.nk_pad;
    a.acc_P = acc_P;
    a.Pn = Pn;
    a.t0 = t0;
    a.n_units = 2 * ((p.nk + 127) / 128);
    a.n_stage = static_cast<int32_t>(p.nk_pad / kO64Kj);
    constexpr O64Layout L = o64_layout();
    const size_t stage_bytes = L.slot_bytes + kO64Kj * kO64RecBytes;
    int64_t chunk = static_cast<int64_t>(kO64ChunkBytes / stage_bytes);
    if (chunk < 64) chunk = 64;
    a.chunk = static_cast<int32_t>(chunk < a.n_stage ? chunk : a.n_stage);
    a.flush = flush > 0 ? flush : 512;
    a.err = err;
    cudaError_t e = cudaFuncSetAttribute(k_hess_o64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L.total));
    if (e != cudaSuccess) return e;
    const int grid = static_cast<int>(a.n_units < n_sm ? a.n_units : n_sm);
    k_hess_o64<<<grid, kO64Threads, L.total, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4],
                                                   maps[5], maps[6], a);
    return cudaGetLastError();
}

}  // namespace vv10
