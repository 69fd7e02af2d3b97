// The weight-derivative sums (Sec. II.B, E_i^{Bw}, U_i^{Bw}, W_i^{Bw}) on tensor cores: with
// y_j = -3/2 rho_j v_j for a direction v and inv = 1/(g g' s) (so that y_j inv = v_j rho_j Phi_ij),
//   E^v = K1 y,  U^v = -K2 y,  W^v = -K3 y,
//   K1_ij = inv,  K2_ij = inv (1/s + 1/g),  K3_ij = K2_ij R^2,
// three N x N kernel matrices times the N x P direction matrix, split-TF32 (hi*hi + hi*lo +
// lo*hi) on tcgen05.
//
// Work unit ("task"): 128 rows i x one group of at most 64 directions (N of the MMA) x every
// j.  A persistent CTA walks its tasks; per stage of 16 j:
//   * 16 generator warps (4 per row quadrant, 4 j each) evaluate K1, K2, K3 for their row in
//     FP32 and split them into TF32 hi/lo: the three hi tiles go to tensor memory (their MMAs
//     read no shared memory for A), the three lo tiles to shared memory in the
//     64-byte-swizzled K-major layout (both double-buffered);
//   * the producer warp fetches the stage's j-records (1-D bulk copy) and the two 16 x Ppad
//     direction tiles y_hi, y_lo (2-D TMA, 64-byte swizzle) into a ring;
//   * one thread issues 6 MMAs per kind (2 k-steps x 3 products; B from shared memory, A from
//     tensor memory (hi) or shared memory (lo)) into that kind's TMEM accumulator
//     (double-buffered: 3 kinds x 2 x 64 columns), the first of each kind overwriting it,
//     and commits the stage once;
//   * the generator warps drain the finished stage's accumulators into FP32 registers,
//     release the ring slot, and every `flush` stages add the registers into the FP64
//     outputs (each task's rows and directions are owned by one CTA: no atomics).
// As in the Hessian contraction, each TMEM accumulation run is one stage with the hi*lo and
// lo*hi products first and the hi*hi products last (the tensor core truncates).
#include <cstring>
#include <cuda.h>

#include "common.cuh"
#include "kernels.hpp"
#include "tc.cuh"

namespace vv10 {

namespace {

constexpr int kWtKj = 16;                       // j per stage
constexpr int kWtGenWarps = 16;                 // generator / drain warps (4 per row quadrant)
constexpr int kWtProducerWarp = kWtGenWarps;    // TMA producer
constexpr int kWtMmaWarp = kWtGenWarps + 1;     // MMA issuer + TMEM owner
constexpr int kWtThreads = (kWtGenWarps + 2) * 32;
constexpr int kWtRing = 4;                      // stages of direction tiles in flight
constexpr int kWtKinds = 3;                     // E, U, W
constexpr int kWtMaxPpad = 64;
constexpr uint32_t kWtTmemCols = 512;
constexpr uint32_t kWtATile = 128u * 64u;       // one 128 x 16 tf32 operand tile (bytes)
constexpr uint32_t kWtABuf = kWtKinds * kWtATile;  // the lo parts of the three kernel tiles
constexpr uint32_t kWtAHiCol = 384u;            // TMEM: hi tiles of buffer b, kind k at 384 + 48 b + 16 k

struct WtLayout {
    uint32_t ring_off;    // direction-tile ring (after the two A buffers)
    uint32_t tile_bytes;  // one 16 x Ppad direction tile
    uint32_t ring_bytes;  // y_hi + y_lo
    uint32_t rec_off;     // j-records
    uint32_t bar_off;     // barriers
    uint32_t total;
};
__host__ __device__ inline WtLayout wt_layout(int ppad) {
    WtLayout L;
    L.ring_off = 2u * kWtABuf;
    L.tile_bytes = static_cast<uint32_t>(ppad) * 64u;
    L.ring_bytes = 2u * L.tile_bytes;
    L.rec_off = L.ring_off + kWtRing * L.ring_bytes;
    L.bar_off = L.rec_off + kWtRing * 512u;
    L.total = L.bar_off + 256u + 1024u;  // barriers + slack for 1024-B alignment
    return L;
}

struct WtArgs {
    const float4* r32a;   // row records (x, y, z, c) and (omega, kappa, p, q)
    const float4* r32b;
    const float4* r32p;   // pair-packed column records
    const int64_t* orig;  // kept -> caller index
    double* out[kWtKinds];  // E, U, W: P x n in caller order (each may be null), zero on entry
    int64_t nk, nk_pad, n;
    int32_t P;            // directions
    int32_t n_groups;     // direction groups of Ppad
    int64_t n_tasks;      // row tiles x groups
    int flush;            // stages per FP64 flush
    int* err;
};

__device__ __forceinline__ bool wt_wait(uint64_t* bar, uint32_t parity, int* err,
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

__device__ __forceinline__ float2 wlo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 whi2(float4 v) { return make_float2(v.z, v.w); }

// K1, K2, K3 for two j at once from a pair-packed record v0..v2 = {-x,-y}, {-z,om}, {ka,..}.
__device__ __forceinline__ void weight_tiles2(float2 xi, float2 yi, float2 zi, float2 oi,
                                              float2 ki, const float4 v0, const float4 v1,
                                              const float4 v2, float2 (&k)[kWtKinds]) {
    const float2 dx = __fadd2_rn(xi, wlo2(v0));
    const float2 dy = __fadd2_rn(yi, whi2(v0));
    const float2 dz = __fadd2_rn(zi, wlo2(v1));
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    const float2 g = __ffma2_rn(oi, r2, ki);
    const float2 gp = __ffma2_rn(whi2(v1), r2, wlo2(v2));
    const float2 s = __fadd2_rn(g, gp);
    const float2 ggp = __fmul2_rn(g, gp);
    const float2 den = __fmul2_rn(ggp, s);
    float2 inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv.x) : "f"(den.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv.y) : "f"(den.y));
    const float2 t1 = __fmul2_rn(__ffma2_rn(gp, s, ggp), inv);  // 1/s + 1/g
    k[0] = inv;
    k[1] = __fmul2_rn(inv, t1);
    k[2] = __fmul2_rn(k[1], r2);
}

__device__ __forceinline__ uint32_t tf32_hi_bits(float x) {
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;  // round to nearest on the bit pattern
}

// TMEM accumulator of kind k, buffer b.
__device__ __forceinline__ uint32_t wt_dcol(int k, int b) { return 64u * (2 * k + b); }

template <int PQ>  // accumulator columns per generator thread and kind (= Ppad / 4)
__global__ void __launch_bounds__(kWtThreads, 1)
k_wresp_tc(const __grid_constant__ CUtensorMap tm_yh, const __grid_constant__ CUtensorMap tm_yl,
           WtArgs args) {
    constexpr int PPAD = 4 * PQ;
    static_assert(PPAD <= kWtMaxPpad && PQ % 8 == 0, "Ppad must be 32 or 64");
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const WtLayout L = wt_layout(PPAD);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* b_full = bars;                      // [kWtRing]
    uint64_t* b_empty = bars + kWtRing;           // [kWtRing]
    uint64_t* a_full = bars + 2 * kWtRing;        // [2]
    uint64_t* mma_done = bars + 2 * kWtRing + 2;  // [2]
    uint64_t* fin = bars + 2 * kWtRing + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kWtRing + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * kWtRing + 6);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_stage = static_cast<int>(args.nk_pad / kWtKj);

    if (threadIdx.x == 0) {
        for (int b = 0; b < kWtRing; ++b) {
            mbar_init(&b_full[b], 1);
            mbar_init(&b_empty[b], kWtGenWarps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&a_full[b], kWtGenWarps);
            mbar_init(&mma_done[b], 1);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kWtMmaWarp) tc::tmem_alloc(tmem_slot, kWtTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == kWtProducerWarp) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            tc::prefetch_tmap(&tm_yh);
            tc::prefetch_tmap(&tm_yl);
            int slot = 0;
            uint32_t ph = 0;
            int64_t issued = 0;
            bool ok = true;
            for (int64_t q = blockIdx.x; q < args.n_tasks && ok; q += gridDim.x) {
                const int t0 = static_cast<int>(q % args.n_groups) * PPAD;
                for (int s = 0; s < n_stage; ++s) {
                    if (!wt_wait(&b_empty[slot], ph ^ 1u, args.err, abort_flag)) {
                        ok = false;
                        break;
                    }
                    uint8_t* base = smem + L.ring_off + slot * L.ring_bytes;
                    uint8_t* rec = smem + L.rec_off + slot * 512;
                    const int j0 = s * kWtKj;
                    mbar_expect_tx(&b_full[slot], L.ring_bytes + 512u);
                    bulk_g2s(rec, args.r32p + 2 * j0, 512u, &b_full[slot]);
                    tc::tma_load_2d(base, &tm_yh, j0, t0, &b_full[slot]);
                    tc::tma_load_2d(base + L.tile_bytes, &tm_yl, j0, t0, &b_full[slot]);
                    ++issued;
                    if (++slot == kWtRing) {
                        slot = 0;
                        ph ^= 1u;
                    }
                }
            }
            // copies in flight must land before the CTA exits
            for (int64_t k = (issued > kWtRing ? issued - kWtRing : 0); k < issued; ++k)
                mbar_wait(&b_full[k % kWtRing], static_cast<uint32_t>((k / kWtRing) & 1), args.err);
        }
    } else if (warp == kWtMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(128, PPAD);
            constexpr uint64_t kStep = 32u >> 4;  // +32 B (8 tf32 along K) in the address field
            int slot = 0, ab = 0;
            uint32_t ph = 0, aph = 0;
            bool ok = true, issued_any = false;
            for (int64_t q = blockIdx.x; q < args.n_tasks && ok; q += gridDim.x) {
                for (int s = 0; s < n_stage; ++s) {
                    if (!wt_wait(&a_full[ab], aph, args.err, abort_flag) ||
                        !wt_wait(&b_full[slot], ph, args.err, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t yb = smem_u32(smem + L.ring_off + slot * L.ring_bytes);
                    const uint64_t dyh = tc::sdesc_kmajor_sw64(yb);
                    const uint64_t dyl = tc::sdesc_kmajor_sw64(yb + L.tile_bytes);
                    const uint32_t abase = smem_u32(smem + ab * kWtABuf);
#pragma unroll
                    for (int k = 0; k < kWtKinds; ++k) {
                        const uint32_t d = tmem + wt_dcol(k, ab);
                        const uint32_t ah = tmem + kWtAHiCol + 48u * ab + 16u * k;
                        const uint64_t dal = tc::sdesc_kmajor_sw64(abase + k * kWtATile);
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            tc::mma_tf32_ts(d, ah + 8 * kk, dyl + kStep * kk, idesc, kk);  // the first overwrites
                            tc::mma_tf32_ss(d, dal + kStep * kk, dyh + kStep * kk, idesc, 1);
                        }
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
                            tc::mma_tf32_ts(d, ah + 8 * kk, dyh + kStep * kk, idesc, 1);
                    }
                    issued_any = true;
                    tc::commit(&mma_done[ab]);  // the ring slot is released by the generators
                    if (++slot == kWtRing) {
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
        const int r = quad * 32 + lane;  // row within the 128-row tile
        // this thread's 16-byte chunk (its warp's 4 j) in each operand row, 64-B swizzle
        const uint32_t a_row = static_cast<uint32_t>(r) * 64u +
                               (static_cast<uint32_t>(part ^ ((r >> 1) & 3)) << 4);
        float acc[kWtKinds][PQ];
#pragma unroll
        for (int k = 0; k < kWtKinds; ++k)
#pragma unroll
            for (int c = 0; c < PQ; ++c) acc[k][c] = 0.0f;
        bool ok = true;

        auto drain = [&](int db, uint32_t dphase) -> bool {
            const bool got = wt_wait(&mma_done[db], dphase, args.err, abort_flag);
            if (!__all_sync(0xffffffffu, got)) return false;  // warp-uniform exit
            tc::fence_after();
#pragma unroll
            for (int k = 0; k < kWtKinds; ++k) {
                uint32_t rr[PQ];
#pragma unroll
                for (int c = 0; c < PQ; c += 8) {
                    uint32_t (&rc)[8] = *reinterpret_cast<uint32_t(*)[8]>(&rr[c]);
                    tc::ld_x8(tmem + lane_off + wt_dcol(k, db) + part * PQ + c, rc);
                }
                tc::wait_ld();
#pragma unroll
                for (int c = 0; c < PQ; c += 2) {
                    const float2 v = __fadd2_rn(make_float2(acc[k][c], acc[k][c + 1]),
                                                make_float2(__uint_as_float(rr[c]), __uint_as_float(rr[c + 1])));
                    acc[k][c] = v.x;
                    acc[k][c + 1] = v.y;
                }
            }
            tc::fence_before();
            return true;
        };
        auto flush = [&](int t0, int64_t i) {
            const bool row_ok = i < args.nk;
            const int64_t oi = row_ok ? args.orig[i] : 0;
#pragma unroll
            for (int k = 0; k < kWtKinds; ++k) {
                double* o = args.out[k];
#pragma unroll
                for (int c = 0; c < PQ; ++c) {
                    const int t = t0 + part * PQ + c;
                    if (o && row_ok && t < args.P) {
                        const double v = static_cast<double>(acc[k][c]);
                        o[static_cast<int64_t>(t) * args.n + oi] += (k == 0) ? v : -v;
                    }
                    acc[k][c] = 0.0f;
                }
            }
        };

        int slot = 0, ab = 0;
        uint32_t ph = 0, aph = 0;
        int pslot = 0, dbuf = 0;
        uint32_t dph = 0;
        for (int64_t q = blockIdx.x; q < args.n_tasks && ok; q += gridDim.x) {
            const int64_t row_tile = q / args.n_groups;
            const int t0 = static_cast<int>(q % args.n_groups) * PPAD;
            const int64_t i = row_tile * 128 + r;
            float xi = 0.f, yi = 0.f, zi = 0.f, oi = 1.f, ki = 1.f;
            if (i < args.nk) {
                const float4 a = args.r32a[i];
                const float4 b = args.r32b[i];
                xi = a.x; yi = a.y; zi = a.z; oi = b.x; ki = b.y;
            }
            const float2 X = make_float2(xi, xi), Y = make_float2(yi, yi), Z = make_float2(zi, zi);
            const float2 O = make_float2(oi, oi), K = make_float2(ki, ki);
            int until_flush = args.flush;
            for (int s = 0; s < n_stage; ++s) {
                // operand buffer ab is free once the MMAs of the stage two back are done
                bool got = wt_wait(&b_full[slot], ph, args.err, abort_flag);
                got = got && wt_wait(&mma_done[ab], aph ^ 1u, args.err, abort_flag);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                const float4* rec = reinterpret_cast<const float4*>(smem + L.rec_off + slot * 512);
                uint32_t hi[kWtKinds][4], lo[kWtKinds][4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float4* v = rec + 4 * (2 * part + h);
                    float2 kv[kWtKinds];
                    weight_tiles2(X, Y, Z, O, K, v[0], v[1], v[2], kv);
#pragma unroll
                    for (int k = 0; k < kWtKinds; ++k) {
                        const uint32_t h0 = tf32_hi_bits(kv[k].x), h1 = tf32_hi_bits(kv[k].y);
                        hi[k][2 * h] = h0;
                        hi[k][2 * h + 1] = h1;
                        lo[k][2 * h] = __float_as_uint(kv[k].x - __uint_as_float(h0));
                        lo[k][2 * h + 1] = __float_as_uint(kv[k].y - __uint_as_float(h1));
                    }
                }
                const uint32_t abuf = smem_u32(smem + ab * kWtABuf) + a_row;
                const uint32_t ahi = tmem + lane_off + kWtAHiCol + 48u * ab + part * 4;
#pragma unroll
                for (int k = 0; k < kWtKinds; ++k) {
                    tc::st_x4(ahi + 16u * k, hi[k]);
                    tc::st_shared_v4(abuf + k * kWtATile, lo[k][0], lo[k][1], lo[k][2], lo[k][3]);
                }
                tc::wait_st();
                tc::fence_before();
                tc::fence_proxy_async_smem();  // the operands are read by the tensor core
                __syncwarp();
                if (lane == 0) mbar_arrive(&a_full[ab]);
                // drain the previous stage while this stage's MMAs run
                if (s > 0) {
                    if (!drain(dbuf, dph)) {
                        ok = false;
                        break;
                    }
                    if (lane == 0) mbar_arrive(&b_empty[pslot]);
                    if (--until_flush == 0) {
                        flush(t0, i);
                        until_flush = args.flush;
                    }
                }
                dbuf = ab;
                dph = aph;
                pslot = slot;
                if (++slot == kWtRing) {
                    slot = 0;
                    ph ^= 1u;
                }
                ab ^= 1;
                if (ab == 0) aph ^= 1u;
            }
            if (!ok) break;
            if (!drain(dbuf, dph)) {
                ok = false;
                break;
            }
            if (lane == 0) mbar_arrive(&b_empty[pslot]);
            flush(t0, i);
        }
        tc::wait_st();  // nothing of ours is in flight to or from TMEM on any exit path
        tc::wait_ld();
    }

    tc::fence_before();
    __syncthreads();
    if (warp == kWtMmaWarp) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kWtTmemCols);
    }
}

// y (Pn x nk_pad FP64, -3/2 rho v) -> TF32 hi and FP32 lo, rows x nk_pad (rows >= Pn are zero).
__global__ void k_wdir_split(const double* __restrict__ yk, int32_t Pn, int64_t nk_pad,
                             float* __restrict__ yh, float* __restrict__ yl) {
    const int t = blockIdx.y;
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= nk_pad) return;
    const int64_t o = static_cast<int64_t>(t) * nk_pad + p;
    const float a = t < Pn ? static_cast<float>(yk[o]) : 0.0f;
    const float ah = __uint_as_float(tc::to_tf32(a));
    yh[o] = ah;
    yl[o] = a - ah;
}

template <int PQ>
cudaError_t launch_wt(const CUtensorMap* maps, const WtArgs& a, int n_sm, cudaStream_t st) {
    const WtLayout L = wt_layout(4 * PQ);
    cudaError_t e = cudaFuncSetAttribute(k_wresp_tc<PQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L.total));
    if (e != cudaSuccess) return e;
    const int grid = static_cast<int>(a.n_tasks < n_sm ? a.n_tasks : n_sm);
    if (grid <= 0) return cudaSuccess;
    k_wresp_tc<PQ><<<grid, kWtThreads, L.total, st>>>(maps[0], maps[1], a);
    return cudaGetLastError();
}

}  // namespace

// Direction groups for P directions: (groups, padded width 32 or 64).
void weight_tc_groups(int32_t P, int* n_groups, int* ppad) {
    const int ng = (P + kWtMaxPpad - 1) / kWtMaxPpad;
    const int pg = (P + ng - 1) / ng;
    *n_groups = ng;
    *ppad = pg <= 32 ? 32 : 64;
}

cudaError_t launch_weight_split(const double* yk, int32_t Pn, int32_t rows, int64_t nk_pad,
                                float* yh, float* yl, cudaStream_t st) {
    if (nk_pad == 0 || rows <= 0) return cudaSuccess;
    const dim3 g(static_cast<unsigned>((nk_pad + 255) / 256), static_cast<unsigned>(rows));
    k_wdir_split<<<g, 256, 0, st>>>(yk, Pn, nk_pad, yh, yl);
    return cudaGetLastError();
}

cudaError_t launch_weight_tc(const PointsDev& p, int32_t Pn, const float* yh, const float* yl,
                             int32_t rows, double* E, double* U, double* W, int n_sm, int* err,
                             cudaStream_t st) {
    if (p.nk == 0 || Pn <= 0) return cudaSuccess;
    int ng = 0, ppad = 0;
    weight_tc_groups(Pn, &ng, &ppad);
    if (rows < ng * ppad) return cudaErrorInvalidValue;
    CUtensorMap maps[2];
    if (!tc_make_map_f32(&maps[0], yh, p.nk_pad, rows, ppad) ||
        !tc_make_map_f32(&maps[1], yl, p.nk_pad, rows, ppad))
        return cudaErrorInvalidValue;
    WtArgs a;
    a.r32a = p.r32a;
    a.r32b = p.r32b;
    a.r32p = p.r32p;
    a.orig = p.orig;
    a.out[0] = E;
    a.out[1] = U;
    a.out[2] = W;
    a.nk = p.nk;
    a.nk_pad = p.nk_pad;
    a.n = p.n;
    a.P = Pn;
    a.n_groups = ng;
    a.n_tasks = static_cast<int64_t>(ng) * ((p.nk + 127) / 128);
    a.flush = 512;
    a.err = err;
    return ppad == 32 ? launch_wt<8>(maps, a, n_sm, st) : launch_wt<16>(maps, a, n_sm, st);
}

}  // namespace vv10
