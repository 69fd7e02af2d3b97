// K3 on tensor cores: the pair part of Eq. frhot (Sec. II.B) as a product of generated
// kernel tiles with the trial matrix, split-TF32 (hi*hi + hi*lo + lo*hi) on tcgen05.
//
// Work unit ("tile"): 128 rows i (TMEM lanes) x one output kind (0: f^{rho,t} with
// kernel tiles T1 | T2, 1: f^{gamma,t} / sigma_i with T3 | T4) x all P trials (N of the
// MMA, padded to a multiple of 32, <= 192) x every j.  A persistent CTA walks its tiles;
// per stage of 16 j:
//   * 8 generator warps (2 per TMEM lane quadrant, 8 j each) evaluate the two kernel
//     tiles for their row in FP32, split them into TF32 hi/lo and store the four 128x16
//     operand tiles into tensor memory (tcgen05.st);
//   * the producer warp fetches the stage's j-records (1-D bulk copy) and the four
//     16 x P trial tiles u_hi, u_lo, y_hi, y_lo (2-D TMA, 64-byte swizzle) into a ring;
//   * one thread issues 12 MMAs (2 k-steps x 6 products) into a TMEM accumulator
//     (double-buffered), the first of each stage overwriting it;
//   * the generator warps drain the finished stage's accumulator into FP32 registers
//     (round-to-nearest adds) and every `flush` stages add those into the FP64 partial
//     output in global memory (each tile's rows are owned by one CTA: no atomics).
// The tensor core accumulates with truncation, so each TMEM accumulation run is kept to
// one stage (12 adds); the register and FP64 levels bound the rest of the rounding.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.hpp"
#include "tc.cuh"

namespace vv10 {

constexpr int kTcKj = 16;                        // j per stage
constexpr int kTcGenWarps = 8;                   // generator / drain warps
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

struct TcArgs {
    PointsDev P;
    int32_t Pn;       // trials in this launch
    int32_t t0;       // first trial of this launch (row offset into the split arrays)
    int64_t acc_P;    // trial count of the FP64 accumulator layout
    int64_t n_row_tiles;
    int flush;        // stages per FP64 flush
    double* acc;      // [2][acc_P][nk_pad], zero on entry
    int* err;
};

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

// Kernel tiles of one pair: kind 0 -> (T1, T2), kind 1 -> (T3, T4); FP32.
__device__ __forceinline__ void pair_tiles(int kind, float xi, float yi, float zi, float oi,
                                           float ki, float pi_, float qi, const float4& a,
                                           const float4& b, float& ta, float& tb) {
    const float dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
    float r2 = dx * dx;
    r2 = __fmaf_rn(dy, dy, r2);
    r2 = __fmaf_rn(dz, dz, r2);
    const float g = __fmaf_rn(oi, r2, ki);
    const float gp = __fmaf_rn(b.x, r2, b.y);
    const float s = g + gp;
    const float ggp = g * gp;
    const float inv = rcp_refined(ggp * s);
    const float phi = -1.5f * inv;
    const float L = ggp * inv;
    const float Gi = (gp * s) * inv;
    const float Gj = (g * s) * inv;
    const float M = 2.0f * __fmaf_rn(L, L, Gi * Gj);
    const float Ai = __fmaf_rn(qi, r2, pi_);   // rho_i a_i
    const float Aj = __fmaf_rn(b.w, r2, b.z);  // rho_j a_j
    const float rp = r2 * phi;
    if (kind == 0) {
        const float LGi = L + Gi, LGj = L + Gj;
        float br = __fmaf_rn(-Ai, LGi, 1.0f);
        br = __fmaf_rn(-Aj, LGj, br);
        br = __fmaf_rn(Ai * Aj, M, br);
        ta = phi * br;                            // T1
        tb = rp * __fmaf_rn(Ai, M, -LGj);         // T2
    } else {
        ta = rp * __fmaf_rn(Aj, M, -(L + Gi));    // T3
        tb = (rp * r2) * M;                       // T4
    }
}

template <int PH>  // accumulator columns per generator thread (= Ppad / 2)
__global__ void __launch_bounds__(kTcThreads, 1)
k_hess_tc(const __grid_constant__ CUtensorMap tm_uh, const __grid_constant__ CUtensorMap tm_ul,
          const __grid_constant__ CUtensorMap tm_yh, const __grid_constant__ CUtensorMap tm_yl,
          TcArgs args) {
    constexpr int PPAD = 2 * PH;
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
    const PointsDev& P = args.P;
    const int64_t n_stage = P.nk_pad / kTcKj;
    const int64_t n_tiles = 2 * args.n_row_tiles;

    if (threadIdx.x == 0) {
        for (int b = 0; b < kTcRing; ++b) {
            mbar_init(&b_full[b], 1);
            mbar_init(&b_empty[b], 1 + kTcGenWarps);
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
            tc::prefetch_tmap(&tm_uh);
            tc::prefetch_tmap(&tm_ul);
            tc::prefetch_tmap(&tm_yh);
            tc::prefetch_tmap(&tm_yl);
            int64_t gs = 0;
            bool ok = true;
            for (int64_t q = blockIdx.x; q < n_tiles && ok; q += gridDim.x) {
                for (int64_t s = 0; s < n_stage && ok; ++s, ++gs) {
                    const int slot = static_cast<int>(gs % kTcRing);
                    const uint32_t ph = static_cast<uint32_t>((gs / kTcRing) & 1);
                    if (!wait_or_abort(&b_empty[slot], ph ^ 1u, args.err, abort_flag)) {
                        ok = false;
                        break;
                    }
                    uint8_t* base = smem + slot * L.ring_bytes;
                    uint8_t* rec = smem + L.rec_off + slot * 512;
                    const int j0 = static_cast<int>(s * kTcKj);
                    mbar_expect_tx(&b_full[slot], L.ring_bytes + 512u);
                    bulk_g2s(rec, P.r32a + j0, 256u, &b_full[slot]);
                    bulk_g2s(rec + 256, P.r32b + j0, 256u, &b_full[slot]);
                    tc::tma_load_2d(base + 0 * L.tile_bytes, &tm_uh, j0, args.t0, &b_full[slot]);
                    tc::tma_load_2d(base + 1 * L.tile_bytes, &tm_ul, j0, args.t0, &b_full[slot]);
                    tc::tma_load_2d(base + 2 * L.tile_bytes, &tm_yh, j0, args.t0, &b_full[slot]);
                    tc::tma_load_2d(base + 3 * L.tile_bytes, &tm_yl, j0, args.t0, &b_full[slot]);
                }
            }
            // copies in flight must land before the CTA exits
            for (int64_t k = (gs > kTcRing ? gs - kTcRing : 0); k < gs; ++k)
                mbar_wait(&b_full[k % kTcRing], static_cast<uint32_t>((k / kTcRing) & 1), args.err);
        }
    } else if (warp == kTcMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(128, PPAD);
            int64_t gs = 0;
            bool ok = true, issued_any = false;
            for (int64_t q = blockIdx.x; q < n_tiles && ok; q += gridDim.x) {
                for (int64_t s = 0; s < n_stage; ++s, ++gs) {
                    const int slot = static_cast<int>(gs % kTcRing);
                    const int ab = static_cast<int>(gs & 1);
                    if (!wait_or_abort(&a_full[ab], static_cast<uint32_t>((gs >> 1) & 1), args.err, abort_flag) ||
                        !wait_or_abort(&b_full[slot], static_cast<uint32_t>((gs / kTcRing) & 1), args.err, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint32_t base = smem_u32(smem + slot * L.ring_bytes);
                    const uint32_t d = tmem + kDCol * ab;
                    const uint32_t a = tmem + kACol0 + 64u * ab;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint32_t ko = 32u * kk;  // 8 tf32 along K inside the 64-B row
                        const uint64_t duh = tc::sdesc_kmajor_sw64(base + 0 * L.tile_bytes + ko);
                        const uint64_t dul = tc::sdesc_kmajor_sw64(base + 1 * L.tile_bytes + ko);
                        const uint64_t dyh = tc::sdesc_kmajor_sw64(base + 2 * L.tile_bytes + ko);
                        const uint64_t dyl = tc::sdesc_kmajor_sw64(base + 3 * L.tile_bytes + ko);
                        const uint32_t ah = a + 0 + 8 * kk, al = a + 16 + 8 * kk;
                        const uint32_t bh = a + 32 + 8 * kk, bl = a + 48 + 8 * kk;
                        tc::mma_tf32_ts(d, ah, duh, idesc, kk);  // first MMA of the stage overwrites
                        tc::mma_tf32_ts(d, ah, dul, idesc, 1);
                        tc::mma_tf32_ts(d, al, duh, idesc, 1);
                        tc::mma_tf32_ts(d, bh, dyh, idesc, 1);
                        tc::mma_tf32_ts(d, bh, dyl, idesc, 1);
                        tc::mma_tf32_ts(d, bl, dyh, idesc, 1);
                    }
                    issued_any = true;
                    tc::commit(&mma_done[ab]);
                    tc::commit(&b_empty[slot]);
                }
            }
            if (issued_any) {  // every MMA finished before TMEM is released
                tc::commit(fin);
                mbar_wait(fin, 0, args.err);
            }
        }
    } else {
        // ------------------------------------------------------------ generators
        const int quad = warp & 3, half = warp >> 2;
        const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
        float acc[PH];
#pragma unroll
        for (int k = 0; k < PH; ++k) acc[k] = 0.0f;
        int64_t gs = 0;
        bool ok = true;

        auto drain = [&](int64_t st) -> bool {
            const int db = static_cast<int>(st & 1);
            const bool got = wait_or_abort(&mma_done[db], static_cast<uint32_t>((st >> 1) & 1), args.err, abort_flag);
            if (!__all_sync(0xffffffffu, got)) return false;  // warp-uniform exit
            tc::fence_after();
#pragma unroll
            for (int c = 0; c < PH / 16; ++c) {
                uint32_t r[16];
                tc::ld_x16(tmem + lane_off + kDCol * db + half * PH + 16 * c, r);
                tc::wait_ld();
#pragma unroll
                for (int k = 0; k < 16; ++k) acc[16 * c + k] += __uint_as_float(r[k]);
            }
            tc::fence_before();
            return true;
        };
        auto flush = [&](int kind, int64_t i) {
            if (i < P.nk) {
#pragma unroll
                for (int k = 0; k < PH; ++k) {
                    const int t = half * PH + k;
                    if (t < args.Pn) {
                        double* o = args.acc + ((static_cast<int64_t>(kind) * args.acc_P + args.t0 + t) * P.nk_pad + i);
                        *o += static_cast<double>(acc[k]);
                    }
                    acc[k] = 0.0f;
                }
            } else {
#pragma unroll
                for (int k = 0; k < PH; ++k) acc[k] = 0.0f;
            }
        };

        for (int64_t q = blockIdx.x; q < n_tiles && ok; q += gridDim.x) {
            const int kind = static_cast<int>(q & 1);
            const int64_t i = (q >> 1) * 128 + quad * 32 + lane;
            float xi = 0.f, yi = 0.f, zi = 0.f, oi = 1.f, ki = 1.f, pi_ = 0.f, qi = 0.f;
            if (i < P.nk) {
                const float4 a = P.r32a[i], b = P.r32b[i];
                xi = a.x; yi = a.y; zi = a.z; oi = b.x; ki = b.y; pi_ = b.z; qi = b.w;
            }
            for (int64_t s = 0; s < n_stage; ++s, ++gs) {
                const int slot = static_cast<int>(gs % kTcRing);
                const int ab = static_cast<int>(gs & 1);
                // operand buffer ab is free once the MMAs of stage gs-2 are done
                bool got = wait_or_abort(&b_full[slot], static_cast<uint32_t>((gs / kTcRing) & 1), args.err, abort_flag);
                got = got && wait_or_abort(&mma_done[ab], static_cast<uint32_t>(((gs >> 1) & 1) ^ 1), args.err, abort_flag);
                if (!__all_sync(0xffffffffu, got)) {  // warp-uniform exit
                    ok = false;
                    break;
                }
                tc::fence_after();  // the MMAs that read this operand buffer are complete
                const float4* recA = reinterpret_cast<const float4*>(smem + L.rec_off + slot * 512);
                const float4* recB = recA + 16;
                uint32_t ah[8], al[8], bh[8], bl[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int jj = half * 8 + k;
                    float ta, tb;
                    pair_tiles(kind, xi, yi, zi, oi, ki, pi_, qi, recA[jj], recB[jj], ta, tb);
                    ah[k] = tc::to_tf32(ta);
                    al[k] = __float_as_uint(ta - __uint_as_float(ah[k]));
                    bh[k] = tc::to_tf32(tb);
                    bl[k] = __float_as_uint(tb - __uint_as_float(bh[k]));
                }
                const uint32_t a = tmem + lane_off + kACol0 + 64u * ab + half * 8;
                tc::st_x8(a + 0, ah);
                tc::st_x8(a + 16, al);
                tc::st_x8(a + 32, bh);
                tc::st_x8(a + 48, bl);
                tc::wait_st();
                tc::fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&a_full[ab]);
                    mbar_arrive(&b_empty[slot]);
                }
                if (s > 0) {
                    if (!drain(gs - 1)) {
                        ok = false;
                        break;
                    }
                    if (s % args.flush == 0) flush(kind, i);
                }
            }
            if (!ok) break;
            if (!drain(gs - 1)) {
                ok = false;
                break;
            }
            flush(kind, i);
        }
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
    if (t < P) {
        a = static_cast<float>(u[o]);
        b = static_cast<float>(y[o]);
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

int hess_tc_ppad(int32_t P) {
    const int p = ((P + 31) / 32) * 32;
    return p < 32 ? 32 : p;
}

template <int PH>
static cudaError_t launch_tc_t(const CUtensorMap* maps, const TcArgs& a, int grid, cudaStream_t st) {
    const TcSmemLayout L = tc_layout(2 * PH);
    cudaError_t e = cudaFuncSetAttribute(k_hess_tc<PH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(L.total));
    if (e != cudaSuccess) return e;
    k_hess_tc<PH><<<grid, kTcThreads, L.total, st>>>(maps[0], maps[1], maps[2], maps[3], a);
    return cudaGetLastError();
}

// Contract the trials [t0, t0 + Pn) (Pn <= 192); split arrays have `rows` rows.
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
    a.P = p;
    a.Pn = Pn;
    a.t0 = t0;
    a.acc_P = acc_P;
    a.n_row_tiles = (p.nk + 127) / 128;
    a.flush = flush > 0 ? flush : 128;
    a.acc = acc;
    a.err = err;
    const int64_t n_tiles = 2 * a.n_row_tiles;
    const int grid = static_cast<int>(n_tiles < n_sm ? n_tiles : n_sm);
    switch (ppad / 2) {
        case 16: return launch_tc_t<16>(maps, a, grid, st);
        case 32: return launch_tc_t<32>(maps, a, grid, st);
        case 48: return launch_tc_t<48>(maps, a, grid, st);
        case 64: return launch_tc_t<64>(maps, a, grid, st);
        case 80: return launch_tc_t<80>(maps, a, grid, st);
        default: return launch_tc_t<96>(maps, a, grid, st);
    }
}

}  // namespace vv10
