// tcgen05 pass 1 of the BF16 form at large padded rank (RP in {256, 512}; Algorithm 1
// steps 2-5 and 10), as two kernels:
//
//   ratios    Z[o, s] = sum_r X[o, r] Y[s, r] once per (o-block, chunk of 128 values of s),
//             X resident in tensor memory (the A operand, RP / 2 columns), Y streamed
//             through a ring of 128-wide K-slices and V through a ring of half chunks
//             (both by TMA); the epilogue forms q = v / z and
//             qbar = q / z (one reciprocal) and writes both as bf16 rows Q[o][s], Qbar[o][s]
//             to a workspace (the operands GEMM2 / GEMM3 take in bf16 anyway);
//   contract  A[o, r] += sum_s Q[o, s] Yt[r, s] and B[o, r] += sum_s Qbar[o, s] Y2t[r, s]:
//             a plain GEMM over (A or B, pair of o-blocks, 256-wide r-block, split of s)
//             tiles, two 128 x 256 accumulators in tensor memory sharing each Yt (Y2t)
//             K-slice of 64 values of s, the Q (Qbar) slices of both o-blocks brought in by
//             TMA beside it, the accumulators written out per split as in the other pass-1
//             kernels ([split][R][O]).
//
// Against one fused kernel per r-block (which forms Z once per r-block of 128) this forms
// Z once, and each SM brings in about half the bytes per unit of useful work: the ratios
// kernel brings in Y (64 bytes per MAC row of 128) and V and writes Q, Qbar; the contract
// kernel brings in 64 KB per 64-value slice for 2 x 128 x 256 x 64 MACs.  The price is the
// Q, Qbar round trip through HBM (4 bytes per element of V, written once and read once per
// r-block, the second read mostly from L2).
//
// Every barrier wait is bounded (wait_phase) and aborts the CTA; after an abort the
// producer waits for its armed copies and each MMA-issuing thread for its MMAs before the
// CTA frees its tensor memory, and STATUS_TIMEOUT is reported.
#include <algorithm>
#include <cfloat>
#include <type_traits>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dna_internal.h"
#include "tc_common.cuh"

namespace dna {
namespace tc {
namespace mat {

constexpr int SC = 128;                      // values of s per chunk of the ratios kernel
constexpr int EPI = 16;                      // epilogue warps of the ratios kernel
constexpr int W_PROD_A = EPI, W_MMA_A = EPI + 1;
constexpr int A_THREADS = (EPI + 2) * 32;

template <int RP>
struct LayoutA {
    // a K-slice is 128 values of r: two [128 s][64 r] bf16 sub-tiles, 8 MMAs per wait /
    // commit pair of the issuing thread (each costs the tensor pipe a few hundred cycles)
    static constexpr int KST = 3, VST = 3;
    static constexpr uint32_t Y_SUB = SC * 64 * 2;       // [128 s][64 r] bf16
    static constexpr uint32_t Y_SLICE = 2 * Y_SUB;
    static constexpr uint32_t V_HALF = 64 * OBLK * 4;    // [64 s][128 o] float32
    static constexpr uint32_t VR = KST * Y_SLICE;
    static constexpr uint32_t BAR = VR + VST * V_HALF;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;
    static constexpr uint32_t TX = 0;                    // X: RP / 2 columns (bf16 pairs)
    static constexpr uint32_t TZ = RP / 2;               // two Z buffers of 128 columns
    static_assert(TZ + 2 * SC <= NCOLS, "tensor memory budget");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};
enum { A_KFULL = 0, A_KEMPTY = 3, A_VFULL = 6, A_QREADY = 9, A_XFULL = 12, A_ZFULL = 13,
       A_ZEMPTY = 15, A_DRAIN = 17, A_COUNT = 18 };

struct RatioArgs {
    int64_t S, O, s_per;       // s_per: a multiple of SC
    const float* V;            // V_so, element (s, o) at V[s * vs + o]
    int64_t vs;
    const bf16* X;             // [O_pad][rp]
    int64_t rp;
    bf16* Q;                   // [O_pad][ldq]
    bf16* Qb;
    int64_t ldq;
    int* status;
};

struct ATile {
    int64_t o0, s_begin;
    int nch;
};
__device__ __forceinline__ ATile a_tile(int t, int nsplit, const RatioArgs& a) {
    ATile x;
    x.o0 = (int64_t)(t / nsplit) * OBLK;
    x.s_begin = (int64_t)(t % nsplit) * a.s_per;
    const int64_t s_end = min(a.S, x.s_begin + a.s_per);
    x.nch = s_end > x.s_begin ? (int)((s_end - x.s_begin + SC - 1) / SC) : 0;
    return x;
}

constexpr int B_EPI = 8;                     // epilogue warps of the contract kernel
constexpr int W_PROD_B = B_EPI, W_MMA_B = B_EPI + 1;
constexpr int B_THREADS = (B_EPI + 2) * 32;
constexpr int RB = 256;                      // r per tile of the contract kernel

// A tile covers two o-blocks (M = 256 as two 128-row MMAs that share each Yt slice), one
// 256-wide r-block, one split of s and one accumulator kind (A, or B): shared-memory
// bytes per MAC are 2 (1/256 + 1/256), two thirds of what a 128 x 256 tile of both kinds
// takes, for the same tensor work.  Tensor memory holds the two 128 x 256 accumulators.
struct LayoutB {
    static constexpr int KST = 3;
    static constexpr uint32_t Q_TILE = OBLK * 64 * 2;    // [128 o][64 s]
    static constexpr uint32_t Y_TILE = RB * 64 * 2;      // [256 r][64 s]
    // Q (or Qbar) of the two o-blocks, then Yt (or Y2t)
    static constexpr uint32_t STAGE = 2 * Q_TILE + Y_TILE;
    static constexpr uint32_t BAR = KST * STAGE;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;               // o-block 0: 256 | o-block 1: 256
    static_assert(STAGE % 1024 == 0, "alignment");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};
enum { C_KFULL = 0, C_KEMPTY = 3, C_ACCFULL = 6, C_ACCEMPTY = 7, C_DRAIN = 8, C_COUNT = 9 };

struct ContractArgs {
    int64_t S, O, R, s_per;    // s_per: a multiple of 64
    float* Apart;              // [splits][R][O]
    float* Bpart;
};

struct BTile {
    int64_t o0, s_begin;       // o0: the first of the tile's two o-blocks
    int nsl, rb, split, which;
};
// tiles: which slowest, then the split, then the o-block pair, r-block fastest.  CTA i of
// G takes tiles i, i + G, i + 2 G, ..., so with G even the r-blocks of one (pair, split)
// run at the same time on CTAs i and i + 1 and the second read of each Q slice comes from
// L2 (CTAs running together also share the Yt slices of one split).  A contiguous range
// of tiles per CTA ran the r-blocks back to back instead, and at 2 MB of Q per tile the
// second read missed L2 behind the other CTAs' tiles.
__device__ __forceinline__ BTile b_tile(int t, int nop, int nrb, int nsplit,
                                        const ContractArgs& a) {
    BTile x;
    const int per_which = nrb * nop * nsplit;
    x.which = t / per_which;
    const int u = t % per_which;
    x.rb = u % nrb;
    const int rest = u / nrb;
    x.o0 = (int64_t)(rest % nop) * 2 * OBLK;
    x.split = rest / nop;
    x.s_begin = (int64_t)x.split * a.s_per;
    const int64_t s_end = min(a.S, x.s_begin + a.s_per);
    x.nsl = s_end > x.s_begin ? (int)((s_end - x.s_begin + 63) / 64) : 0;
    return x;
}

}  // namespace mat

// ---------------------------------------------------------------- ratios kernel
template <int RP, bool WITH_B>
__global__ void __launch_bounds__(mat::A_THREADS, 1)
    k_tc_ratios(mat::RatioArgs a, int nsplit, int ntiles, const __grid_constant__ CUtensorMap tmY,
                const __grid_constant__ CUtensorMap tmV, const __grid_constant__ CUtensorMap tmQ,
                const __grid_constant__ CUtensorMap tmQb) {
    using namespace mat;
    using L = LayoutA<RP>;
    constexpr int KST = L::KST, VST = L::VST, KS = RP / 128;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + A_COUNT * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L::BAR + A_COUNT * 8 + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t_begin = (int)((int64_t)blockIdx.x * ntiles / gridDim.x);
    const int t_end = (int)((int64_t)(blockIdx.x + 1) * ntiles / gridDim.x);

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == W_PROD_A * 32) {
        for (int i = 0; i < KST; ++i) {
            mbar_init(&bar[A_KFULL + i], 1);
            mbar_init(&bar[A_KEMPTY + i], 1);
        }
        for (int i = 0; i < VST; ++i) {
            mbar_init(&bar[A_VFULL + i], 1);
            mbar_init(&bar[A_QREADY + i], EPI);   // every epilogue warp wrote its Q part
        }
        mbar_init(&bar[A_XFULL], EPI);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar[A_ZFULL + i], 1);
            mbar_init(&bar[A_ZEMPTY + i], EPI);
        }
        mbar_init(&bar[A_DRAIN], 1);
        *abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == W_PROD_A) {
        // One thread services three queues in whatever order they allow progress: Y
        // K-slices [128 s][128 r] of every chunk (in the MMA thread's order); V half chunks
        // [64 s][128 o] (in the epilogue's order); and the stores of the Q, Qbar tiles the
        // epilogue writes over a V stage once it has read it.  A V stage takes its next
        // half chunk only after the stores out of it have finished reading it.
        if (lane == 0 && t_begin < t_end) {
            tma_prefetch_desc(&tmY);
            tma_prefetch_desc(&tmV);
            tma_prefetch_desc(&tmQ);
            if (WITH_B) tma_prefetch_desc(&tmQb);
            int ty = t_begin, ky = 0, sy = 0, kk = 0;     // Y cursor: tile, chunk, K-slice
            int tv = t_begin, kv = 0, hv = 0, jv = 0;     // V loads: tile, chunk, half
            int tq = t_begin, kq_ = 0, hq = 0, jq = 0;    // Q stores: tile, chunk, half
            ATile xy = a_tile(ty, nsplit, a), xv = xy, xq = xy;
            long long t0 = clock64();
            while (ty < t_end || tv < t_end || tq < t_end) {
                bool prog = false;
                if (ty < t_end && mbar_test(&bar[A_KEMPTY + kk % KST], ((kk / KST) & 1) ^ 1)) {
                    const int st = kk % KST;
                    const uint32_t dst = sbase + st * L::Y_SLICE;
                    const int32_t r0 = 128 * sy;
                    const int32_t s0 = (int32_t)(xy.s_begin + (int64_t)ky * SC);
                    mbar_arrive_expect_tx(&bar[A_KFULL + st], L::Y_SLICE);
#pragma unroll
                    for (int hs = 0; hs < 2; ++hs)     // sub-tile hs: r0 + 64 hs .. + 63, 128 s
                        tma_load_2d(dst + hs * L::Y_SUB, &tmY, r0 + 64 * hs, s0, &bar[A_KFULL + st]);
                    ++kk;
                    if (++sy == KS) {
                        sy = 0;
                        if (++ky == xy.nch) { ky = 0; if (++ty < t_end) xy = a_tile(ty, nsplit, a); }
                    }
                    prog = true;
                }
                // Q, Qbar tiles of half chunk jq, written by the epilogue into V stage jq % VST
                if (tq < t_end && jq < jv &&
                    mbar_test(&bar[A_QREADY + jq % VST], (jq / VST) & 1)) {
                    const uint32_t src = sbase + L::VR + (jq % VST) * L::V_HALF;
                    const int32_t s0 = (int32_t)(xq.s_begin + (int64_t)kq_ * SC + 64 * hq);
                    tma_store_2d(&tmQ, src, s0, (int32_t)xq.o0);
                    if (WITH_B) tma_store_2d(&tmQb, src + OBLK * 128u, s0, (int32_t)xq.o0);
                    bulk_commit();
                    ++jq;
                    if (++hq == 2) {
                        hq = 0;
                        if (++kq_ == xq.nch) { kq_ = 0; if (++tq < t_end) xq = a_tile(tq, nsplit, a); }
                    }
                    prog = true;
                }
                // V half chunk jv into stage jv % VST once the stores of half jv - VST, which
                // left from that stage, have been issued (and, below, have read it)
                if (tv < t_end && jv - jq < VST) {
                    if (jv >= VST) bulk_wait_read_all();
                    const int st = jv % VST;
                    const uint32_t dst = sbase + L::VR + st * L::V_HALF;
                    const int32_t s0 = (int32_t)(xv.s_begin + (int64_t)kv * SC + 64 * hv);
                    mbar_arrive_expect_tx(&bar[A_VFULL + st], L::V_HALF);
                    tma_load_2d(dst, &tmV, (int32_t)xv.o0, s0, &bar[A_VFULL + st]);
                    ++jv;
                    if (++hv == 2) {
                        hv = 0;
                        if (++kv == xv.nch) { kv = 0; if (++tv < t_end) xv = a_tile(tv, nsplit, a); }
                    }
                    prog = true;
                }
                if (prog) {
                    t0 = clock64();
                } else {
                    if (*abort) break;
                    if (clock64() - t0 > WAIT_LIMIT) { *abort = 1; break; }
                    __nanosleep(20);
                }
            }
            bulk_wait_all();   // the Q stores are complete before the CTA exits
            if (*abort) {      // let the copies already issued land before the CTA exits
                for (int k = max(0, kk - KST); k < kk; ++k)
                    drain_phase(&bar[A_KFULL + k % KST], (k / KST) & 1);
                for (int k = max(jq, jv - VST); k < jv; ++k)
                    drain_phase(&bar[A_VFULL + k % VST], (k / VST) & 1);
            }
        }
    } else if (warp == W_MMA_A) {
        // Z(m) = X Y(m)^t into buffer m & 1, X from tensor memory
        if (lane == 0) {
            bool ok = true;
            int m = 0, j = 0, nx = 0;
            constexpr uint32_t idesc = idesc_bf16(OBLK, SC);
            for (int t = t_begin; ok && t < t_end; ++t) {
                const ATile x = a_tile(t, nsplit, a);
                const int nch = x.nch;
                // a new o-block: the epilogue has written its X
                if (t == t_begin || a_tile(t - 1, nsplit, a).o0 != x.o0) {
                    if (!(ok = wait_phase(&bar[A_XFULL], nx & 1, abort))) break;
                    ++nx;
                }
                tc_fence_after();
                for (int k = 0; ok && k < nch; ++k, ++m) {
                    const int b = m & 1;
                    // the epilogue has read chunk m - 2 out of this buffer
                    if (m >= 2 &&
                        !(ok = wait_phase(&bar[A_ZEMPTY + b], ((m - 2) >> 1) & 1, abort)))
                        break;
                    tc_fence_after();
                    const uint32_t tz = tmem + L::TZ + b * SC;
#pragma unroll 1
                    for (int ks = 0; ks < KS; ++ks, ++j) {
                        if (!(ok = wait_phase(&bar[A_KFULL + j % KST], (j / KST) & 1, abort)))
                            break;
                        tc_fence_after();
                        const uint32_t ys = sbase + (j % KST) * L::Y_SLICE;
#pragma unroll
                        for (int kq = 0; kq < 8; ++kq)
                            mma_bf16_tmem_a(tz, tmem + L::TX + (uint32_t)(8 * ks + kq) * 8u,
                                            desc_sw128(ys + (kq >> 2) * L::Y_SUB + 32u * (kq & 3)),
                                            idesc, (ks > 0 || kq > 0) ? 1u : 0u);
                        mma_commit(&bar[A_KEMPTY + j % KST]);
                    }
                    if (ok) mma_commit(&bar[A_ZFULL + b]);
                }
            }
            if (!ok) {
                mma_commit(&bar[A_DRAIN]);
                drain_phase(&bar[A_DRAIN], 0);
            }
        }
    } else {
        // epilogue warps: lanes o = o0 + 32 qd + lane; in half h of a chunk the 16 values
        // s = 64 h + 16 cg .. + 15 of Z buffer columns 64 h + 16 cg .., their v from the
        // V ring (half chunk jv = 2 m + h: [64 s][128 o], lanes read consecutive o).  Once
        // every epilogue warp has read a V stage (a named barrier), the same 32 KB take the
        // half chunk's Q and Qbar tiles ([128 o][64 s] bf16 each, 128-byte swizzled), which
        // the producer thread stores with TMA (coalesced rows).  The waits' outcomes are
        // OR-ed over the epilogue warps at a named barrier, so all of them leave together on
        // an abort and none is left waiting at a barrier.
        constexpr uint32_t NB = 1, NT_EPI = EPI * 32;
        const int qd = warp & 3, cg = warp >> 2;
        const int row = 32 * qd + lane;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        float qbmax = 0.f;   // an infinite qbar: z = 0 where v > 0 (infinite cost)
        bool ok = true;
        int m = 0;
        for (int t = t_begin; ok && t < t_end; ++t) {
            const ATile x = a_tile(t, nsplit, a);
            const int64_t o = x.o0 + row;
            if (t == t_begin || a_tile(t - 1, nsplit, a).o0 != x.o0) {
                // a new o-block: its X rows into tensor memory (every GEMM1 of the previous
                // tile has completed: its last Z was read below)
                for (int unit = cg; unit < RP / 32; unit += 4)
                    x_to_tmem(a.X, a.rp, o, unit, tmem + L::TX + lane_off);
                tmem_st_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[A_XFULL]);
            }
            for (int k = 0; ok && k < x.nch; ++k, ++m) {
                const int b = m & 1;
                bool w_ok = wait_phase(&bar[A_ZFULL + b], (m >> 1) & 1, abort);
                tc_fence_after();
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    const int jv = 2 * m + h, sv = jv % VST;
                    w_ok = w_ok && wait_phase(&bar[A_VFULL + sv], (jv / VST) & 1, abort);
                    if (named_any(NB, NT_EPI, !w_ok)) { ok = false; break; }
                    uint32_t zr[16];
                    tmem_ld16(tmem + L::TZ + b * SC + 64 * h + 16 * cg + lane_off, zr);
                    unsigned char* stage = sm + L::VR + (size_t)sv * L::V_HALF;
                    const float* vh =
                        reinterpret_cast<const float*>(stage) + (16 * cg) * OBLK + row;
                    tmem_ld_wait();
                    // z >= 0 (products of non-negative operands); with v' = max(v, 0) and
                    // z' = max(z, FLT_MIN), q = v' / z' and qbar = q / z' are 0 where v = 0
                    // (the V ring holds zeros outside the problem) and equal v / z, v / z^2
                    // elsewhere, unless z = 0 where v > 0, which makes qbar infinite
                    uint32_t qp[8], qbp[8];
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        float q[2], qb[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const float v = fmaxf(vh[(j + u) * OBLK], 0.f);
                            const float z = fmaxf(__uint_as_float(zr[j + u]), FLT_MIN);
                            const float rz = rcp_ftz(z);
                            q[u] = v * rz;
                            qb[u] = q[u] * rz;
                            qbmax = fmaxf(qbmax, qb[u]);
                        }
                        qp[j / 2] = pack_bf16x2(q[0], q[1]);
                        qbp[j / 2] = pack_bf16x2(qb[0], qb[1]);
                    }
                    named_sync(NB, NT_EPI);     // every warp has read this V stage
                    // 16-byte chunks 2 cg and 2 cg + 1 of row `row` (128 bytes = 64 values of s)
                    const uint32_t q0 = smem_u32(stage);
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint32_t off = (uint32_t)row * 128u +
                                             ((((uint32_t)(2 * cg + c)) ^ ((uint32_t)row & 7u)) << 4);
                        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(q0 + off),
                                     "r"(qp[4 * c]), "r"(qp[4 * c + 1]), "r"(qp[4 * c + 2]),
                                     "r"(qp[4 * c + 3])
                                     : "memory");
                        if (WITH_B)
                            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                                             q0 + OBLK * 128u + off),
                                         "r"(qbp[4 * c]), "r"(qbp[4 * c + 1]), "r"(qbp[4 * c + 2]),
                                         "r"(qbp[4 * c + 3])
                                         : "memory");
                    }
                    fence_proxy_async_smem();   // visible to the TMA (async proxy)
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar[A_QREADY + sv]);
                }
                if (!ok) break;
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[A_ZEMPTY + b]);
            }
        }
        if (!(qbmax <= FLT_MAX)) atomicOr(a.status, STATUS_NONFINITE);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(a.status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

// ---------------------------------------------------------------- contract kernel
template <bool WITH_B>
__global__ void __launch_bounds__(mat::B_THREADS, 1)
    k_tc_contract(mat::ContractArgs a, int nob, int nop, int nrb, int nsplit, int ntiles,
                  int* status,
                  const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmQb,
                  const __grid_constant__ CUtensorMap tmYt,
                  const __grid_constant__ CUtensorMap tmY2t) {
    using namespace mat;
    using L = LayoutB;
    constexpr int KST = L::KST;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + C_COUNT * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L::BAR + C_COUNT * 8 + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // tiles blockIdx.x, + gridDim.x, ... (see b_tile)
    const int t_first = (int)blockIdx.x, t_step = (int)gridDim.x;

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == W_PROD_B * 32) {
        for (int i = 0; i < KST; ++i) {
            mbar_init(&bar[C_KFULL + i], 1);
            mbar_init(&bar[C_KEMPTY + i], 1);
        }
        mbar_init(&bar[C_ACCFULL], 1);
        mbar_init(&bar[C_ACCEMPTY], B_EPI);
        mbar_init(&bar[C_DRAIN], 1);
        *abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == W_PROD_B) {
        if (lane == 0 && t_first < ntiles) {
            tma_prefetch_desc(&tmQ); tma_prefetch_desc(&tmYt);
            if (WITH_B) { tma_prefetch_desc(&tmQb); tma_prefetch_desc(&tmY2t); }
            int kk = 0;
            bool ok = true;
            for (int t = t_first; ok && t < ntiles; t += t_step) {
                const BTile x = b_tile(t, nop, nrb, nsplit, a);
                const CUtensorMap* mq = x.which ? &tmQb : &tmQ;
                const CUtensorMap* my = x.which ? &tmY2t : &tmYt;
                // the pair's second o-block exists unless the o-block count is odd
                const bool two = x.o0 / OBLK + 1 < nob;
                for (int sl = 0; sl < x.nsl; ++sl, ++kk) {
                    const int st = kk % KST;
                    if (!(ok = wait_phase(&bar[C_KEMPTY + st], ((kk / KST) & 1) ^ 1, abort)))
                        break;
                    const uint32_t dst = sbase + st * L::STAGE;
                    const int32_t s0 = (int32_t)(x.s_begin + 64 * (int64_t)sl);
                    const int32_t r0 = RB * x.rb, o0 = (int32_t)x.o0;
                    uint64_t* fb = &bar[C_KFULL + st];
                    mbar_arrive_expect_tx(fb, L::STAGE - (two ? 0u : L::Q_TILE));
                    tma_load_2d(dst, mq, s0, o0, fb);                              // [128 o][64 s]
                    if (two) tma_load_2d(dst + L::Q_TILE, mq, s0, o0 + OBLK, fb);
                    tma_load_2d(dst + 2 * L::Q_TILE, my, s0, r0, fb);              // [256 r][64 s]
                }
            }
            if (*abort)
                for (int k = max(0, kk - KST); k < kk; ++k)
                    drain_phase(&bar[C_KFULL + k % KST], (k / KST) & 1);
        }
    } else if (warp == W_MMA_B) {
        if (lane == 0) {
            bool ok = true;
            int j = 0, tt = 0;
            constexpr uint32_t idesc = idesc_bf16(OBLK, RB);
            for (int t = t_first; ok && t < ntiles; t += t_step, ++tt) {
                const BTile x = b_tile(t, nop, nrb, nsplit, a);
                const int nsl = x.nsl;
                const bool two = x.o0 / OBLK + 1 < nob;
                // the epilogue has copied the previous tile's accumulators out
                if (tt > 0 && !(ok = wait_phase(&bar[C_ACCEMPTY], (tt - 1) & 1, abort))) break;
                tc_fence_after();
#pragma unroll 1
                for (int sl = 0; sl < nsl; ++sl, ++j) {
                    if (!(ok = wait_phase(&bar[C_KFULL + j % KST], (j / KST) & 1, abort))) break;
                    tc_fence_after();
                    const uint32_t q0 = sbase + (j % KST) * L::STAGE, q1 = q0 + L::Q_TILE;
                    const uint32_t ys = q0 + 2 * L::Q_TILE;
#pragma unroll
                    for (int kq = 0; kq < 4; ++kq) {
                        const uint32_t acc = (sl > 0 || kq > 0) ? 1u : 0u;
                        const uint64_t yd = desc_sw128(ys + 32u * kq);
                        mma_bf16(tmem, desc_sw128(q0 + 32u * kq), yd, idesc, acc);
                        if (two) mma_bf16(tmem + RB, desc_sw128(q1 + 32u * kq), yd, idesc, acc);
                    }
                    mma_commit(&bar[C_KEMPTY + j % KST]);
                }
                if (ok) mma_commit(&bar[C_ACCFULL]);
            }
            if (!ok) {
                mma_commit(&bar[C_DRAIN]);
                drain_phase(&bar[C_DRAIN], 0);
            }
        }
    } else {
        // epilogue warps: lane quadrant qd, o-block h of the pair; rows
        // o = o0 + 128 h + 32 qd + lane, the accumulator's 256 columns in eight loads
        const int qd = warp & 3, h = warp >> 2;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        int tt = 0;
        for (int t = t_first; t < ntiles; t += t_step, ++tt) {
            const BTile x = b_tile(t, nop, nrb, nsplit, a);
            bool ok = wait_phase(&bar[C_ACCFULL], tt & 1, abort);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const int64_t o = x.o0 + OBLK * h + 32 * qd + lane;
            if (WITH_B || x.which == 0) {
                float* dst = x.which ? a.Bpart : a.Apart;
                const int64_t base = (int64_t)x.split * a.R;
#pragma unroll 1
                for (int c = 0; c < RB / 32; ++c) {
                    uint32_t r32[32];
                    tmem_ld32(tmem + (uint32_t)(RB * h + 32 * c) + lane_off, r32);
                    tmem_ld_wait();
                    if (o < a.O)
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const int64_t r = (int64_t)RB * x.rb + 32 * c + i;
                            if (r < a.R) dst[(base + r) * a.O + o] = __uint_as_float(r32[i]);
                        }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[C_ACCEMPTY]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

// ---------------------------------------------------------------- launch
template <int RP, bool WITH_B>
int launch_mat(const TcOperands& op, const TcMaps& m, float* Apart, float* Bpart, int splits,
               int64_t s_per, int* status, cudaStream_t st) {
    using namespace mat;
    const int nob = (int)(op.O_pad / OBLK);
    if (nob == 0) return DNA_OK;
    // ratios: tiles (o-block, range of chunks), about four per SM
    const int64_t chunks = (op.S + SC - 1) / SC;
    const int64_t want = std::max<int64_t>(1, (4LL * std::max(op.ctas, 1) + nob - 1) / nob);
    const int64_t nsa = std::min<int64_t>(chunks, want);
    RatioArgs ra{};
    ra.S = op.S; ra.O = op.O;
    ra.s_per = (chunks + nsa - 1) / nsa * SC;
    const int splits_a = (int)((op.S + ra.s_per - 1) / ra.s_per);
    ra.V = op.V; ra.vs = op.vs;
    ra.X = static_cast<const bf16*>(op.Xk); ra.rp = RP;
    ra.Q = static_cast<bf16*>(op.Qg); ra.Qb = static_cast<bf16*>(op.Qbg); ra.ldq = op.ldq;
    ra.status = status;
    {
        const uint32_t smem = LayoutA<RP>::TOTAL + 1024;
        auto k = k_tc_ratios<RP, WITH_B>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return DNA_ERR_CUDA;
        const int ntiles = nob * splits_a;
        const int grid = op.ctas > 0 ? std::min(op.ctas, ntiles) : ntiles;
        k<<<grid, A_THREADS, smem, st>>>(ra, splits_a, ntiles, m.y128, m.v, m.q, m.qb);
        if (int e = after_launch()) return e;
    }
    ContractArgs ca{};
    ca.S = op.S; ca.O = op.O; ca.R = op.R; ca.s_per = s_per;
    ca.Apart = Apart; ca.Bpart = Bpart;
    const uint32_t smem = LayoutB::TOTAL + 1024;
    auto k = k_tc_contract<WITH_B>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    const int nop = (nob + 1) / 2, nrb = RP / RB;
    const int ntiles = (WITH_B ? 2 : 1) * nrb * nop * splits;
    const int grid = op.ctas > 0 ? std::min(op.ctas, ntiles) : ntiles;
    k<<<grid, B_THREADS, smem, st>>>(ca, nob, nop, nrb, splits, ntiles, status, m.q, m.qb,
                                     m.yt256, m.y2t256);
    return after_launch();
}

}  // namespace tc

int TcBf16::pass1_mat(const TcOperands& op, const TcMaps& maps, float* Apart, float* Bpart,
                      int splits, int64_t s_per, bool with_b, int* status, cudaStream_t st) {
    const int rp = rank_pad(op.R);
    if (!op.Qg || !op.Qbg || op.ldq % tc::mat::SC != 0 || s_per % 64 != 0) return DNA_ERR_ARG;
    if (splits != (int)((op.S + s_per - 1) / s_per)) return DNA_ERR_ARG;
    if (rp == 256)
        return with_b ? tc::launch_mat<256, true>(op, maps, Apart, Bpart, splits, s_per, status, st)
                      : tc::launch_mat<256, false>(op, maps, Apart, Bpart, splits, s_per, status, st);
    if (rp == 512)
        return with_b ? tc::launch_mat<512, true>(op, maps, Apart, Bpart, splits, s_per, status, st)
                      : tc::launch_mat<512, false>(op, maps, Apart, Bpart, splits, s_per, status, st);
    return DNA_ERR_UNSUPPORTED;
}

}  // namespace dna
