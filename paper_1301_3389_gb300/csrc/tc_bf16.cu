// tcgen05 tensor-core kernels of the DNA half-step, BF16 operands with FP32 accumulation
// in TMEM (the precision form): pass 1 for padded rank RP in {64, 128}.  Both passes at
// RP = 512, and pass 1 at RP = 256, are in tc_ks.cu; pass 2 at RP <= 256 is the balanced
// kernel of tc_split.cu, which takes the BF16 form with one operand plane.
//
// Pass 1 (Algorithm 1 steps 2-5 and 10), per CTA = 128 values of o (the TMEM lanes) and
// an s-range streamed in chunks of 64:
//   GEMM1  Z[o, s]  = sum_r X[o, r] Y[s, r]            M = 128, N = 64, K = RP
//   epilogue (16 warps; warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. 32 values of o,
//          and 16 chunk columns): z from TMEM, v from shared memory, q = v / z,
//          qbar = q / z (0 where v = 0), rounded to bf16 into tensor memory
//   GEMM2  A[o, r] += sum_s Q[o, s] Yt[r, s]           M = 128, N = RP, K = 64
//   GEMM3  B[o, r] += sum_s Qbar[o, s] Y2t[r, s]       (Y2t = (Y o Y)^t)
// A and B stay in TMEM for the whole s-range; Z and Q never reach global memory.
//
// The kernels are warp-specialised pipelines: a producer warp issues TMA copies into
// rings (V, Y, Y^t and (Y o Y)^t tiles), MMA-issuing warps (one thread each) issue the
// tcgen05 MMAs, the epilogue warps read Z from TMEM.  Z is double-buffered in TMEM so
// GEMM1 of the next chunk overlaps the epilogue of this one.  Every hand-off is an
// mbarrier; every wait is bounded and aborts the CTA (with DNA_ERR_TIMEOUT reported)
// instead of hanging.
#include <algorithm>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "dna_internal.h"
#include "tc_common.cuh"

namespace dna {
namespace tc {

// Pass 1.  Shared memory: V ring (4 x [64][128] fp32), Y ring (2 x [64][RP] bf16), Y^t /
// (Y o Y)^t ring (2 x 2 x [RP][64] bf16).  Tensor memory: Z x 2 | A | B | X | Q | Qbar.
template <int RP>
struct P1Layout {
    static constexpr int VST = 4, YST = 2, TST = 2;
    static constexpr uint32_t V_BYTES = SCH * OBLK * 4;
    static constexpr uint32_t Y_BYTES = SCH * RP * 2;
    static constexpr uint32_t YT_BYTES = RP * SCH * 2;
    static constexpr uint32_t T_STAGE = 2 * YT_BYTES;
    static constexpr uint32_t VR = 0;
    static constexpr uint32_t YR = VR + VST * V_BYTES;
    static constexpr uint32_t TR = YR + YST * Y_BYTES;
    static constexpr uint32_t BAR = TR + TST * T_STAGE;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;
    static constexpr uint32_t TA = 2 * SCH, TB = TA + RP, TX = TB + RP, TQ = TX + RP / 2,
                              TQB = TQ + SCH / 2;
    static_assert(TQB + SCH / 2 <= NCOLS, "tensor memory budget");
    static_assert(YR % 1024 == 0 && TR % 1024 == 0 && Y_BYTES % 1024 == 0 &&
                      YT_BYTES % 1024 == 0,
                  "tiles must be 1024-byte aligned");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};

// Barrier slots of pass 1.  ZFULL[b] (GEMM1 of chunk m done, m % 2 == b) also frees the
// Y stage of chunk m; QEMPTY[b] (GEMM2/3 of chunk m done) also frees its Y^t stage and,
// for the last chunk, marks A and B final.
enum { B_XFULL = 0, B_VFULL = 1, B_VEMPTY = 5, B_YFULL = 9, B_TFULL = 11, B_ZFULL = 13,
       B_ZEMPTY = 15, B_QFULL = 17, B_QEMPTY = 18, B_DRAIN = 20, B_COUNT = 22 };

// The tile (o-block bx, split by of s) of pass 1; the tensor maps may live in kernel
// parameters or in global memory (the grouped form keeps one set per problem there).
template <int RP, bool WITH_B>
__device__ __forceinline__ void pass1_body(const P1Args& a, int64_t bx, int64_t by,
                                           const CUtensorMap* tmY, const CUtensorMap* tmYt,
                                           const CUtensorMap* tmY2t, const CUtensorMap* tmV) {
    using L = P1Layout<RP>;
    constexpr int VST = L::VST, YST = L::YST, TST = L::TST;
    static_assert(YST == 2 && TST == 2, "stage reuse is signalled by the 2-deep commit barriers");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + B_COUNT * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L::BAR + B_COUNT * 8 + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t o0 = bx * OBLK;
    const int64_t s_begin = by * a.s_per;
    const int64_t s_end = min(a.S, s_begin + a.s_per);
    const int nch = s_end > s_begin ? (int)((s_end - s_begin + SCH - 1) / SCH) : 0;

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == W_PRODUCER * 32) {
        mbar_init(&bar[B_XFULL], W_EPI);
        for (int i = 0; i < VST; ++i) {
            mbar_init(&bar[B_VFULL + i], 1);
            mbar_init(&bar[B_VEMPTY + i], W_EPI);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar[B_YFULL + i], 1);
            mbar_init(&bar[B_TFULL + i], 1);
            mbar_init(&bar[B_ZFULL + i], 1);
            mbar_init(&bar[B_ZEMPTY + i], W_EPI);
            mbar_init(&bar[B_QEMPTY + i], 1);
            mbar_init(&bar[B_DRAIN + i], 1);
        }
        mbar_init(&bar[B_QFULL], W_EPI);
        *abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == W_PRODUCER) {
        // One thread services the three rings in whatever order their slots free up.
        if (lane == 0 && nch > 0) {
            tma_prefetch_desc(tmY); tma_prefetch_desc(tmYt); tma_prefetch_desc(tmY2t);
            tma_prefetch_desc(tmV);
            int kv = 0, ky = 0, kt = 0;
            long long t0 = clock64();
            while (kv < nch || ky < nch || kt < nch) {
                bool prog = false;
                if (kv < nch && mbar_test(&bar[B_VEMPTY + kv % VST], ((kv / VST) & 1) ^ 1)) {
                    const int st = kv % VST;
                    mbar_arrive_expect_tx(&bar[B_VFULL + st], L::V_BYTES);
                    tma_load_2d(sbase + L::VR + st * L::V_BYTES, tmV, (int32_t)o0,
                                (int32_t)(s_begin + (int64_t)kv * SCH), &bar[B_VFULL + st]);
                    ++kv;
                    prog = true;
                }
                // Y(ky) reuses the stage of chunk m = ky - 2, free once GEMM1(m) is done
                if (ky < nch && (ky < YST || mbar_test(&bar[B_ZFULL + (ky & 1)],
                                                       ((ky - 2) >> 1) & 1))) {
                    const int st = ky % YST;
                    const uint32_t dst = sbase + L::YR + st * L::Y_BYTES;
                    mbar_arrive_expect_tx(&bar[B_YFULL + st], L::Y_BYTES);
                    for (int at = 0; at < RP / 64; ++at)
                        tma_load_2d(dst + at * SCH * 128, tmY, 64 * at,
                                    (int32_t)(s_begin + (int64_t)ky * SCH), &bar[B_YFULL + st]);
                    ++ky;
                    prog = true;
                }
                // Y^t(kt) reuses the stage of chunk m = kt - 2, free once GEMM2/3(m) are done
                if (kt < nch && (kt < TST || mbar_test(&bar[B_QEMPTY + (kt & 1)],
                                                       ((kt - 2) >> 1) & 1))) {
                    const int st = kt % TST;
                    const uint32_t dst = sbase + L::TR + st * L::T_STAGE;
                    const int32_t s0 = (int32_t)(s_begin + (int64_t)kt * SCH);
                    mbar_arrive_expect_tx(&bar[B_TFULL + st], (WITH_B ? 2 : 1) * L::YT_BYTES);
                    tma_load_2d(dst, tmYt, s0, 0, &bar[B_TFULL + st]);
                    if (WITH_B) tma_load_2d(dst + L::YT_BYTES, tmY2t, s0, 0, &bar[B_TFULL + st]);
                    ++kt;
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
            if (*abort) {  // let the copies already issued land before the CTA exits
                for (int k = max(0, kv - VST); k < kv; ++k)
                    drain_phase(&bar[B_VFULL + k % VST], (k / VST) & 1);
                for (int k = max(0, ky - YST); k < ky; ++k)
                    drain_phase(&bar[B_YFULL + k % YST], (k / YST) & 1);
                for (int k = max(0, kt - TST); k < kt; ++k)
                    drain_phase(&bar[B_TFULL + k % TST], (k / TST) & 1);
            }
        }
    } else if (warp == W_MMA_Z) {
        // GEMM1 of every chunk m into Z buffer m & 1, A = X in TMEM
        if (lane == 0 && nch > 0) {
            bool ok = wait_phase(&bar[B_XFULL], 0, abort);
            for (int m = 0; ok && m < nch; ++m) {
                const int zb = m & 1;
                if (!(ok = wait_phase(&bar[B_YFULL + m % YST], (m / YST) & 1, abort))) break;
                if (m >= 2 &&
                    !(ok = wait_phase(&bar[B_ZEMPTY + zb], ((m >> 1) & 1) ^ 1, abort)))
                    break;
                tc_fence_after();
                const uint32_t yb = sbase + L::YR + (m % YST) * L::Y_BYTES;
#pragma unroll
                for (int kk = 0; kk < RP / 16; ++kk) {
                    const uint32_t kb = 32u * kk, at = kb >> 7, within = kb & 127u;
                    mma_bf16_tmem_a(tmem + zb * SCH, tmem + L::TX + 8 * kk,
                                    desc_sw128(yb + at * SCH * 128 + within),
                                    idesc_bf16(OBLK, SCH), kk > 0);
                }
                mma_commit(&bar[B_ZFULL + zb]);
            }
            if (!ok) {  // no MMA of this thread may still be writing TMEM when it is released
                mma_commit(&bar[B_DRAIN + 0]);
                drain_phase(&bar[B_DRAIN + 0], 0);
            }
        }
    } else if (warp == W_MMA_AB) {
        // GEMM2 / GEMM3 of every chunk m, A = Q / Qbar in TMEM
        if (lane == 0 && nch > 0) {
            bool ok = true;
            for (int m = 0; ok && m < nch; ++m) {
                if (!(ok = wait_phase(&bar[B_QFULL], m & 1, abort))) break;
                if (!(ok = wait_phase(&bar[B_TFULL + m % TST], (m / TST) & 1, abort))) break;
                tc_fence_after();
                const uint32_t tb = sbase + L::TR + (m % TST) * L::T_STAGE;
#pragma unroll
                for (int kk = 0; kk < SCH / 16; ++kk) {
                    const uint32_t acc = (m > 0 || kk > 0) ? 1u : 0u;
                    mma_bf16_tmem_a(tmem + L::TA, tmem + L::TQ + 8 * kk,
                                    desc_sw128(tb + 32u * kk), idesc_bf16(OBLK, RP), acc);
                    if (WITH_B)
                        mma_bf16_tmem_a(tmem + L::TB, tmem + L::TQB + 8 * kk,
                                        desc_sw128(tb + L::YT_BYTES + 32u * kk),
                                        idesc_bf16(OBLK, RP), acc);
                }
                mma_commit(&bar[B_QEMPTY + (m & 1)]);
            }
            if (!ok) {
                mma_commit(&bar[B_DRAIN + 1]);
                drain_phase(&bar[B_DRAIN + 1], 0);
            }
        }
    } else {
        // epilogue warps 0-15: lane quadrant qd = warp % 4 (o = o0 + 32 qd + lane), chunk
        // columns 16 cg .. 16 cg + 15 with cg = warp / 4
        const int qd = warp & 3, cg = warp >> 2;
        const int row = 32 * qd + lane;
        const int64_t o = o0 + row;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        if (nch > 0) {   // X of this o-block into tensor memory (GEMM1's A operand)
            for (int u = cg; u < RP / 32; u += 4)
                x_to_tmem(static_cast<const bf16*>(a.X), a.rp, o, u, tmem + L::TX + lane_off);
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[B_XFULL]);
        }
        // min over v > 0 of z: a z there below the smallest normal float (read as 0 by the
        // reciprocal) is an infinite cost (a NaN z makes NaN candidates, which pass 2
        // reports)
        float zmin = 1.f;
        bool ok = true;
        for (int k = 0; k < nch; ++k) {
            const int zb = k & 1, vs = k % VST;
            ok = wait_phase(&bar[B_ZFULL + zb], (k >> 1) & 1, abort);
            ok = ok && wait_phase(&bar[B_VFULL + vs], (k / VST) & 1, abort);
            if (!(ok = __all_sync(0xffffffffu, ok))) break;   // keep the warp converged
            tc_fence_after();
            uint32_t zr[16];
            tmem_ld16(tmem + zb * SCH + lane_off + 16 * cg, zr);
            // V rows s = 16 cg + j of this stage; TMA zero-fills v outside the problem
            const float* Vs = reinterpret_cast<const float*>(sm + L::VR + vs * L::V_BYTES) +
                              16 * cg * OBLK + row;
            float vv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) vv[j] = Vs[j * OBLK];
            tmem_ld_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[B_ZEMPTY + zb]);
            uint32_t qp[8], qbp[8];
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                float q[2], qb[2];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const float v = vv[j + t];
                    const float z = __uint_as_float(zr[j + t]);
                    const float rz = rcp_ftz(z);
                    const bool pos = v > 0.f;
                    zmin = fminf(zmin, pos ? z : 1.f);
                    q[t] = pos ? v * rz : 0.f;
                    qb[t] = pos ? q[t] * rz : 0.f;
                }
                qp[j / 2] = pack_bf16x2(q[0], q[1]);
                qbp[j / 2] = pack_bf16x2(qb[0], qb[1]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[B_VEMPTY + vs]);   // v of this stage consumed
            if (k >= 1) {   // GEMM2/3 of chunk k - 1 have read the Q buffer
                const int kp = k - 1;
                ok = wait_phase(&bar[B_QEMPTY + (kp & 1)], (kp >> 1) & 1, abort);
                if (!(ok = __all_sync(0xffffffffu, ok))) break;
                tc_fence_after();
            }
            tmem_st8(tmem + L::TQ + 8 * cg + lane_off, qp);
            if (WITH_B) tmem_st8(tmem + L::TQB + 8 * cg + lane_off, qbp);
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[B_QFULL]);
        }
        if (!(zmin >= FLT_MIN_NORMAL)) atomicOr(a.status, STATUS_NONFINITE);
        if (ok && nch > 0) {   // GEMM2/3 of the last chunk done: A and B are final
            const int kl = nch - 1;
            ok = __all_sync(0xffffffffu,
                            wait_phase(&bar[B_QEMPTY + (kl & 1)], (kl >> 1) & 1, abort));
        }
        if (ok && nch > 0) {
            tc_fence_after();
            const int64_t base = by * a.R;
            constexpr int G = RP / 32;   // 32-column groups of A (then of B)
#pragma unroll 1
            for (int u = cg; u < (WITH_B ? 2 : 1) * G; u += 4) {
                const bool isb = u >= G;
                const int g = isb ? u - G : u;
                uint32_t r32[32];
                tmem_ld32(tmem + (isb ? L::TB : L::TA) + lane_off + 32 * g, r32);
                tmem_ld_wait();
                float* dst = isb ? a.Bpart : a.Apart;
                if (o < a.O)
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int64_t r = 32 * g + i;
                        if (r < a.R) dst[(base + r) * a.O + o] = __uint_as_float(r32[i]);
                    }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(a.status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

template <int RP, bool WITH_B>
__global__ void __launch_bounds__(P1_THREADS, 1)
    k_tc_pass1(P1Args a, const __grid_constant__ CUtensorMap tmY,
               const __grid_constant__ CUtensorMap tmYt, const __grid_constant__ CUtensorMap tmY2t,
               const __grid_constant__ CUtensorMap tmV) {
    pass1_body<RP, WITH_B>(a, blockIdx.x, blockIdx.y, &tmY, &tmYt, &tmY2t, &tmV);
}

// Persistent grouped pass 1 (padded rank 64): CTA i runs tiles i, i + G, i + 2G, ... of
// the list (problem, o-block, split) (G CTAs; the host sorts the list longest first), with
// the rings, the Z and Q buffers and every barrier phase running on across tiles, so a
// tile's start (its X into tensor memory, the first copies) overlaps the previous tile's
// last chunks.  Per tile the epilogue loads the next tile's X once it has read the last Z
// of this one (GEMM1 no longer reads X), then drains A and B once the last GEMM2/3 is done
// and releases them (ACCEMPTY) for the next tile's first GEMM2/3.  The chunk work is that
// of pass1_body, with Q and Qbar double-buffered in tensor memory.
struct GP1Tile {
    const TcGView* v;
    int64_t o0, s_begin, split;
    int nch;
};
__device__ __forceinline__ GP1Tile gp1_tile(const TcGView* gv, const int4* tiles, int ti,
                                            int w) {
    const int4 t = tiles[ti];
    GP1Tile x;
    x.v = &gv[2 * t.x + w];
    x.o0 = (int64_t)t.y * OBLK;
    x.split = t.z;
    x.s_begin = x.split * x.v->s_per1;
    const int64_t s_end = min(x.v->S, x.s_begin + x.v->s_per1);
    x.nch = s_end > x.s_begin ? (int)((s_end - x.s_begin + SCH - 1) / SCH) : 0;
    return x;
}

template <bool WITH_B>
__global__ void __launch_bounds__(P1_THREADS, 1)
    k_tc_gpass1p(const TcGView* __restrict__ gv, const int4* __restrict__ tiles, int n, int w,
                 int* status) {
    constexpr int RP = 64;
    using L = P1Layout<RP>;
    constexpr int VST = L::VST, YST = L::YST, TST = L::TST;
    // two Q / Qbar buffers in tensor memory (chunk g uses buffer g & 1), each with its own
    // QFULL barrier, so the epilogue writes chunk g + 1's Q while GEMM2/3 read chunk g's
    constexpr int B_ACCEMPTY = B_COUNT, B_QFULL1 = B_COUNT + 1, NBAR = B_COUNT + 2;
    static_assert(NBAR * 8 + 16 <= 256, "barrier area");
    constexpr uint32_t TQ2 = L::TQB + SCH / 2;   // second Q buffer, then second Qbar buffer
    static_assert(TQ2 + SCH <= L::NCOLS, "tensor memory budget");
    auto tq = [](int b) { return b ? TQ2 : L::TQ; };
    auto tqb = [](int b) { return b ? TQ2 + SCH / 2 : L::TQB; };
    auto qfull = [](int b) { return b ? B_QFULL1 : B_QFULL; };
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + NBAR * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L::BAR + NBAR * 8 + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = (int)gridDim.x, t0 = (int)blockIdx.x;   // tiles t0, t0 + G, ...

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == W_PRODUCER * 32) {
        mbar_init(&bar[B_XFULL], W_EPI);
        mbar_init(&bar[B_ACCEMPTY], W_EPI);
        for (int i = 0; i < VST; ++i) {
            mbar_init(&bar[B_VFULL + i], 1);
            mbar_init(&bar[B_VEMPTY + i], W_EPI);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar[B_YFULL + i], 1);
            mbar_init(&bar[B_TFULL + i], 1);
            mbar_init(&bar[B_ZFULL + i], 1);
            mbar_init(&bar[B_ZEMPTY + i], W_EPI);
            mbar_init(&bar[B_QEMPTY + i], 1);
            mbar_init(&bar[B_DRAIN + i], 1);
        }
        mbar_init(&bar[B_QFULL], W_EPI);
        mbar_init(&bar[B_QFULL1], W_EPI);
        *abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == W_PRODUCER) {
        // three ring cursors, each over (tile, chunk) of this CTA's tiles
        if (lane == 0 && t0 < n) {
            struct Cur {
                int ti, k, g;
                GP1Tile x;
            };
            auto start = [&](Cur& c) {
                c.ti = t0; c.k = 0; c.g = 0;
                c.x = gp1_tile(gv, tiles, c.ti, w);
            };
            auto next = [&](Cur& c) {
                ++c.g;
                if (++c.k < c.x.nch) return;
                c.k = 0;
                c.ti += G;
                if (c.ti < n) c.x = gp1_tile(gv, tiles, c.ti, w);
            };
            Cur cv, cy, ct;
            start(cv); start(cy); start(ct);
            long long tw = clock64();
            while (cv.ti < n || cy.ti < n || ct.ti < n) {
                bool prog = false;
                if (cv.ti < n && mbar_test(&bar[B_VEMPTY + cv.g % VST], ((cv.g / VST) & 1) ^ 1)) {
                    const int st = cv.g % VST;
                    mbar_arrive_expect_tx(&bar[B_VFULL + st], L::V_BYTES);
                    tma_load_2d(sbase + L::VR + st * L::V_BYTES, &cv.x.v->v, (int32_t)cv.x.o0,
                                (int32_t)(cv.x.s_begin + (int64_t)cv.k * SCH), &bar[B_VFULL + st]);
                    next(cv);
                    prog = true;
                }
                // Y(g) reuses the stage of chunk g - 2, free once its GEMM1 is done
                if (cy.ti < n && (cy.g < YST || mbar_test(&bar[B_ZFULL + (cy.g & 1)],
                                                          ((cy.g - 2) >> 1) & 1))) {
                    const int st = cy.g % YST;
                    const uint32_t dst = sbase + L::YR + st * L::Y_BYTES;
                    mbar_arrive_expect_tx(&bar[B_YFULL + st], L::Y_BYTES);
                    tma_load_2d(dst, &cy.x.v->y, 0, (int32_t)(cy.x.s_begin + (int64_t)cy.k * SCH),
                                &bar[B_YFULL + st]);
                    next(cy);
                    prog = true;
                }
                // Y^t(g) reuses the stage of chunk g - 2, free once its GEMM2/3 are done
                if (ct.ti < n && (ct.g < TST || mbar_test(&bar[B_QEMPTY + (ct.g & 1)],
                                                          ((ct.g - 2) >> 1) & 1))) {
                    const int st = ct.g % TST;
                    const uint32_t dst = sbase + L::TR + st * L::T_STAGE;
                    const int32_t s0 = (int32_t)(ct.x.s_begin + (int64_t)ct.k * SCH);
                    mbar_arrive_expect_tx(&bar[B_TFULL + st], (WITH_B ? 2 : 1) * L::YT_BYTES);
                    tma_load_2d(dst, &ct.x.v->yt, s0, 0, &bar[B_TFULL + st]);
                    if (WITH_B) tma_load_2d(dst + L::YT_BYTES, &ct.x.v->y2t, s0, 0, &bar[B_TFULL + st]);
                    next(ct);
                    prog = true;
                }
                if (prog) {
                    tw = clock64();
                } else {
                    if (*abort) break;
                    if (clock64() - tw > WAIT_LIMIT) { *abort = 1; break; }
                    __nanosleep(20);
                }
            }
            if (*abort) {  // let the copies already issued land before the CTA exits
                for (int k = max(0, cv.g - VST); k < cv.g; ++k)
                    drain_phase(&bar[B_VFULL + k % VST], (k / VST) & 1);
                for (int k = max(0, cy.g - YST); k < cy.g; ++k)
                    drain_phase(&bar[B_YFULL + k % YST], (k / YST) & 1);
                for (int k = max(0, ct.g - TST); k < ct.g; ++k)
                    drain_phase(&bar[B_TFULL + k % TST], (k / TST) & 1);
            }
        }
    } else if (warp == W_MMA_Z) {
        // GEMM1 of every chunk (global index m) into Z buffer m & 1, A = the tile's X
        if (lane == 0 && t0 < n) {
            bool ok = true;
            int m = 0, j = 0;
            for (int ti = t0; ok && ti < n; ti += G, ++j) {
                const int nch = gp1_tile(gv, tiles, ti, w).nch;
                if (!(ok = wait_phase(&bar[B_XFULL], j & 1, abort))) break;
                for (int k = 0; ok && k < nch; ++k, ++m) {
                    const int zb = m & 1;
                    if (!(ok = wait_phase(&bar[B_YFULL + m % YST], (m / YST) & 1, abort))) break;
                    if (m >= 2 &&
                        !(ok = wait_phase(&bar[B_ZEMPTY + zb], ((m >> 1) & 1) ^ 1, abort)))
                        break;
                    tc_fence_after();
                    const uint32_t yb = sbase + L::YR + (m % YST) * L::Y_BYTES;
#pragma unroll
                    for (int kk = 0; kk < RP / 16; ++kk)
                        mma_bf16_tmem_a(tmem + zb * SCH, tmem + L::TX + 8 * kk,
                                        desc_sw128(yb + 32u * kk), idesc_bf16(OBLK, SCH), kk > 0);
                    mma_commit(&bar[B_ZFULL + zb]);
                }
            }
            if (!ok) {
                mma_commit(&bar[B_DRAIN + 0]);
                drain_phase(&bar[B_DRAIN + 0], 0);
            }
        }
    } else if (warp == W_MMA_AB) {
        // GEMM2 / GEMM3 of every chunk; a tile's first overwrites A and B once the
        // epilogue has drained the previous tile's
        if (lane == 0 && t0 < n) {
            bool ok = true;
            int m = 0, j = 0;
            for (int ti = t0; ok && ti < n; ti += G, ++j) {
                const int nch = gp1_tile(gv, tiles, ti, w).nch;
                if (j > 0 && !(ok = wait_phase(&bar[B_ACCEMPTY], (j - 1) & 1, abort))) break;
                for (int k = 0; ok && k < nch; ++k, ++m) {
                    const int qb = m & 1;
                    if (!(ok = wait_phase(&bar[qfull(qb)], (m >> 1) & 1, abort))) break;
                    if (!(ok = wait_phase(&bar[B_TFULL + m % TST], (m / TST) & 1, abort))) break;
                    tc_fence_after();
                    const uint32_t tb = sbase + L::TR + (m % TST) * L::T_STAGE;
#pragma unroll
                    for (int kk = 0; kk < SCH / 16; ++kk) {
                        const uint32_t acc = (k > 0 || kk > 0) ? 1u : 0u;
                        mma_bf16_tmem_a(tmem + L::TA, tmem + tq(qb) + 8 * kk,
                                        desc_sw128(tb + 32u * kk), idesc_bf16(OBLK, RP), acc);
                        if (WITH_B)
                            mma_bf16_tmem_a(tmem + L::TB, tmem + tqb(qb) + 8 * kk,
                                            desc_sw128(tb + L::YT_BYTES + 32u * kk),
                                            idesc_bf16(OBLK, RP), acc);
                    }
                    mma_commit(&bar[B_QEMPTY + (m & 1)]);
                }
            }
            if (!ok) {
                mma_commit(&bar[B_DRAIN + 1]);
                drain_phase(&bar[B_DRAIN + 1], 0);
            }
        }
    } else {
        // epilogue warps 0-15: lane quadrant qd = warp % 4, chunk columns 16 cg .. + 15
        const int qd = warp & 3, cg = warp >> 2;
        const int row = 32 * qd + lane;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        auto load_x = [&](const GP1Tile& x) {   // the tile's X into tensor memory
            for (int u = cg; u < RP / 32; u += 4)
                x_to_tmem(static_cast<const bf16*>(x.v->Xk), RP, x.o0 + row, u,
                          tmem + L::TX + lane_off);
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[B_XFULL]);
        };
        float zmin = 1.f;
        bool ok = true;
        int g = 0;   // global chunk index
        GP1Tile x = {};
        if (t0 < n) {
            x = gp1_tile(gv, tiles, t0, w);
            load_x(x);
        }
        for (int ti = t0; ok && ti < n; ti += G) {
            const int64_t o = x.o0 + row;
            for (int k = 0; k < x.nch; ++k, ++g) {
                const int zb = g & 1, vs = g % VST;
                ok = wait_phase(&bar[B_ZFULL + zb], (g >> 1) & 1, abort);
                ok = ok && wait_phase(&bar[B_VFULL + vs], (g / VST) & 1, abort);
                if (!(ok = __all_sync(0xffffffffu, ok))) break;
                tc_fence_after();
                uint32_t zr[16];
                tmem_ld16(tmem + zb * SCH + lane_off + 16 * cg, zr);
                const float* Vs = reinterpret_cast<const float*>(sm + L::VR + vs * L::V_BYTES) +
                                  16 * cg * OBLK + row;
                float vv[16];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) vv[jj] = Vs[jj * OBLK];
                tmem_ld_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[B_ZEMPTY + zb]);
                uint32_t qp[8], qbp[8];
#pragma unroll
                for (int jj = 0; jj < 16; jj += 2) {
                    float q[2], qb[2];
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const float v = vv[jj + t];
                        const float z = __uint_as_float(zr[jj + t]);
                        const float rz = rcp_ftz(z);
                        const bool pos = v > 0.f;
                        zmin = fminf(zmin, pos ? z : 1.f);
                        q[t] = pos ? v * rz : 0.f;
                        qb[t] = pos ? q[t] * rz : 0.f;
                    }
                    qp[jj / 2] = pack_bf16x2(q[0], q[1]);
                    qbp[jj / 2] = pack_bf16x2(qb[0], qb[1]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[B_VEMPTY + vs]);
                const int qb = g & 1;
                if (g >= 2) {   // GEMM2/3 of chunk g - 2 have read Q buffer g & 1
                    const int gp = g - 2;
                    ok = wait_phase(&bar[B_QEMPTY + qb], (gp >> 1) & 1, abort);
                    if (!(ok = __all_sync(0xffffffffu, ok))) break;
                    tc_fence_after();
                }
                tmem_st8(tmem + tq(qb) + 8 * cg + lane_off, qp);
                if (WITH_B) tmem_st8(tmem + tqb(qb) + 8 * cg + lane_off, qbp);
                tmem_st_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[qfull(qb)]);
            }
            if (!ok) break;
            // every Z of this tile has been read, so GEMM1 is done with X: the next tile's
            // X goes in now, while the last GEMM2/3 of this one runs
            const GP1Tile cur = x;
            if (ti + G < n) {
                x = gp1_tile(gv, tiles, ti + G, w);
                load_x(x);
            }
            if (cur.nch > 0) {   // GEMM2/3 of the last chunk done: A and B are final
                const int gl = g - 1;
                ok = __all_sync(0xffffffffu,
                                wait_phase(&bar[B_QEMPTY + (gl & 1)], (gl >> 1) & 1, abort));
                if (!ok) break;
                tc_fence_after();
                const TcGView& v = *cur.v;
                const int64_t base = cur.split * v.R;
                constexpr int GR = RP / 32;
#pragma unroll 1
                for (int u = cg; u < (WITH_B ? 2 : 1) * GR; u += 4) {
                    const bool isb = u >= GR;
                    const int gg = isb ? u - GR : u;
                    uint32_t r32[32];
                    tmem_ld32(tmem + (isb ? L::TB : L::TA) + lane_off + 32 * gg, r32);
                    tmem_ld_wait();
                    float* dst = isb ? v.B : v.A;
                    if (o < v.O)
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const int64_t r = 32 * gg + i;
                            if (r < v.R) dst[(base + r) * v.O + o] = __uint_as_float(r32[i]);
                        }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[B_ACCEMPTY]);
        }
        if (!(zmin >= FLT_MIN_NORMAL)) atomicOr(status, STATUS_NONFINITE);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

// dst[i][j] (leading dimension ld, padded to rows_pad x cols_pad with zeros) =
// bf16(src(i, j)) (squared first when `square`), where src(i, j) = src[i * si + j * sj]
// for i < rows, j < cols, and one of si, sj is 1.  32 x 32 tiles through shared memory.
__device__ __forceinline__ void to_bf16_tile(const float* __restrict__ src, int64_t si, int64_t sj,
                                             int64_t rows, int64_t cols, bf16* __restrict__ dst,
                                             int64_t ld, bool square, int64_t bx, int64_t by) {
    __shared__ float tile[32][33];
    const int64_t i0 = by * 32, j0 = bx * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (sj == 1) {
        for (int k = ty; k < 32; k += 8) {
            const int64_t i = i0 + k, j = j0 + tx;
            tile[k][tx] = (i < rows && j < cols) ? src[i * si + j] : 0.f;
        }
    } else {
        for (int k = ty; k < 32; k += 8) {
            const int64_t j = j0 + k, i = i0 + tx;
            tile[tx][k] = (i < rows && j < cols) ? src[i * si + j * sj] : 0.f;
        }
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int64_t i = i0 + k, j = j0 + tx;
        float x = tile[k][tx];
        if (square) x = x * x;
        dst[i * ld + j] = __float2bfloat16_rn(x);
    }
}
__global__ void k_to_bf16(const float* __restrict__ src, int64_t si, int64_t sj, int64_t rows,
                          int64_t cols, bf16* __restrict__ dst, int64_t ld, bool square) {
    to_bf16_tile(src, si, sj, rows, cols, dst, ld, square, blockIdx.x, blockIdx.y);
}

// The three operands derived from Y in one pass over a 32 x 32 tile of y(s, r):
//   Yk[s][r] = bf16(y), Ytk[r][s] = bf16(y), Y2tk[r][s] = bf16(y * y), zero-padded.
// y(s, r) at Y[s * ys + r * yr] with ys == 1 or yr == 1.  Grid covers S_pad x RP.
__device__ __forceinline__ void y_operands_tile(const float* __restrict__ Y, int64_t ys, int64_t yr,
                                                int64_t S, int64_t R, bf16* __restrict__ Yk,
                                                int64_t rp, bf16* __restrict__ Ytk,
                                                bf16* __restrict__ Y2tk, int64_t s_pad,
                                                bool with_sq, int64_t bx, int64_t by) {
    __shared__ float tile[32][33];   // tile[s][r]
    const int64_t s0 = bx * 32, r0 = by * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (yr == 1) {   // rows of Y contiguous along r
        for (int k = ty; k < 32; k += 8) {
            const int64_t s = s0 + k, r = r0 + tx;
            tile[k][tx] = (s < S && r < R) ? Y[s * ys + r] : 0.f;
        }
    } else {         // contiguous along s
        for (int k = ty; k < 32; k += 8) {
            const int64_t r = r0 + k, s = s0 + tx;
            tile[tx][k] = (s < S && r < R) ? Y[s + r * yr] : 0.f;
        }
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int64_t s = s0 + k, r = r0 + tx;     // Yk: r fastest
        Yk[s * rp + r] = __float2bfloat16_rn(tile[k][tx]);
        const int64_t r2 = r0 + k, s2 = s0 + tx;   // Ytk, Y2tk: s fastest
        const float y = tile[tx][k];
        Ytk[r2 * s_pad + s2] = __float2bfloat16_rn(y);
        if (with_sq) Y2tk[r2 * s_pad + s2] = __float2bfloat16_rn(y * y);
    }
}
__global__ void k_y_operands(const float* __restrict__ Y, int64_t ys, int64_t yr, int64_t S,
                             int64_t R, bf16* __restrict__ Yk, int64_t rp,
                             bf16* __restrict__ Ytk, bf16* __restrict__ Y2tk, int64_t s_pad,
                             bool with_sq) {
    y_operands_tile(Y, ys, yr, S, R, Yk, rp, Ytk, Y2tk, s_pad, with_sq, blockIdx.x, blockIdx.y);
}

// Grouped bf16 operands of view w, one 64 x 64 tile per CTA step: tiles[t] = (problem,
// what, block, -), what = 0: X -> Xk [O_pad][64] rows o of the block (x(r, o) at
// X[r xr + o xo]); what = 1: Y -> Yk [S_pad][64], Ytk and Y2tk [64][S_pad] for the block's
// 64 values of s (y(s, r) at Y[s ys + r yr]).  The tile is read along the matrix's
// contiguous index and written as bf16 pairs, 128 bytes per row and warp; entries past R
// or past O (S) are zeros.  CTA = 32 x 8 threads.
__global__ void __launch_bounds__(256)
    k_g_operands(const TcGView* __restrict__ gv, const int4* __restrict__ tiles, int n, int w) {
    __shared__ float tile[64][65];   // [r][i]
    const int lane = threadIdx.x, ty = threadIdx.y;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int4 tt = tiles[t];
        const TcGView& v = gv[2 * tt.x + w];
        const bool isx = tt.y == 0;
        const float* M = isx ? v.X : v.Y;
        const int64_t cnt = isx ? v.O : v.S;
        const int64_t si = isx ? v.xo : v.ys, sr = isx ? v.xr : v.yr;
        const int64_t R = v.R, i0 = (int64_t)tt.z * 64;
        if (si == 1) {   // contiguous along i: lanes walk i
            for (int r = ty; r < 64; r += 8)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t i = i0 + 32 * h + lane;
                    tile[r][32 * h + lane] = (r < R && i < cnt) ? M[r * sr + i] : 0.f;
                }
        } else {         // contiguous along r: lanes walk r
            for (int k = ty; k < 64; k += 8)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t i = i0 + k, r = 32 * h + lane;
                    tile[r][k] = (r < R && i < cnt) ? M[i * si + r * sr] : 0.f;
                }
        }
        __syncthreads();
        // rows [i][64] with r contiguous: Xk (X) or Yk (Y); lanes walk pairs of r (values
        // r >= R stay as the zeros the buffers were created with)
        bf16* RM = static_cast<bf16*>(isx ? v.Xk : v.Yk);
        const int64_t ipad = isx ? v.O_pad : v.S_pad;
        for (int k = ty; k < 64; k += 8) {
            const int64_t i = i0 + k;
            if (i < ipad && 2 * lane < R)
                *reinterpret_cast<uint32_t*>(RM + i * 64 + 2 * lane) =
                    pack_bf16x2(tile[2 * lane][k], tile[2 * lane + 1][k]);
        }
        if (!isx) {   // Ytk, Y2tk rows r < R, [64][ldt] with s contiguous; lanes walk pairs of s
            bf16* Yt = static_cast<bf16*>(v.Ytk);
            bf16* Y2t = static_cast<bf16*>(v.Y2tk);
            for (int r = ty; r < R; r += 8) {
                const int64_t i = i0 + 2 * lane;
                if (i < v.S_pad) {
                    const float y0 = tile[r][2 * lane], y1 = tile[r][2 * lane + 1];
                    *reinterpret_cast<uint32_t*>(Yt + r * v.ldt + i) = pack_bf16x2(y0, y1);
                    *reinterpret_cast<uint32_t*>(Y2t + r * v.ldt + i) =
                        pack_bf16x2(y0 * y0, y1 * y1);
                }
            }
        }
        __syncthreads();   // the tile is reused by the next step
    }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// 2-D tensor map: inner extent `inner` elements, `outer` rows `row_bytes` apart.
int make_map(CUtensorMap* m, CUtensorMapDataType dt, const void* ptr, uint64_t inner,
             uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
             CUtensorMapSwizzle swz) {
    auto fn = encode_fn();
    if (!fn) return DNA_ERR_CUDA;
    if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0 || row_bytes % 16 != 0) return DNA_ERR_ARG;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, dt, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? DNA_OK : DNA_ERR_CUDA;
}

template <int RP, bool WITH_B>
int launch_pass1(const P1Args& a, const TcMaps& m, int64_t O_pad, int splits, cudaStream_t st) {
    const uint32_t smem = P1Layout<RP>::TOTAL + 1024;
    auto k = k_tc_pass1<RP, WITH_B>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    dim3 grid((unsigned)(O_pad / OBLK), (unsigned)splits);
    k<<<grid, P1_THREADS, smem, st>>>(a, m.y, m.yt, m.y2t, m.v);
    return after_launch();
}

}  // namespace tc

int TcBf16::rank_pad(int64_t R) {
    return R <= 64 ? 64 : (R <= 128 ? 128 : (R <= 256 ? 256 : (R <= 512 ? 512 : 0)));
}

int TcBf16::make_maps(TcMaps* m, const TcOperands& op, const float* V, int64_t vs,
                      const void* Xmk, const void* Xdk) {
    using namespace tc;
    const uint64_t rp = (uint64_t)rank_pad(op.R);
    const auto BF = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const auto SW = CU_TENSOR_MAP_SWIZZLE_128B;
    int e = make_map(&m->x, BF, op.Xk, rp, op.O_pad, rp * 2, 64, OBLK, SW);
    if (!e) e = make_map(&m->y, BF, op.Yk, rp, op.S_pad, rp * 2, 64, SCH, SW);
    const uint32_t ytbox = (uint32_t)(rp < 128 ? rp : 128);   // rows of one r-block
    const uint64_t ldt = (uint64_t)(op.ldt ? op.ldt : op.S_pad);
    if (!e) e = make_map(&m->yt, BF, op.Ytk, op.S_pad, rp, ldt * 2, SCH, ytbox, SW);
    if (!e) e = make_map(&m->y2t, BF, op.Y2tk, op.S_pad, rp, ldt * 2, SCH, ytbox, SW);
    if (!e) e = make_map(&m->xm, BF, Xmk, rp, op.O_pad, rp * 2, 64, OBLK, SW);
    if (!e) e = make_map(&m->xd, BF, Xdk, rp, op.O_pad, rp * 2, 64, OBLK, SW);
    if (!e)
        e = make_map(&m->v, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, V, (uint64_t)op.O, (uint64_t)op.S,
                     (uint64_t)vs * 4, OBLK, SCH, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (!e && op.Qg) {      // the Q, Qbar workspace of pass 1 at RP > 128, and larger boxes
        e = make_map(&m->q, BF, op.Qg, (uint64_t)op.ldq, op.O_pad, (uint64_t)op.ldq * 2, 64, OBLK, SW);
        if (!e) e = make_map(&m->qb, BF, op.Qbg, (uint64_t)op.ldq, op.O_pad, (uint64_t)op.ldq * 2, 64,
                             OBLK, SW);
        if (!e) e = make_map(&m->y128, BF, op.Yk, rp, op.S_pad, rp * 2, 64, 128, SW);
        if (!e) e = make_map(&m->yt256, BF, op.Ytk, op.S_pad, rp, op.S_pad * 2, SCH, 256, SW);
        if (!e) e = make_map(&m->y2t256, BF, op.Y2tk, op.S_pad, rp, op.S_pad * 2, SCH, 256, SW);
    }
    if (!e && op.Qg && op.plane) {   // lo planes of pass 1 of the split form at RP > 128
        const bf16* ql = static_cast<const bf16*>(op.Qg) + op.qplane;
        const bf16* qbl = static_cast<const bf16*>(op.Qbg) + op.qplane;
        e = make_map(&m->q_l, BF, ql, (uint64_t)op.ldq, op.O_pad, (uint64_t)op.ldq * 2, 64, OBLK, SW);
        if (!e) e = make_map(&m->qb_l, BF, qbl, (uint64_t)op.ldq, op.O_pad, (uint64_t)op.ldq * 2, 64,
                             OBLK, SW);
        if (!e) e = make_map(&m->y128_l, BF, static_cast<const bf16*>(op.Yk) + op.plane, rp, op.S_pad,
                             rp * 2, 64, 128, SW);
        if (!e) e = make_map(&m->yt256_l, BF, static_cast<const bf16*>(op.Ytk) + op.plane, op.S_pad,
                             rp, op.S_pad * 2, SCH, 256, SW);
        if (!e) e = make_map(&m->y2t256_l, BF, static_cast<const bf16*>(op.Y2tk) + op.plane,
                             op.S_pad, rp, op.S_pad * 2, SCH, 256, SW);
    }
    if (!e && op.plane) {   // lo planes of the split FP32 form
        const bf16* yl = static_cast<const bf16*>(op.Yk) + op.plane;
        const bf16* ytl = static_cast<const bf16*>(op.Ytk) + op.plane;
        const bf16* y2tl = static_cast<const bf16*>(op.Y2tk) + op.plane;
        const bf16* xl = static_cast<const bf16*>(op.Xk) + op.plane;
        e = make_map(&m->x_l, BF, xl, rp, op.O_pad, rp * 2, 64, OBLK, SW);
        if (!e) e = make_map(&m->xm_l, BF, static_cast<const bf16*>(Xmk) + op.plane, rp, op.O_pad,
                             rp * 2, 64, OBLK, SW);
        if (!e) e = make_map(&m->xd_l, BF, static_cast<const bf16*>(Xdk) + op.plane, rp, op.O_pad,
                             rp * 2, 64, OBLK, SW);
        if (!e) e = make_map(&m->y_l, BF, yl, rp, op.S_pad, rp * 2, 64, SCH, SW);
        if (!e) e = make_map(&m->yt_l, BF, ytl, op.S_pad, rp, op.S_pad * 2, SCH, ytbox, SW);
        if (!e) e = make_map(&m->y2t_l, BF, y2tl, op.S_pad, rp, op.S_pad * 2, SCH, ytbox, SW);
    }
    return e;
}

int TcBf16::to_bf16(const float* src, int64_t si, int64_t sj, int64_t rows, int64_t cols,
                    void* dst, int64_t ld, int64_t rows_pad, int64_t cols_pad, bool square,
                    cudaStream_t st) {
    dim3 blk(32, 8);
    dim3 grid((unsigned)((cols_pad + 31) / 32), (unsigned)((rows_pad + 31) / 32));
    tc::k_to_bf16<<<grid, blk, 0, st>>>(src, si, sj, rows, cols, static_cast<tc::bf16*>(dst), ld,
                                         square);
    return after_launch();
}

int TcBf16::y_operands(const float* Y, int64_t ys, int64_t yr, const TcOperands& op,
                       bool with_sq, cudaStream_t st) {
    const int64_t rp = rank_pad(op.R);
    dim3 grid((unsigned)(op.S_pad / 32), (unsigned)(rp / 32));
    tc::k_y_operands<<<grid, dim3(32, 8), 0, st>>>(
        Y, ys, yr, op.S, op.R, static_cast<tc::bf16*>(const_cast<void*>(op.Yk)), rp,
        static_cast<tc::bf16*>(const_cast<void*>(op.Ytk)),
        static_cast<tc::bf16*>(const_cast<void*>(op.Y2tk)), op.S_pad, with_sq);
    return after_launch();
}

int TcBf16::group_operands(const TcGView* gv, const void* tiles, int n, int w, int grid,
                           cudaStream_t st) {
    if (n <= 0) return DNA_OK;
    tc::k_g_operands<<<std::max(1, std::min(n, grid)), dim3(32, 8), 0, st>>>(
        gv, static_cast<const int4*>(tiles), n, w);
    return after_launch();
}

int TcBf16::group_pass1(const TcGView* gv, const void* tiles, int n, int w, bool with_b,
                        int ctas, int* status, cudaStream_t st) {
    if (n <= 0) return DNA_OK;
    const uint32_t smem = tc::P1Layout<64>::TOTAL + 1024;
    auto k = with_b ? tc::k_tc_gpass1p<true> : tc::k_tc_gpass1p<false>;
    const int grid = std::max(1, std::min(n, ctas));
    k<<<grid, tc::P1_THREADS, smem, st>>>(gv, static_cast<const int4*>(tiles), n, w, status);
    return after_launch();
}

int TcBf16::group_prepare() {
    const int s1 = (int)(tc::P1Layout<64>::TOTAL + 1024);
    if (cudaFuncSetAttribute(tc::k_tc_gpass1p<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             s1) != cudaSuccess ||
        cudaFuncSetAttribute(tc::k_tc_gpass1p<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             s1) != cudaSuccess)
        return DNA_ERR_CUDA;
    return group_prepare_pass2();
}

int TcBf16::pass1(const TcOperands& op, const TcMaps& maps, float* Apart, float* Bpart,
                  int splits, int64_t s_per, bool with_b, int* status, cudaStream_t st) {
    tc::P1Args a{};
    a.S = op.S; a.O = op.O; a.R = op.R; a.s_per = s_per;
    a.Apart = Apart; a.Bpart = Bpart; a.status = status;
    a.V = op.V; a.vs = op.vs; a.X = op.Xk; a.rp = rank_pad(op.R);
    const int rp = rank_pad(op.R);
    if (rp == 64)
        return with_b ? tc::launch_pass1<64, true>(a, maps, op.O_pad, splits, st)
                      : tc::launch_pass1<64, false>(a, maps, op.O_pad, splits, st);
    if (rp == 128)
        return with_b ? tc::launch_pass1<128, true>(a, maps, op.O_pad, splits, st)
                      : tc::launch_pass1<128, false>(a, maps, op.O_pad, splits, st);
    if (rp == 256 || rp == 512)
        return pass1_mat(op, maps, Apart, Bpart, splits, s_per, with_b, status, st);
    return DNA_ERR_UNSUPPORTED;
}

int TcBf16::chunk() { return tc::SCH; }
int TcBf16::oblock() { return tc::OBLK; }

namespace tc {
// The timeout path of the bounded barrier waits (wait_phase_limit, the wait of every
// tcgen05 kernel here), with no asynchronous copy or MMA in flight: warp 0 waits on a
// barrier phase that nothing completes and gives up after `limit` cycles, raising the
// CTA's abort flag; warp 1, waiting on another such phase, leaves on the flag (or after
// 1000 x limit); the CTA then reports STATUS_TIMEOUT as the tcgen05 kernels do.
__global__ void k_wait_timeout_check(long long limit, int* status) {
    __shared__ uint64_t bar[2];
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    volatile int* abort = &abort_flag;
    if ((threadIdx.x & 31) == 0) {
        if (threadIdx.x == 0)
            wait_phase_limit(&bar[0], 0, abort, limit);
        else
            wait_phase_limit(&bar[1], 0, abort, 1000 * limit);
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort) atomicOr(status, STATUS_TIMEOUT);
}
}  // namespace tc

int TcBf16::check_wait_timeout(long long limit, int* status, cudaStream_t st) {
    tc::k_wait_timeout_check<<<1, 64, 0, st>>>(limit, status);
    return after_launch();
}

}  // namespace dna
