// tcgen05 kernels of the FP32 form on the tensor cores: every float32 operand x is held as
// two bf16 numbers, x_hi = bf16(x) and x_lo = bf16(x - x_hi), and every product as
// x_hi y_hi + x_hi y_lo + x_lo y_hi (the dropped x_lo y_lo is below 2^-16 |x y|), summed in
// float32 in tensor memory.  The kernels have the structure of the BF16 ones
// (tc_bf16.cu): TMA rings for V and the B operands, the o-block's A operands in tensor
// memory, sixteen epilogue warps, a producer warp and two MMA-issuing warps.
//
// Pass 1 splits by accumulator to fit tensor memory: CTAs with which = 0 form q and
// accumulate A = Y^t Q (Algorithm 1 step 5), CTAs with which = 1 form qbar and
// accumulate B = (Y o Y)^t Qbar (step 10).  Each recomputes Z for its o-block (Z x 2,
// one accumulator, X hi / lo and Q hi / lo take 448 of the 512 columns).
// Pass 2 keeps both candidates in one CTA (Z x 2 for each, four operand planes).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dna_internal.h"
#include "tc_common.cuh"

namespace dna {
namespace tc {

// v -> (hi, lo) bf16 pairs of two values: hi = bf16(v), lo = bf16(v - hi).
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
    hi = pack_bf16x2(v0, v1);
    const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
    lo = pack_bf16x2(v0 - h0, v1 - h1);
}

template <int RP>
struct P1SLayout {
    static constexpr int VST = 3, YST = 2, TST = 2;
    static constexpr uint32_t V_BYTES = SCH * OBLK * 4;   // [64][128] fp32
    static constexpr uint32_t Y_BYTES = SCH * RP * 2;     // one plane [64][RP] bf16
    static constexpr uint32_t Y_STAGE = 2 * Y_BYTES;      // hi, lo
    static constexpr uint32_t T_BYTES = RP * SCH * 2;     // one plane [RP][64] bf16
    static constexpr uint32_t T_STAGE = 2 * T_BYTES;
    static constexpr uint32_t VR = 0;
    static constexpr uint32_t YR = VR + VST * V_BYTES;
    static constexpr uint32_t TR = YR + YST * Y_STAGE;
    static constexpr uint32_t BAR = TR + TST * T_STAGE;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;
    // tensor memory columns: Z x 2 | accumulator | X hi | X lo | Q hi | Q lo
    static constexpr uint32_t TACC = 2 * SCH, TXH = TACC + RP, TXL = TXH + RP / 2,
                              TQH = TXL + RP / 2, TQL = TQH + SCH / 2;
    static_assert(TQL + SCH / 2 <= NCOLS, "tensor memory budget");
    static_assert(YR % 1024 == 0 && TR % 1024 == 0 && Y_BYTES % 1024 == 0 &&
                      T_BYTES % 1024 == 0,
                  "tiles must be 1024-byte aligned");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};

enum { S_XFULL = 0, S_VFULL = 1, S_VEMPTY = 4, S_YFULL = 7, S_TFULL = 9, S_ZFULL = 11,
       S_ZEMPTY = 13, S_QFULL = 15, S_QEMPTY = 16, S_DRAIN = 18, S_COUNT = 20 };

// grid = (O_pad / 128, nwhich x splits): which = blockIdx.y % nwhich (nwhich = 2 for
// DNA, 1 for the MU step, which needs A only), split = blockIdx.y / nwhich.
template <int RP>
__global__ void __launch_bounds__(P1_THREADS, 1)
    k_tc_pass1s(P1Args a, int64_t xplane, int nwhich, const __grid_constant__ CUtensorMap tmY,
                const __grid_constant__ CUtensorMap tmYl, const __grid_constant__ CUtensorMap tmYt,
                const __grid_constant__ CUtensorMap tmYtl,
                const __grid_constant__ CUtensorMap tmY2t,
                const __grid_constant__ CUtensorMap tmY2tl,
                const __grid_constant__ CUtensorMap tmV) {
    using L = P1SLayout<RP>;
    constexpr int VST = L::VST, YST = L::YST, TST = L::TST;
    static_assert(YST == 2 && TST == 2, "stage reuse is signalled by the commit barriers");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + S_COUNT * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L::BAR + S_COUNT * 8 + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int which = (int)blockIdx.y % nwhich, split = (int)blockIdx.y / nwhich;
    const int64_t o0 = (int64_t)blockIdx.x * OBLK;
    const int64_t s_begin = (int64_t)split * a.s_per;
    const int64_t s_end = min(a.S, s_begin + a.s_per);
    const int nch = s_end > s_begin ? (int)((s_end - s_begin + SCH - 1) / SCH) : 0;
    const CUtensorMap* tmTh = which ? &tmY2t : &tmYt;
    const CUtensorMap* tmTl = which ? &tmY2tl : &tmYtl;

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == W_PRODUCER * 32) {
        mbar_init(&bar[S_XFULL], W_EPI);
        for (int i = 0; i < VST; ++i) {
            mbar_init(&bar[S_VFULL + i], 1);
            mbar_init(&bar[S_VEMPTY + i], W_EPI);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar[S_YFULL + i], 1);
            mbar_init(&bar[S_TFULL + i], 1);
            mbar_init(&bar[S_ZFULL + i], 1);
            mbar_init(&bar[S_ZEMPTY + i], W_EPI);
            mbar_init(&bar[S_QEMPTY + i], 1);
            mbar_init(&bar[S_DRAIN + i], 1);
        }
        mbar_init(&bar[S_QFULL], W_EPI);
        *abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == W_PRODUCER) {
        if (lane == 0 && nch > 0) {
            tma_prefetch_desc(&tmY); tma_prefetch_desc(&tmYl); tma_prefetch_desc(tmTh);
            tma_prefetch_desc(tmTl); tma_prefetch_desc(&tmV);
            int kv = 0, ky = 0, kt = 0;
            long long t0 = clock64();
            while (kv < nch || ky < nch || kt < nch) {
                bool prog = false;
                if (kv < nch && mbar_test(&bar[S_VEMPTY + kv % VST], ((kv / VST) & 1) ^ 1)) {
                    const int st = kv % VST;
                    mbar_arrive_expect_tx(&bar[S_VFULL + st], L::V_BYTES);
                    tma_load_2d(sbase + L::VR + st * L::V_BYTES, &tmV, (int32_t)o0,
                                (int32_t)(s_begin + (int64_t)kv * SCH), &bar[S_VFULL + st]);
                    ++kv;
                    prog = true;
                }
                // Y(ky) reuses the stage of chunk ky - 2, free once GEMM1 of it is done
                if (ky < nch && (ky < YST || mbar_test(&bar[S_ZFULL + (ky & 1)],
                                                       ((ky - 2) >> 1) & 1))) {
                    const int st = ky % YST;
                    const uint32_t dst = sbase + L::YR + st * L::Y_STAGE;
                    const int32_t s0 = (int32_t)(s_begin + (int64_t)ky * SCH);
                    mbar_arrive_expect_tx(&bar[S_YFULL + st], L::Y_STAGE);
                    for (int at = 0; at < RP / 64; ++at) {
                        tma_load_2d(dst + at * SCH * 128, &tmY, 64 * at, s0, &bar[S_YFULL + st]);
                        tma_load_2d(dst + L::Y_BYTES + at * SCH * 128, &tmYl, 64 * at, s0,
                                    &bar[S_YFULL + st]);
                    }
                    ++ky;
                    prog = true;
                }
                // the Y^t (or (Y o Y)^t) stage of chunk kt - 2 is free once GEMM2 of it is done
                if (kt < nch && (kt < TST || mbar_test(&bar[S_QEMPTY + (kt & 1)],
                                                       ((kt - 2) >> 1) & 1))) {
                    const int st = kt % TST;
                    const uint32_t dst = sbase + L::TR + st * L::T_STAGE;
                    const int32_t s0 = (int32_t)(s_begin + (int64_t)kt * SCH);
                    mbar_arrive_expect_tx(&bar[S_TFULL + st], L::T_STAGE);
                    tma_load_2d(dst, tmTh, s0, 0, &bar[S_TFULL + st]);
                    tma_load_2d(dst + L::T_BYTES, tmTl, s0, 0, &bar[S_TFULL + st]);
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
                    drain_phase(&bar[S_VFULL + k % VST], (k / VST) & 1);
                for (int k = max(0, ky - YST); k < ky; ++k)
                    drain_phase(&bar[S_YFULL + k % YST], (k / YST) & 1);
                for (int k = max(0, kt - TST); k < kt; ++k)
                    drain_phase(&bar[S_TFULL + k % TST], (k / TST) & 1);
            }
        }
    } else if (warp == W_MMA_Z) {
        // Z(m) = X Y(m)^t as x_hi y_hi + x_hi y_lo + x_lo y_hi, into buffer m & 1
        if (lane == 0 && nch > 0) {
            bool ok = wait_phase(&bar[S_XFULL], 0, abort);
            for (int m = 0; ok && m < nch; ++m) {
                const int zb = m & 1;
                if (!(ok = wait_phase(&bar[S_YFULL + m % YST], (m / YST) & 1, abort))) break;
                if (m >= 2 &&
                    !(ok = wait_phase(&bar[S_ZEMPTY + zb], ((m >> 1) & 1) ^ 1, abort)))
                    break;
                tc_fence_after();
                const uint32_t yh = sbase + L::YR + (m % YST) * L::Y_STAGE, yl = yh + L::Y_BYTES;
                const uint32_t tz = tmem + zb * SCH;
                constexpr uint32_t idesc = idesc_bf16(OBLK, SCH);
#pragma unroll
                for (int kk = 0; kk < RP / 16; ++kk) {
                    const uint32_t kb = 32u * kk, at = kb >> 7, within = kb & 127u;
                    const uint32_t off = at * SCH * 128 + within;
                    mma_bf16_tmem_a(tz, tmem + L::TXH + 8 * kk, desc_sw128(yh + off), idesc, kk > 0);
                    mma_bf16_tmem_a(tz, tmem + L::TXH + 8 * kk, desc_sw128(yl + off), idesc, 1u);
                    mma_bf16_tmem_a(tz, tmem + L::TXL + 8 * kk, desc_sw128(yh + off), idesc, 1u);
                }
                mma_commit(&bar[S_ZFULL + zb]);
            }
            if (!ok) {
                mma_commit(&bar[S_DRAIN + 0]);
                drain_phase(&bar[S_DRAIN + 0], 0);
            }
        }
    } else if (warp == W_MMA_AB) {
        // accumulator += Q(m) T(m) as q_hi t_hi + q_hi t_lo + q_lo t_hi
        if (lane == 0 && nch > 0) {
            bool ok = true;
            for (int m = 0; ok && m < nch; ++m) {
                if (!(ok = wait_phase(&bar[S_QFULL], m & 1, abort))) break;
                if (!(ok = wait_phase(&bar[S_TFULL + m % TST], (m / TST) & 1, abort))) break;
                tc_fence_after();
                const uint32_t th = sbase + L::TR + (m % TST) * L::T_STAGE, tl = th + L::T_BYTES;
                constexpr uint32_t idesc = idesc_bf16(OBLK, RP);
#pragma unroll
                for (int kk = 0; kk < SCH / 16; ++kk) {
                    const uint32_t acc = (m > 0 || kk > 0) ? 1u : 0u;
                    mma_bf16_tmem_a(tmem + L::TACC, tmem + L::TQH + 8 * kk,
                                    desc_sw128(th + 32u * kk), idesc, acc);
                    mma_bf16_tmem_a(tmem + L::TACC, tmem + L::TQH + 8 * kk,
                                    desc_sw128(tl + 32u * kk), idesc, 1u);
                    mma_bf16_tmem_a(tmem + L::TACC, tmem + L::TQL + 8 * kk,
                                    desc_sw128(th + 32u * kk), idesc, 1u);
                }
                mma_commit(&bar[S_QEMPTY + (m & 1)]);
            }
            if (!ok) {
                mma_commit(&bar[S_DRAIN + 1]);
                drain_phase(&bar[S_DRAIN + 1], 0);
            }
        }
    } else {
        // epilogue warps 0-15: lane quadrant qd = warp % 4 (o = o0 + 32 qd + lane), chunk
        // columns 16 cg .. 16 cg + 15 with cg = warp / 4
        const int qd = warp & 3, cg = warp >> 2;
        const int row = 32 * qd + lane;
        const int64_t o = o0 + row;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        if (nch > 0) {   // X hi and lo of this o-block into tensor memory
            constexpr int UP = RP / 32;
            const bf16* X = static_cast<const bf16*>(a.X);
            for (int u = cg; u < 2 * UP; u += 4) {
                const bool lo = u >= UP;
                x_to_tmem(X + (lo ? xplane : 0), a.rp, o, lo ? u - UP : u,
                          tmem + (lo ? L::TXL : L::TXH) + lane_off);
            }
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[S_XFULL]);
        }
        float zmin = 1.f;   // min over v > 0 of z (see the BF16 pass 1)
        bool ok = true;
        for (int k = 0; k < nch; ++k) {
            const int zb = k & 1, vs = k % VST;
            ok = wait_phase(&bar[S_ZFULL + zb], (k >> 1) & 1, abort);
            ok = ok && wait_phase(&bar[S_VFULL + vs], (k / VST) & 1, abort);
            if (!(ok = __all_sync(0xffffffffu, ok))) break;   // keep the warp converged
            tc_fence_after();
            uint32_t zr[16];
            tmem_ld16(tmem + zb * SCH + lane_off + 16 * cg, zr);
            const float* Vs = reinterpret_cast<const float*>(sm + L::VR + vs * L::V_BYTES) +
                              16 * cg * OBLK + row;
            float vv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) vv[j] = Vs[j * OBLK];
            tmem_ld_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[S_ZEMPTY + zb]);
            uint32_t hp[8], lp[8];
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                float w[2];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const float v = vv[j + t];
                    const float z = __uint_as_float(zr[j + t]);
                    const float rz = __fdividef(1.0f, z);
                    const bool pos = v > 0.f;
                    zmin = fminf(zmin, pos ? z : 1.f);
                    const float q = v * rz;
                    w[t] = pos ? (which ? q * rz : q) : 0.f;   // q, or qbar = q / z
                }
                split2(w[0], w[1], hp[j / 2], lp[j / 2]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[S_VEMPTY + vs]);
            if (k >= 1) {   // GEMM2 of chunk k - 1 has read the Q buffer
                const int kp = k - 1;
                ok = wait_phase(&bar[S_QEMPTY + (kp & 1)], (kp >> 1) & 1, abort);
                if (!(ok = __all_sync(0xffffffffu, ok))) break;
                tc_fence_after();
            }
            tmem_st8(tmem + L::TQH + 8 * cg + lane_off, hp);
            tmem_st8(tmem + L::TQL + 8 * cg + lane_off, lp);
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[S_QFULL]);
        }
        if (!(zmin > 0.f)) atomicOr(a.status, STATUS_NONFINITE);
        if (ok && nch > 0) {
            const int kl = nch - 1;
            ok = __all_sync(0xffffffffu,
                            wait_phase(&bar[S_QEMPTY + (kl & 1)], (kl >> 1) & 1, abort));
        }
        if (ok && nch > 0) {
            tc_fence_after();
            const int64_t base = (int64_t)split * a.R;
            float* dst = which ? a.Bpart : a.Apart;
#pragma unroll 1
            for (int g = cg; g < RP / 32; g += 4) {
                uint32_t r32[32];
                tmem_ld32(tmem + L::TACC + lane_off + 32 * g, r32);
                tmem_ld_wait();
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

// Pass 2 of the split form: Z_MU and Z_DNA from hi / lo candidates and a hi / lo Y.
template <int RP>
struct P2SLayout {
    static constexpr int VST = 4, YST = 2;
    static constexpr uint32_t V_BYTES = SCH * OBLK * 4;
    static constexpr uint32_t Y_BYTES = SCH * RP * 2;
    static constexpr uint32_t Y_STAGE = 2 * Y_BYTES;
    static constexpr uint32_t VR = 0;
    static constexpr uint32_t YR = VR + VST * V_BYTES;
    static constexpr uint32_t RED = YR + YST * Y_STAGE;   // [4 column groups][2][128] float64
    static constexpr uint32_t BAR = RED + 4 * 2 * OBLK * 8;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;
    // tensor memory: (Z_mu, Z_dna) x 2 | X_mu hi | X_mu lo | X_dna hi | X_dna lo
    static constexpr uint32_t TX = 4 * SCH;
    static_assert(TX + 4 * (RP / 2) <= NCOLS, "tensor memory budget");
    static_assert(YR % 1024 == 0 && Y_BYTES % 1024 == 0, "tiles must be 1024-byte aligned");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};

enum { T_XFULL = 0, T_VFULL = 1, T_VEMPTY = 5, T_YFULL = 9, T_ZFULL = 11, T_ZEMPTY = 15,
       T_DRAIN = 17, T_COUNT = 19 };

template <int RP>
__global__ void __launch_bounds__(P1_THREADS, 1)
    k_tc_pass2s(P2Args a, int64_t xplane, const __grid_constant__ CUtensorMap tmY,
                const __grid_constant__ CUtensorMap tmYl, const __grid_constant__ CUtensorMap tmV) {
    using L = P2SLayout<RP>;
    constexpr int VST = L::VST, YST = L::YST;
    static_assert(YST == 2, "stage reuse is signalled by the commit barriers");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + T_COUNT * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L::BAR + T_COUNT * 8 + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t o0 = (int64_t)blockIdx.x * OBLK;
    const int64_t s_begin = (int64_t)blockIdx.y * a.s_per;
    const int64_t s_end = min(a.S, s_begin + a.s_per);
    const int nch = s_end > s_begin ? (int)((s_end - s_begin + SCH - 1) / SCH) : 0;

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == W_PRODUCER * 32) {
        mbar_init(&bar[T_XFULL], W_EPI);
        for (int i = 0; i < VST; ++i) {
            mbar_init(&bar[T_VFULL + i], 1);
            mbar_init(&bar[T_VEMPTY + i], W_EPI);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar[T_YFULL + i], 1);
            mbar_init(&bar[T_ZFULL + i], 1);
            mbar_init(&bar[T_ZFULL + 2 + i], 1);
            mbar_init(&bar[T_ZEMPTY + i], W_EPI);
            mbar_init(&bar[T_DRAIN + i], 1);
        }
        *abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == W_PRODUCER) {
        if (lane == 0 && nch > 0) {
            tma_prefetch_desc(&tmY); tma_prefetch_desc(&tmYl); tma_prefetch_desc(&tmV);
            int kv = 0, ky = 0;
            long long t0 = clock64();
            while (kv < nch || ky < nch) {
                bool prog = false;
                if (kv < nch && mbar_test(&bar[T_VEMPTY + kv % VST], ((kv / VST) & 1) ^ 1)) {
                    const int st = kv % VST;
                    mbar_arrive_expect_tx(&bar[T_VFULL + st], L::V_BYTES);
                    tma_load_2d(sbase + L::VR + st * L::V_BYTES, &tmV, (int32_t)o0,
                                (int32_t)(s_begin + (int64_t)kv * SCH), &bar[T_VFULL + st]);
                    ++kv;
                    prog = true;
                }
                // Y(ky) reuses the stage of chunk ky - 2, free once both GEMMs of it are done
                if (ky < nch &&
                    (ky < YST || (mbar_test(&bar[T_ZFULL + (ky & 1)], ((ky - 2) >> 1) & 1) &&
                                  mbar_test(&bar[T_ZFULL + 2 + (ky & 1)], ((ky - 2) >> 1) & 1)))) {
                    const int st = ky % YST;
                    const uint32_t dst = sbase + L::YR + st * L::Y_STAGE;
                    const int32_t s0 = (int32_t)(s_begin + (int64_t)ky * SCH);
                    mbar_arrive_expect_tx(&bar[T_YFULL + st], L::Y_STAGE);
                    for (int at = 0; at < RP / 64; ++at) {
                        tma_load_2d(dst + at * SCH * 128, &tmY, 64 * at, s0, &bar[T_YFULL + st]);
                        tma_load_2d(dst + L::Y_BYTES + at * SCH * 128, &tmYl, 64 * at, s0,
                                    &bar[T_YFULL + st]);
                    }
                    ++ky;
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
            if (*abort) {
                for (int k = max(0, kv - VST); k < kv; ++k)
                    drain_phase(&bar[T_VFULL + k % VST], (k / VST) & 1);
                for (int k = max(0, ky - YST); k < ky; ++k)
                    drain_phase(&bar[T_YFULL + k % YST], (k / YST) & 1);
            }
        }
    } else if (warp == W_MMA_Z || warp == W_MMA_AB) {
        // candidate c: Z_c(m) = X_c Y(m)^t in the split form, into buffer m & 1
        const int c = warp == W_MMA_AB ? 1 : 0;
        if (lane == 0 && nch > 0) {
            bool ok = wait_phase(&bar[T_XFULL], 0, abort);
            const uint32_t xh = tmem + L::TX + (uint32_t)(2 * c) * (RP / 2);
            const uint32_t xl = xh + RP / 2;
            for (int m = 0; ok && m < nch; ++m) {
                const int zb = m & 1;
                if (!(ok = wait_phase(&bar[T_YFULL + m % YST], (m / YST) & 1, abort))) break;
                if (m >= 2 &&
                    !(ok = wait_phase(&bar[T_ZEMPTY + zb], ((m >> 1) & 1) ^ 1, abort)))
                    break;
                tc_fence_after();
                const uint32_t yh = sbase + L::YR + (m % YST) * L::Y_STAGE, yl = yh + L::Y_BYTES;
                const uint32_t tz = tmem + zb * 2 * SCH + c * SCH;
                constexpr uint32_t idesc = idesc_bf16(OBLK, SCH);
#pragma unroll
                for (int kk = 0; kk < RP / 16; ++kk) {
                    const uint32_t kb = 32u * kk, at = kb >> 7, within = kb & 127u;
                    const uint32_t off = at * SCH * 128 + within;
                    mma_bf16_tmem_a(tz, xh + 8 * kk, desc_sw128(yh + off), idesc, kk > 0);
                    mma_bf16_tmem_a(tz, xh + 8 * kk, desc_sw128(yl + off), idesc, 1u);
                    mma_bf16_tmem_a(tz, xl + 8 * kk, desc_sw128(yh + off), idesc, 1u);
                }
                mma_commit(&bar[T_ZFULL + 2 * c + zb]);
            }
            if (!ok) {
                mma_commit(&bar[T_DRAIN + c]);
                drain_phase(&bar[T_DRAIN + c], 0);
            }
        }
    } else {
        const int qd = warp & 3, cg = warp >> 2;
        const int row = 32 * qd + lane;
        const int64_t o = o0 + row;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        if (nch > 0) {   // X_mu, X_dna (hi, lo) of this o-block into tensor memory
            constexpr int UP = RP / 32;   // 16-column units per plane
            for (int u = cg; u < 4 * UP; u += 4) {
                const int mat = u / UP;   // 0 mu hi, 1 mu lo, 2 dna hi, 3 dna lo
                const bf16* X = static_cast<const bf16*>(mat < 2 ? a.Xm : a.Xd) +
                                ((mat & 1) ? xplane : 0);
                x_to_tmem(X, a.rp, o, u % UP, tmem + L::TX + (uint32_t)mat * (RP / 2) + lane_off);
            }
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[T_XFULL]);
        }
        double acc_m = 0.0, acc_d = 0.0;
        bool ok = true;
        for (int k = 0; k < nch; ++k) {
            const int zb = k & 1, vs = k % VST;
            const uint32_t zpar = (k >> 1) & 1;
            ok = wait_phase(&bar[T_ZFULL + zb], zpar, abort);
            ok = ok && wait_phase(&bar[T_ZFULL + 2 + zb], zpar, abort);
            ok = ok && wait_phase(&bar[T_VFULL + vs], (k / VST) & 1, abort);
            if (!(ok = __all_sync(0xffffffffu, ok))) break;   // keep the warp converged
            tc_fence_after();
            const uint32_t tz = tmem + zb * 2 * SCH + lane_off + 16 * cg;
            uint32_t zm[16], zd[16];
            tmem_ld16(tz, zm);
            tmem_ld16(tz + SCH, zd);
            const float* Vs = reinterpret_cast<const float*>(sm + L::VR + vs * L::V_BYTES) +
                              16 * cg * OBLK + row;
            float vv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) vv[j] = Vs[j * OBLK];
            tmem_ld_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[T_ZEMPTY + zb]);
            float run_m = 0.f, run_d = 0.f;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float v = vv[j];
                const float z1 = __uint_as_float(zm[j]), z2 = __uint_as_float(zd[j]);
                const bool pos = v > 0.f;
                // the hardware logarithm (absolute error near 2^-21 around 1, relative
                // 2^-21 elsewhere): well inside the split form's 1e-4 near-tie margin
                const float l1 = __logf(z1), l2 = __logf(z2);
                run_m += pos ? z1 - v * l1 : z1;
                run_d += pos ? z2 - v * l2 : z2;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[T_VEMPTY + vs]);
            acc_m += (double)run_m;
            acc_d += (double)run_d;
        }
        if (!(fabs(acc_m) < INFINITY && fabs(acc_d) < INFINITY))
            atomicOr(a.status, STATUS_NONFINITE);
        double* red = reinterpret_cast<double*>(sm + L::RED);
        red[(cg * 2 + 0) * OBLK + row] = acc_m;
        red[(cg * 2 + 1) * OBLK + row] = acc_d;
        asm volatile("bar.sync 1, %0;" ::"r"(W_EPI * 32) : "memory");
        if (cg == 0 && ok && nch > 0 && !*abort && o < a.O) {
            double m = red[0 * OBLK + row], d = red[1 * OBLK + row];
            for (int g = 1; g < 4; ++g) {
                m += red[(g * 2 + 0) * OBLK + row];
                d += red[(g * 2 + 1) * OBLK + row];
            }
            a.dpart[((int64_t)blockIdx.y * 2 + 0) * a.O + o] = m;
            a.dpart[((int64_t)blockIdx.y * 2 + 1) * a.O + o] = d;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(a.status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

template <int RP>
int launch_pass1s(const P1Args& a, int64_t xplane, bool with_b, const TcMaps& m, int64_t O_pad,
                  int splits, cudaStream_t st) {
    const uint32_t smem = P1SLayout<RP>::TOTAL + 1024;
    auto k = k_tc_pass1s<RP>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    const int nwhich = with_b ? 2 : 1;
    dim3 grid((unsigned)(O_pad / OBLK), (unsigned)(nwhich * splits));
    k<<<grid, P1_THREADS, smem, st>>>(a, xplane, nwhich, m.y, m.y_l, m.yt, m.yt_l, m.y2t,
                                       m.y2t_l, m.v);
    return after_launch();
}

template <int RP>
int launch_pass2s(const P2Args& a, int64_t xplane, const TcMaps& m, int64_t O_pad, int splits,
                  cudaStream_t st) {
    const uint32_t smem = P2SLayout<RP>::TOTAL + 1024;
    auto k = k_tc_pass2s<RP>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    dim3 grid((unsigned)(O_pad / OBLK), (unsigned)splits);
    k<<<grid, P1_THREADS, smem, st>>>(a, xplane, m.y, m.y_l, m.v);
    return after_launch();
}

}  // namespace tc

int TcBf16::pass1_split(const TcOperands& op, const TcMaps& maps, float* Apart, float* Bpart,
                        int splits, int64_t s_per, bool with_b, int* status, cudaStream_t st) {
    tc::P1Args a{};
    a.S = op.S; a.O = op.O; a.R = op.R; a.s_per = s_per;
    a.Apart = Apart; a.Bpart = Bpart; a.status = status;
    a.V = op.V; a.vs = op.vs; a.X = op.Xk; a.rp = rank_pad(op.R);
    if (a.rp == 64) return tc::launch_pass1s<64>(a, op.plane, with_b, maps, op.O_pad, splits, st);
    if (a.rp == 128) return tc::launch_pass1s<128>(a, op.plane, with_b, maps, op.O_pad, splits, st);
    return DNA_ERR_UNSUPPORTED;
}

int TcBf16::pass2_split(const TcOperands& op, const TcMaps& maps, double* dpart, int splits,
                        int64_t s_per, int* status, cudaStream_t st) {
    tc::P2Args a{};
    a.S = op.S; a.O = op.O; a.R = op.R; a.s_per = s_per;
    a.dpart = dpart; a.status = status;
    a.V = op.V; a.vs = op.vs; a.Xm = op.Xmk; a.Xd = op.Xdk; a.rp = rank_pad(op.R);
    if (a.rp == 64) return tc::launch_pass2s<64>(a, op.plane, maps, op.O_pad, splits, st);
    if (a.rp == 128) return tc::launch_pass2s<128>(a, op.plane, maps, op.O_pad, splits, st);
    return DNA_ERR_UNSUPPORTED;
}

}  // namespace dna
