// tcgen05 kernels of the FP32 form on the tensor cores: every float32 operand x is held as
// two bf16 numbers, x_hi = bf16(x) and x_lo = bf16(x - x_hi), and every product as
// x_hi y_hi + x_hi y_lo + x_lo y_hi (the dropped x_lo y_lo is below 2^-16 |x y|), summed in
// float32 in tensor memory.
//
// Both kernels stream s in chunks of 128, so that the Z = X Y^t MMAs are 128 x 128 x 16
// (an N = 64 MMA occupies the tensor pipe about as long as an N = 128 one).  Warp roles
// are those of the BF16 kernels (tc_bf16.cu): a producer warp issuing TMA copies of V
// (in half chunks of 64 values of s) and of the B operands, one or two MMA-issuing
// warps, sixteen epilogue warps; the o-block's A operands (X hi and lo) sit in tensor
// memory.
//
// Pass 1 splits by accumulator to fit tensor memory: CTAs with which = 0 form q and
// accumulate A = Y^t Q (Algorithm 1 step 5), CTAs with which = 1 form qbar and accumulate
// B = (Y o Y)^t Qbar (step 10); each recomputes Z.  Q (hi, lo) overwrites Z in place: the
// epilogue warp that reads 16 columns of Z writes the 8 + 8 columns of packed Q pairs of
// the same 16 values of s back into them, which is the A operand layout of the K-step.
// Pass 2 keeps both candidates in one CTA (one Z each, copied out to registers at the top
// of every chunk).
#include <algorithm>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dna_internal.h"
#include "tc_common.cuh"

namespace dna {
namespace tc {

constexpr int SC2 = 128;   // values of s per chunk

template <int RP>
struct P1SLayout {
    static constexpr int NA = RP / 64;                     // 64-wide r-atoms of Y
    static constexpr int GST = 3, HST = 2, VST = 2;
    // G: one r-atom of Y (hi, lo) of one chunk, K-major [128 s][64 r] (GEMM1's B)
    static constexpr uint32_t G_PLANE = SC2 * 128;
    static constexpr uint32_t G_STAGE = 2 * G_PLANE;
    // H: Y^t or (Y o Y)^t (hi, lo) of one half chunk, K-major [RP r][64 s] (GEMM2's B)
    static constexpr uint32_t H_PLANE = RP * SCH * 2;
    static constexpr uint32_t H_STAGE = 2 * H_PLANE;
    // V: one half chunk, [64 s][128 o] float32
    static constexpr uint32_t V_STAGE = SCH * OBLK * 4;
    // X hi or lo of an o-block, [NA][128 o][64 r] bf16, in a G stage
    static constexpr uint32_t X_PLANE = OBLK * RP * 2;
    static_assert(X_PLANE <= G_STAGE, "an X plane fits a G stage");
    static constexpr uint32_t GR = 0;
    static constexpr uint32_t HR = GR + GST * G_STAGE;
    static constexpr uint32_t VR = HR + HST * H_STAGE;
    static constexpr uint32_t BAR = VR + VST * V_STAGE;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;
    // tensor memory columns: ZQ x 2 (Z, then Q hi / lo in place) | accumulator | X hi | X lo
    static constexpr uint32_t TACC = 2 * SC2, TXH = TACC + RP, TXL = TXH + RP / 2;
    static_assert(TXL + RP / 2 <= NCOLS, "tensor memory budget");
    static_assert(HR % 1024 == 0 && VR % 1024 == 0 && G_PLANE % 1024 == 0 &&
                      H_PLANE % 1024 == 0,
                  "tiles must be 1024-byte aligned");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};

// G stages hold X planes and r-atoms of Y in the order of P1SGCursor.  QFULL[2 b + h]:
// the epilogue wrote Q of half h (s 64 h .. 64 h + 63) of the chunk in ZQ buffer b.
// QEMPTY[b]: GEMM2 of that chunk is done (buffer b free for GEMM1 two chunks later; for a
// tile's last chunk the accumulator is final).
enum { S_GFULL = 0, S_GEMPTY = 3, S_HFULL = 6, S_HEMPTY = 8, S_VFULL = 10, S_VEMPTY = 12,
       S_ZFULL = 14, S_QFULL = 16, S_QEMPTY = 20, S_DRAIN = 22, S_COUNT = 24 };

// One tile of pass 1: the accumulator (A if which = 0, B if which = 1) of one o-block over
// one split of s.  Tiles are numbered which-major, then split, then o-block: with the
// tiles spread evenly over the CTAs, CTA i and CTA i + G / 2 work through the same
// (split, o-block) tiles at the same time, so one of them reads each V tile from L2.
struct P1STile {
    int64_t o0, s_begin, s_end;
    int nch, which, split;
};
__device__ __forceinline__ P1STile p1s_tile(int t, int nwhich, int nob, const P1Args& a) {
    P1STile x;
    const int per_which = (int)(nob * ((a.S + a.s_per - 1) / a.s_per));
    x.which = nwhich > 1 ? t / per_which : 0;
    const int rest = nwhich > 1 ? t % per_which : t;
    x.o0 = (int64_t)(rest % nob) * OBLK;
    x.split = rest / nob;
    x.s_begin = (int64_t)x.split * a.s_per;
    x.s_end = min(a.S, x.s_begin + a.s_per);
    x.nch = x.s_end > x.s_begin ? (int)((x.s_end - x.s_begin + SC2 - 1) / SC2) : 0;
    return x;
}

// A walk over the units (tile, chunk, sub) of one CTA's tiles, sub < per_chunk (every tile
// has at least one chunk: the host plans ceil(S / s_per) splits).
struct P1SCursor {
    int t, k, sub;
    P1STile x;
    __device__ __forceinline__ void start(int t0, int nwhich, int nob, const P1Args& a) {
        t = t0; k = 0; sub = 0;
        x = p1s_tile(t, nwhich, nob, a);
    }
    __device__ __forceinline__ void next(int per_chunk, int nwhich, int nob, const P1Args& a) {
        if (++sub < per_chunk) return;
        sub = 0;
        if (++k < x.nch) return;
        k = 0;
        ++t;
        x = p1s_tile(t, nwhich, nob, a);
    }
};

// The G-ring walk of one CTA: per tile the X hi and X lo planes (units 0, 1), then the
// r-atoms of every chunk (units 2 + NA k + at).
struct P1SGCursor {
    int t, u, n;
    P1STile x;
    __device__ __forceinline__ void start(int t0, int na, int nwhich, int nob, const P1Args& a) {
        t = t0; u = 0;
        x = p1s_tile(t, nwhich, nob, a);
        n = 2 + na * x.nch;
    }
    __device__ __forceinline__ void next(int na, int nwhich, int nob, const P1Args& a) {
        if (++u < n) return;
        u = 0;
        ++t;
        x = p1s_tile(t, nwhich, nob, a);
        n = 2 + na * x.nch;
    }
};

// Persistent: CTA i takes the tiles [i T / G, (i + 1) T / G) of the T = nwhich x splits x
// nob tiles (G = gridDim.x); the rings, the ZQ buffers and every barrier phase run on
// across tiles.  X (hi, lo) of each tile comes through the G ring and goes into tensor
// memory by tcgen05.cp from the MMA thread once its last GEMM1 of the previous tile is
// done; the epilogue reads a finished tile's accumulator out while the next tile starts
// (see the epilogue).
template <int RP>
__global__ void __launch_bounds__(P1_THREADS, 1)
    k_tc_pass1s(P1Args a, int nwhich, int nob, int ntiles,
                const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmXl,
                const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmYl,
                const __grid_constant__ CUtensorMap tmYt, const __grid_constant__ CUtensorMap tmYtl,
                const __grid_constant__ CUtensorMap tmY2t,
                const __grid_constant__ CUtensorMap tmY2tl,
                const __grid_constant__ CUtensorMap tmV) {
    using L = P1SLayout<RP>;
    constexpr int NA = L::NA, GST = L::GST, HST = L::HST, VST = L::VST;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + S_COUNT * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L::BAR + S_COUNT * 8 + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t_begin = (int)((int64_t)blockIdx.x * ntiles / gridDim.x);
    const int t_end = (int)((int64_t)(blockIdx.x + 1) * ntiles / gridDim.x);

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == W_PRODUCER * 32) {
        for (int i = 0; i < GST; ++i) {
            mbar_init(&bar[S_GFULL + i], 1);
            mbar_init(&bar[S_GEMPTY + i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar[S_HFULL + i], 1);
            mbar_init(&bar[S_HEMPTY + i], 1);
            mbar_init(&bar[S_VFULL + i], 1);
            mbar_init(&bar[S_VEMPTY + i], W_EPI);
            mbar_init(&bar[S_ZFULL + i], 1);
            mbar_init(&bar[S_QEMPTY + i], 1);
            mbar_init(&bar[S_DRAIN + i], 1);
        }
        for (int i = 0; i < 4; ++i) mbar_init(&bar[S_QFULL + i], W_EPI);
        *abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == W_PRODUCER) {
        // one thread services the three rings in whatever order their slots free up; each
        // ring walks the CTA's units with its own cursor
        if (lane == 0 && t_begin < t_end) {
            tma_prefetch_desc(&tmX); tma_prefetch_desc(&tmXl);
            tma_prefetch_desc(&tmY); tma_prefetch_desc(&tmYl); tma_prefetch_desc(&tmYt);
            tma_prefetch_desc(&tmYtl); tma_prefetch_desc(&tmV);
            if (nwhich > 1) { tma_prefetch_desc(&tmY2t); tma_prefetch_desc(&tmY2tl); }
            P1SGCursor cg_;
            P1SCursor ch_, cv_;
            cg_.start(t_begin, NA, nwhich, nob, a);
            ch_.start(t_begin, nwhich, nob, a);
            cv_.start(t_begin, nwhich, nob, a);
            int kg = 0, kh = 0, kv = 0;   // units issued per ring
            long long t0 = clock64();
            while (cg_.t < t_end || ch_.t < t_end || cv_.t < t_end) {
                bool prog = false;
                if (cv_.t < t_end && mbar_test(&bar[S_VEMPTY + kv % VST], ((kv / VST) & 1) ^ 1)) {
                    const int st = kv % VST;
                    mbar_arrive_expect_tx(&bar[S_VFULL + st], L::V_STAGE);
                    tma_load_2d(sbase + L::VR + st * L::V_STAGE, &tmV, (int32_t)cv_.x.o0,
                                (int32_t)(cv_.x.s_begin + (int64_t)cv_.k * SC2 + SCH * cv_.sub),
                                &bar[S_VFULL + st]);
                    ++kv;
                    cv_.next(2, nwhich, nob, a);
                    prog = true;
                }
                if (cg_.t < t_end && mbar_test(&bar[S_GEMPTY + kg % GST], ((kg / GST) & 1) ^ 1)) {
                    const int st = kg % GST;
                    const uint32_t dst = sbase + L::GR + st * L::G_STAGE;
                    if (cg_.u < 2) {   // X hi or lo of the tile's o-block, [NA][128 o][64 r]
                        mbar_arrive_expect_tx(&bar[S_GFULL + st], L::X_PLANE);
                        for (int at = 0; at < NA; ++at)
                            tma_load_2d(dst + at * OBLK * 128, cg_.u ? &tmXl : &tmX, 64 * at,
                                        (int32_t)cg_.x.o0, &bar[S_GFULL + st]);
                    } else {
                        const int ck = (cg_.u - 2) / NA, at = (cg_.u - 2) % NA;
                        const int32_t s0 = (int32_t)(cg_.x.s_begin + (int64_t)ck * SC2);
                        mbar_arrive_expect_tx(&bar[S_GFULL + st], L::G_STAGE);
                        for (int hs = 0; hs < 2; ++hs) {
                            tma_load_2d(dst + hs * SCH * 128, &tmY, 64 * at, s0 + SCH * hs,
                                        &bar[S_GFULL + st]);
                            tma_load_2d(dst + L::G_PLANE + hs * SCH * 128, &tmYl, 64 * at,
                                        s0 + SCH * hs, &bar[S_GFULL + st]);
                        }
                    }
                    ++kg;
                    cg_.next(NA, nwhich, nob, a);
                    prog = true;
                }
                if (ch_.t < t_end && mbar_test(&bar[S_HEMPTY + kh % HST], ((kh / HST) & 1) ^ 1)) {
                    const int st = kh % HST;
                    const uint32_t dst = sbase + L::HR + st * L::H_STAGE;
                    const int32_t s0 =
                        (int32_t)(ch_.x.s_begin + (int64_t)ch_.k * SC2 + SCH * ch_.sub);
                    const CUtensorMap* mh = ch_.x.which ? &tmY2t : &tmYt;
                    const CUtensorMap* ml = ch_.x.which ? &tmY2tl : &tmYtl;
                    mbar_arrive_expect_tx(&bar[S_HFULL + st], L::H_STAGE);
                    tma_load_2d(dst, mh, s0, 0, &bar[S_HFULL + st]);
                    tma_load_2d(dst + L::H_PLANE, ml, s0, 0, &bar[S_HFULL + st]);
                    ++kh;
                    ch_.next(2, nwhich, nob, a);
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
                for (int k = max(0, kg - GST); k < kg; ++k)
                    drain_phase(&bar[S_GFULL + k % GST], (k / GST) & 1);
                for (int k = max(0, kh - HST); k < kh; ++k)
                    drain_phase(&bar[S_HFULL + k % HST], (k / HST) & 1);
            }
        }
    } else if (warp == W_MMA_Z) {
        // Z(m) = X Y(m)^t as x_hi y_hi + x_hi y_lo + x_lo y_hi, into ZQ buffer m & 1 (m counts
        // the CTA's chunks); per r-atom the three products are issued outer and the K-steps
        // inner (back-to-back MMAs into one accumulator with the same K-slice run the
        // tensor pipe at about 3/4 rate)
        if (lane == 0) {
            bool ok = true;
            int m = 0, j = 0;
            constexpr uint32_t idesc = idesc_bf16(OBLK, SC2);
            for (int t = t_begin; ok && t < t_end; ++t) {
                const P1STile x = p1s_tile(t, nwhich, nob, a);
                // X of the tile into tensor memory once GEMM1 of the previous tile's last
                // chunk (this thread's own MMAs) has finished reading the old X
                if (m >= 1 &&
                    !(ok = wait_phase(&bar[S_ZFULL + ((m - 1) & 1)], ((m - 1) >> 1) & 1, abort)))
                    break;
#pragma unroll 1
                for (int pl = 0; pl < 2; ++pl, ++j) {
                    if (!(ok = wait_phase(&bar[S_GFULL + j % GST], (j / GST) & 1, abort))) break;
                    tc_fence_after();
                    const uint32_t xs = sbase + L::GR + (j % GST) * L::G_STAGE;
#pragma unroll
                    for (int kk = 0; kk < RP / 16; ++kk)
                        tmem_cp_128x256b(tmem + (pl ? L::TXL : L::TXH) + 8 * kk,
                                         desc_sw128(xs + (kk >> 2) * OBLK * 128 + 32u * (kk & 3)));
                    mma_commit(&bar[S_GEMPTY + j % GST]);
                }
                for (int k = 0; ok && k < x.nch; ++k, ++m) {
                    const int b = m & 1;
                    // GEMM2 of chunk m - 2 has read its Q from this buffer
                    if (m >= 2 &&
                        !(ok = wait_phase(&bar[S_QEMPTY + b], ((m - 2) >> 1) & 1, abort)))
                        break;
                    const uint32_t tz = tmem + b * SC2;
#pragma unroll 1
                    for (int at = 0; at < NA; ++at, ++j) {
                        if (!(ok = wait_phase(&bar[S_GFULL + j % GST], (j / GST) & 1, abort)))
                            break;
                        tc_fence_after();
                        const uint32_t gh = sbase + L::GR + (j % GST) * L::G_STAGE,
                                       gl = gh + L::G_PLANE;
                        const uint32_t xh = tmem + L::TXH + 32 * at, xl = tmem + L::TXL + 32 * at;
#pragma unroll
                        for (int p = 0; p < 3; ++p)
#pragma unroll
                            for (int kq = 0; kq < 4; ++kq)
                                mma_bf16_tmem_a(tz, (p == 2 ? xl : xh) + 8 * kq,
                                                desc_sw128((p == 1 ? gl : gh) + 32u * kq), idesc,
                                                (at > 0 || p > 0 || kq > 0) ? 1u : 0u);
                        mma_commit(&bar[S_GEMPTY + j % GST]);
                    }
                    if (ok) mma_commit(&bar[S_ZFULL + b]);
                }
            }
            if (!ok) {
                mma_commit(&bar[S_DRAIN + 0]);
                drain_phase(&bar[S_DRAIN + 0], 0);
            }
        }
    } else if (warp == W_MMA_AB) {
        // accumulator += Q(m) H(m) as q_hi h_hi + q_hi h_lo + q_lo h_hi, one half chunk at a
        // time, products outer; the first MMA of a tile overwrites the accumulator, which
        // the epilogue has copied out before it signals the first Q of the tile
        if (lane == 0) {
            bool ok = true;
            int m = 0;
            constexpr uint32_t idesc = idesc_bf16(OBLK, RP);
            for (int t = t_begin; ok && t < t_end; ++t) {
                const int nch = p1s_tile(t, nwhich, nob, a).nch;
                for (int k = 0; ok && k < nch; ++k, ++m) {
                    const int b = m & 1;
#pragma unroll 1
                    for (int h = 0; ok && h < 2; ++h) {
                        const int jh = 2 * m + h;
                        if (!(ok = wait_phase(&bar[S_QFULL + 2 * b + h], (m >> 1) & 1, abort)))
                            break;
                        if (!(ok = wait_phase(&bar[S_HFULL + jh % HST], (jh / HST) & 1, abort)))
                            break;
                        tc_fence_after();
                        const uint32_t th = sbase + L::HR + (jh % HST) * L::H_STAGE,
                                       tl = th + L::H_PLANE;
                        const uint32_t q0 = tmem + b * SC2 + 64 * h;
#pragma unroll
                        for (int p = 0; p < 3; ++p)
#pragma unroll
                            for (int kq = 0; kq < SCH / 16; ++kq) {
                                const uint32_t acc = (k > 0 || h > 0 || p > 0 || kq > 0) ? 1u : 0u;
                                mma_bf16_tmem_a(tmem + L::TACC, q0 + 16 * kq + (p == 2 ? 8 : 0),
                                                desc_sw128((p == 1 ? tl : th) + 32u * kq), idesc,
                                                acc);
                            }
                        mma_commit(&bar[S_HEMPTY + jh % HST]);
                    }
                    if (ok) mma_commit(&bar[S_QEMPTY + b]);
                }
            }
            if (!ok) {
                mma_commit(&bar[S_DRAIN + 1]);
                drain_phase(&bar[S_DRAIN + 1], 0);
            }
        }
    } else {
        // epilogue warps 0-15: lane quadrant qd = warp % 4 (o = o0 + 32 qd + lane); in half h
        // of a chunk the warp takes the K-step kk = 4 h + cg (cg = warp / 4), i.e. the 16
        // values s = 64 h + 16 cg .. + 15 and the ZQ columns 16 kk .. 16 kk + 15
        const int qd = warp & 3, cg = warp >> 2;
        const int row = 32 * qd + lane;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        float zmin = 1.f;   // min over v > 0 of z (see the BF16 pass 1)
        bool ok = true;
        int m = 0;
        // The accumulator of a finished tile is copied out while the next tile starts: after
        // the epilogue has written Q of the next tile's first half chunk (its QFULL not yet
        // signalled), it waits for the old tile's last GEMM2, reads the accumulator into
        // registers, signals QFULL (the first GEMM2 of the new tile overwrites the
        // accumulator) and only then issues the global stores.
        bool pend = false;   // an accumulator still to copy: tile xp, last chunk mp
        P1STile xp{};
        int mp = 0;
        // this thread's 32 accumulator values of tile y (column group cg) to Apart / Bpart
        auto store_acc = [&](const P1STile& y, const uint32_t (&r32)[32]) {
            const int64_t o = y.o0 + row;
            const int64_t base = (int64_t)y.split * a.R;
            float* dst = y.which ? a.Bpart : a.Apart;
            if (o < a.O)
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int64_t r = 32 * cg + i;
                    if (r < a.R) dst[(base + r) * a.O + o] = __uint_as_float(r32[i]);
                }
        };
        for (int t = t_begin; ok && t < t_end; ++t) {
            const P1STile x = p1s_tile(t, nwhich, nob, a);
            for (int k = 0; k < x.nch; ++k, ++m) {
                const int b = m & 1;
                ok = wait_phase(&bar[S_ZFULL + b], (m >> 1) & 1, abort);
                if (!(ok = __all_sync(0xffffffffu, ok))) break;   // keep the warp converged
                tc_fence_after();
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    const int kv = 2 * m + h, vs = kv % VST;
                    ok = wait_phase(&bar[S_VFULL + vs], (kv / VST) & 1, abort);
                    if (!(ok = __all_sync(0xffffffffu, ok))) break;
                    const uint32_t col = tmem + b * SC2 + 64 * h + 16 * cg + lane_off;
                    uint32_t zr[16];
                    tmem_ld16(col, zr);
                    // V rows s = 16 cg + j of this half; TMA zero-fills v outside the problem
                    const float* Vs = reinterpret_cast<const float*>(sm + L::VR + vs * L::V_STAGE) +
                                      16 * cg * OBLK + row;
                    float vv[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) vv[j] = Vs[j * OBLK];
                    tmem_ld_wait();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar[S_VEMPTY + vs]);
                    uint32_t hp[8], lp[8];
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        float w[2];
#pragma unroll
                        for (int tt = 0; tt < 2; ++tt) {
                            const float v = vv[j + tt];
                            const float z = __uint_as_float(zr[j + tt]);
                            const float rz = rcp_ftz(z);
                            const bool pos = v > 0.f;
                            zmin = fminf(zmin, pos ? z : 1.f);
                            const float q = v * rz;
                            w[tt] = pos ? (x.which ? q * rz : q) : 0.f;   // q, or qbar = q / z
                        }
                        split2(w[0], w[1], hp[j / 2], lp[j / 2]);
                    }
                    tmem_st8(col, hp);
                    tmem_st8(col + 8, lp);
                    tmem_st_wait();
                    uint32_t r32[32];
                    const bool copy = pend && k == 0 && h == 0;
                    if (copy) {   // the previous tile's accumulator, once its last GEMM2 is done
                        ok = __all_sync(0xffffffffu, wait_phase(&bar[S_QEMPTY + (mp & 1)],
                                                                (mp >> 1) & 1, abort));
                        if (!ok) break;
                        tc_fence_after();
                        if (cg < RP / 32) {
                            tmem_ld32(tmem + L::TACC + lane_off + 32 * cg, r32);
                            tmem_ld_wait();
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar[S_QFULL + 2 * b + h]);
                    if (copy) {
                        if (cg < RP / 32) store_acc(xp, r32);
                        pend = false;
                    }
                }
                if (!ok) break;
            }
            if (!ok) break;
            if (t + 1 < t_end) {   // copied out during the next tile's first half chunk
                pend = true;
                xp = x;
                mp = m - 1;
                continue;
            }
            // the CTA's last tile: GEMM2 of its last chunk done, copy the accumulator out
            const int ml = m - 1;
            ok = __all_sync(0xffffffffu,
                            wait_phase(&bar[S_QEMPTY + (ml & 1)], (ml >> 1) & 1, abort));
            if (!ok) break;
            tc_fence_after();
            if (cg < RP / 32) {
                uint32_t r32[32];
                tmem_ld32(tmem + L::TACC + lane_off + 32 * cg, r32);
                tmem_ld_wait();
                store_acc(x, r32);
            }
            tc_fence_before();
        }
        if (!(zmin >= FLT_MIN_NORMAL)) atomicOr(a.status, STATUS_NONFINITE);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(a.status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

// Pass 2 of the split form: Z_MU and Z_DNA from hi / lo candidates and a hi / lo Y in one
// CTA, which reads each Y and V tile once for both.  Tensor memory holds one Z per
// candidate (128 columns each) next to the four X planes; the epilogue copies both Z
// into registers at the top of a chunk and frees them, so the MMAs of the next chunk run
// while it computes.  One MMA-issuing warp per candidate.  Shared memory: G ring (Y hi /
// lo of a chunk, or the X planes of an o-block; 2 stages), V ring (3 half chunks).
//
// Persistent with balanced work: the units (o-block, chunk of 128 values of s) are
// numbered o-block-major and CTA i takes the units [i U / G, (i + 1) U / G) (U units, G
// CTAs), so every SM streams the same number of chunks.  A CTA's run splits into segments
// of one o-block; at the start of a segment the X planes come through the G ring and go
// into tensor memory by tcgen05.cp, at its end every epilogue thread writes its cost sums
// to slot 4 q + cg of the o-block (q = the CTA's rank among the o-block's CTAs), and the
// o-block's last CTA writes zeros into the slots no CTA uses: a fixed number of slots per
// column for the selection kernel to add in order.
template <int RP, int NP>
struct P2SLayout {
    static constexpr int GST = 2, VST = 3;
    static constexpr uint32_t G_PLANE = SC2 * RP * 2;   // [RP / 64 atoms][128 s][64 r] bf16
    static constexpr uint32_t G_STAGE = NP * G_PLANE;
    static constexpr uint32_t X_PLANE = OBLK * RP * 2;  // [RP / 64 atoms][128 o][64 r] bf16
    static constexpr uint32_t V_STAGE = SCH * OBLK * 4;
    static constexpr uint32_t GR = 0;
    static constexpr uint32_t VR = GR + GST * G_STAGE;
    static constexpr uint32_t BAR = VR + VST * V_STAGE;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;
    // tensor memory: Z_mu | Z_dna | X_mu hi (| X_mu lo) | X_dna hi (| X_dna lo)
    static constexpr uint32_t TX = 2 * SC2, XC = NP * RP / 2;   // XC: columns per candidate
    static_assert(TX + 2 * XC <= NCOLS, "tensor memory budget");
    static_assert(NP * X_PLANE <= G_STAGE, "one candidate's X planes fit a G stage");
    static_assert(G_PLANE % 1024 == 0 && VR % 1024 == 0, "tiles must be 1024-byte aligned");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};

// ZFULL[c] / ZEMPTY[c]: Z of candidate c written / copied out (one phase per chunk);
// GEMPTY[st]: both candidates' MMAs (or X copies) from G stage st are done (2 arrivals).
enum { T_GFULL = 0, T_GEMPTY = 2, T_VFULL = 4, T_VEMPTY = 7, T_ZFULL = 10, T_ZEMPTY = 12,
       T_DRAIN = 14, T_COUNT = 16 };

// The CTA (of G) whose unit range [i U / G, (i + 1) U / G) holds unit u.
__host__ __device__ __forceinline__ int p2s_cta_of(int64_t u, int64_t U, int G) {
    return (int)(((u + 1) * G + U - 1) / U - 1);
}

// One CTA's walk over its units in G-ring order: per segment the two X units (MU, DNA
// planes), then its chunks.
struct P2SGCursor {
    int64_t u, u1, nch;
    int xu;   // 0, 1: X units of the segment starting at u; 2: chunk u
    __device__ __forceinline__ bool done() const { return u >= u1; }
    __device__ __forceinline__ void next() {
        if (xu < 2) { ++xu; return; }          // X MU, X DNA, then chunk u
        ++u;
        xu = (u < u1 && u % nch == 0) ? 0 : 2;   // a new o-block: its X first
    }
};

// NP: operand planes, 2 for the split FP32 form (three products), 1 for the BF16 form.
// FULL: d_KL per column instead (eq. 1 terms z + v log(v / z) - v with the accurate
// logarithm), both candidates = the current factor, slot layout [slot][O] of candidate 0.
// The work of CTA `me` of the G CTAs that share one problem's units; the tensor maps may
// live in kernel parameters or in global memory (the grouped form).
template <int RP, int NP, bool FULL>
__device__ __forceinline__ void pass2s_body(const P2Args& a, int64_t nch, int64_t U, int slots,
                                            int me, int G, const CUtensorMap* pXm,
                                            const CUtensorMap* pXml, const CUtensorMap* pXd,
                                            const CUtensorMap* pXdl, const CUtensorMap* pY,
                                            const CUtensorMap* pYl, const CUtensorMap* pV) {
    using L = P2SLayout<RP, NP>;
    constexpr int GST = L::GST, VST = L::VST;
    static_assert(NP == 2 || !FULL, "the d_KL mode runs in the split form");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + T_COUNT * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L::BAR + T_COUNT * 8 + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t u0 = (int64_t)me * U / G, u1 = (int64_t)(me + 1) * U / G;

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == W_PRODUCER * 32) {
        for (int i = 0; i < VST; ++i) {
            mbar_init(&bar[T_VFULL + i], 1);
            mbar_init(&bar[T_VEMPTY + i], W_EPI);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar[T_GFULL + i], 1);
            mbar_init(&bar[T_GEMPTY + i], 2);
            mbar_init(&bar[T_ZFULL + i], 1);
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
        if (lane == 0 && u0 < u1) {
            tma_prefetch_desc(pXm); tma_prefetch_desc(pXml); tma_prefetch_desc(pXd);
            tma_prefetch_desc(pXdl); tma_prefetch_desc(pY); tma_prefetch_desc(pYl);
            tma_prefetch_desc(pV);
            P2SGCursor cg_{u0, u1, nch, 0};
            int64_t uv = u0;   // V: half h of unit uv
            int hv = 0, kg = 0, kv = 0;
            long long t0 = clock64();
            while (!cg_.done() || uv < u1) {
                bool prog = false;
                if (uv < u1 && mbar_test(&bar[T_VEMPTY + kv % VST], ((kv / VST) & 1) ^ 1)) {
                    const int st = kv % VST;
                    const int64_t ob = uv / nch, ck = uv % nch;
                    mbar_arrive_expect_tx(&bar[T_VFULL + st], L::V_STAGE);
                    tma_load_2d(sbase + L::VR + st * L::V_STAGE, pV, (int32_t)(ob * OBLK),
                                (int32_t)(ck * SC2 + SCH * hv), &bar[T_VFULL + st]);
                    ++kv;
                    if (++hv == 2) { hv = 0; ++uv; }
                    prog = true;
                }
                if (!cg_.done() && mbar_test(&bar[T_GEMPTY + kg % GST], ((kg / GST) & 1) ^ 1)) {
                    const int st = kg % GST;
                    const uint32_t dst = sbase + L::GR + st * L::G_STAGE;
                    const int64_t ob = cg_.u / nch, ck = cg_.u % nch;
                    if (cg_.xu < 2) {   // X hi (and lo) of candidate xu, [NA][128 o][64 r] each
                        const CUtensorMap* mh = cg_.xu ? pXd : pXm;
                        const CUtensorMap* ml = cg_.xu ? pXdl : pXml;
                        mbar_arrive_expect_tx(&bar[T_GFULL + st], NP * L::X_PLANE);
                        for (int at = 0; at < RP / 64; ++at) {
                            tma_load_2d(dst + at * OBLK * 128, mh, 64 * at, (int32_t)(ob * OBLK),
                                        &bar[T_GFULL + st]);
                            if (NP == 2)
                                tma_load_2d(dst + L::X_PLANE + at * OBLK * 128, ml, 64 * at,
                                            (int32_t)(ob * OBLK), &bar[T_GFULL + st]);
                        }
                    } else {
                        const int32_t s0 = (int32_t)(ck * SC2);
                        mbar_arrive_expect_tx(&bar[T_GFULL + st], L::G_STAGE);
                        for (int at = 0; at < RP / 64; ++at)
                            for (int hs = 0; hs < 2; ++hs) {
                                const uint32_t off = at * SC2 * 128 + hs * SCH * 128;
                                tma_load_2d(dst + off, pY, 64 * at, s0 + SCH * hs,
                                            &bar[T_GFULL + st]);
                                if (NP == 2)
                                    tma_load_2d(dst + L::G_PLANE + off, pYl, 64 * at,
                                                s0 + SCH * hs, &bar[T_GFULL + st]);
                            }
                    }
                    ++kg;
                    cg_.next();
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
                for (int k = max(0, kg - GST); k < kg; ++k)
                    drain_phase(&bar[T_GFULL + k % GST], (k / GST) & 1);
            }
        }
    } else if (warp == W_MMA_Z || warp == W_MMA_AB) {
        // candidate c: Z_c(m) = X_c Y(m)^t (in the split form three products, outer; see
        // pass 1); at each segment start X_c (from the G unit of candidate c) into tensor
        // memory
        const int c = warp == W_MMA_AB ? 1 : 0;
        if (lane == 0 && u0 < u1) {
            bool ok = true;
            const uint32_t xh = tmem + L::TX + (uint32_t)c * L::XC, xl = xh + RP / 2;
            const uint32_t tz = tmem + (uint32_t)c * SC2;
            constexpr uint32_t idesc = idesc_bf16(OBLK, SC2);
            int j = 0, m = 0;   // G units and chunks consumed
            for (int64_t u = u0; ok && u < u1; ++u, ++m) {
                if (u == u0 || u % nch == 0) {
                    // this thread's previous MMAs have read the old X
                    if (m >= 1 && !(ok = wait_phase(&bar[T_ZFULL + c], (m - 1) & 1, abort))) break;
#pragma unroll 1
                    for (int xu = 0; xu < 2; ++xu, ++j) {
                        if (!(ok = wait_phase(&bar[T_GFULL + j % GST], (j / GST) & 1, abort)))
                            break;
                        if (xu == c) {
                            tc_fence_after();
                            const uint32_t xs = sbase + L::GR + (j % GST) * L::G_STAGE;
#pragma unroll
                            for (int pl = 0; pl < NP; ++pl)
#pragma unroll
                                for (int kk = 0; kk < RP / 16; ++kk)
                                    tmem_cp_128x256b((pl ? xl : xh) + 8 * kk,
                                                     desc_sw128(xs + pl * L::X_PLANE +
                                                                (kk >> 2) * OBLK * 128 +
                                                                32u * (kk & 3)));
                        }
                        mma_commit(&bar[T_GEMPTY + j % GST]);
                    }
                    if (!ok) break;
                }
                const int st = j % GST;
                if (!(ok = wait_phase(&bar[T_GFULL + st], (j / GST) & 1, abort))) break;
                // the epilogue has copied out Z_c of the previous chunk
                if (m >= 1 && !(ok = wait_phase(&bar[T_ZEMPTY + c], (m - 1) & 1, abort))) break;
                tc_fence_after();
                const uint32_t gh = sbase + L::GR + st * L::G_STAGE, gl = gh + L::G_PLANE;
#pragma unroll
                for (int p = 0; p < (NP == 2 ? 3 : 1); ++p)
#pragma unroll
                    for (int kk = 0; kk < RP / 16; ++kk) {
                        const uint32_t off = (kk >> 2) * SC2 * 128 + 32u * (kk & 3);
                        mma_bf16_tmem_a(tz, (p == 2 ? xl : xh) + 8 * kk,
                                        desc_sw128((p == 1 ? gl : gh) + off), idesc,
                                        (p > 0 || kk > 0) ? 1u : 0u);
                    }
                mma_commit(&bar[T_GEMPTY + st]);
                mma_commit(&bar[T_ZFULL + c]);
                ++j;
            }
            if (!ok) {
                mma_commit(&bar[T_DRAIN + c]);
                drain_phase(&bar[T_DRAIN + c], 0);
            }
        }
    } else if (warp < W_EPI) {
        // epilogue warp: lanes o = o0 + 32 qd + lane, in half h the 16 values
        // s = 64 h + 16 cg .. + 15 of the chunk
        const int qd = warp & 3, cg = warp >> 2;
        const int row = 32 * qd + lane;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        double acc_m = 0.0, acc_d = 0.0;
        bool ok = true, finite = true;
        int m = 0;
        for (int64_t u = u0; u < u1; ++u, ++m) {
            ok = wait_phase(&bar[T_ZFULL + 0], m & 1, abort);
            ok = ok && wait_phase(&bar[T_ZFULL + 1], m & 1, abort);
            if (!(ok = __all_sync(0xffffffffu, ok))) break;   // keep the warp converged
            tc_fence_after();
            const uint32_t tz = tmem + 16 * cg + lane_off;
            uint32_t zm[2][16], zd[2][16];
            tmem_ld16(tz, zm[0]);
            tmem_ld16(tz + SCH, zm[1]);
            tmem_ld16(tz + SC2, zd[0]);
            tmem_ld16(tz + SC2 + SCH, zd[1]);
            tmem_ld_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&bar[T_ZEMPTY + 0]);
                mbar_arrive(&bar[T_ZEMPTY + 1]);
            }
            float run_m = 0.f, run_d = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kv = 2 * m + h, vs = kv % VST;
                ok = wait_phase(&bar[T_VFULL + vs], (kv / VST) & 1, abort);
                if (!(ok = __all_sync(0xffffffffu, ok))) break;
                // V rows s = 16 cg + j of this half; TMA zero-fills v beyond S, where Y is
                // zero too (z = 0, no cost)
                const float* Vs = reinterpret_cast<const float*>(sm + L::VR + vs * L::V_STAGE) +
                                  16 * cg * OBLK + row;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const float v = Vs[jj * OBLK];
                    const float z1 = __uint_as_float(zm[h][jj]), z2 = __uint_as_float(zd[h][jj]);
                    const bool pos = v > 0.f;
                    if constexpr (FULL) {
                        run_m += pos ? z1 + v * logf(v / z1) - v : z1;
                    } else {
                        // ln z = ln 2 log2 z with the hardware log2 (relative error about
                        // 2^-22): well inside the split form's 1e-4 near-tie margin
                        run_m += pos ? z1 - v * (LN2F * lg2_ftz(z1)) : z1;
                        run_d += pos ? z2 - v * (LN2F * lg2_ftz(z2)) : z2;
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[T_VEMPTY + vs]);
            }
            if (!ok) break;
            acc_m += (double)run_m;
            acc_d += (double)run_d;
            // end of a segment: this thread's cost sums of the o-block into its slot
            if (FULL && ((u + 1) % nch == 0 || u + 1 == u1)) {
                const int64_t ob = u / nch, o = ob * OBLK + row;
                finite = finite && fabs(acc_m) < INFINITY;
                const int q = me - p2s_cta_of(ob * nch, U, G);
                if (o < a.O) {
                    a.dpart[(int64_t)(4 * q + cg) * a.O + o] = acc_m;
                    if (me == p2s_cta_of((ob + 1) * nch - 1, U, G))
                        for (int s = 4 * (q + 1) + cg; s < slots; s += 4)
                            a.dpart[(int64_t)s * a.O + o] = 0.0;
                }
                acc_m = 0.0;
                acc_d = 0.0;
            } else if ((u + 1) % nch == 0 || u + 1 == u1) {
                const int64_t ob = u / nch, o = ob * OBLK + row;
                finite = finite && fabs(acc_m) < INFINITY && fabs(acc_d) < INFINITY;
                const int q = me - p2s_cta_of(ob * nch, U, G);
                if (o < a.O) {
                    a.dpart[((int64_t)(4 * q + cg) * 2 + 0) * a.O + o] = acc_m;
                    a.dpart[((int64_t)(4 * q + cg) * 2 + 1) * a.O + o] = acc_d;
                    // the o-block's last CTA: zeros in the slots no CTA of it uses
                    const int last = p2s_cta_of((ob + 1) * nch - 1, U, G);
                    if (me == last)
                        for (int s = 4 * (q + 1) + cg; s < slots; s += 4) {
                            a.dpart[((int64_t)s * 2 + 0) * a.O + o] = 0.0;
                            a.dpart[((int64_t)s * 2 + 1) * a.O + o] = 0.0;
                        }
                }
                acc_m = 0.0;
                acc_d = 0.0;
            }
        }
        if (!finite) atomicOr(a.status, STATUS_NONFINITE);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(a.status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

template <int RP>
int launch_pass1s(const P1Args& a, bool with_b, const TcMaps& m, int64_t O_pad, int splits,
                  int ctas, cudaStream_t st) {
    const uint32_t smem = P1SLayout<RP>::TOTAL + 1024;
    auto k = k_tc_pass1s<RP>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    const int nwhich = with_b ? 2 : 1;
    const int nob = (int)(O_pad / OBLK);
    const int ntiles = nwhich * nob * splits;
    if (ntiles == 0) return DNA_OK;
    const int grid = ctas > 0 ? std::min(ctas, ntiles) : ntiles;
    k<<<grid, P1_THREADS, smem, st>>>(a, nwhich, nob, ntiles, m.x, m.x_l, m.y, m.y_l, m.yt,
                                       m.yt_l, m.y2t, m.y2t_l, m.v);
    return after_launch();
}

template <int RP, int NP, bool FULL>
__global__ void __launch_bounds__(P1_THREADS, 1)
    k_tc_pass2s(P2Args a, int64_t nch, int64_t U, int slots,
                const __grid_constant__ CUtensorMap tmXm, const __grid_constant__ CUtensorMap tmXml,
                const __grid_constant__ CUtensorMap tmXd, const __grid_constant__ CUtensorMap tmXdl,
                const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmYl,
                const __grid_constant__ CUtensorMap tmV) {
    pass2s_body<RP, NP, FULL>(a, nch, U, slots, (int)blockIdx.x, (int)gridDim.x, &tmXm, &tmXml,
                              &tmXd, &tmXdl, &tmY, &tmYl, &tmV);
}

// Grouped pass 2 of the BF16 form: CTA i is rank ctas[i].y of the ctas[i].z CTAs that
// share problem ctas[i].x's units (view w), with that problem's tensor maps (global memory).
template <int RP>
__global__ void __launch_bounds__(P1_THREADS, 1)
    k_tc_gpass2(const TcGView* __restrict__ gv, const int4* __restrict__ ctas, int w,
                int* status) {
    const int4 c = ctas[blockIdx.x];
    const TcGView& v = gv[2 * c.x + w];
    P2Args a{};
    a.S = v.S; a.O = v.O; a.R = v.R; a.s_per = 0;
    a.dpart = v.dpart; a.status = status;
    a.Xm = v.Xmk; a.Xd = v.Xdk; a.rp = RP;
    pass2s_body<RP, 1, false>(a, v.nch2, v.U2, v.slots2, c.y, c.z, &v.xm, &v.xm, &v.xd, &v.xd,
                              &v.y, &v.y, &v.v);
}

template <int RP, int NP, bool FULL>
int launch_pass2s(const P2Args& a, const TcMaps& m, int64_t O_pad, int slots, int ctas,
                  cudaStream_t st) {
    const uint32_t smem = P2SLayout<RP, NP>::TOTAL + 1024;
    auto k = k_tc_pass2s<RP, NP, FULL>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    const int64_t nch = (a.S + SC2 - 1) / SC2, U = (O_pad / OBLK) * nch;
    if (U == 0) return DNA_OK;
    const int grid = (int)std::min<int64_t>(ctas > 0 ? ctas : U, U);
    // d_KL: both "candidates" are the current factor, the X operand of the view; the BF16
    // form (NP = 1) has no lo planes (their slots take the hi maps, unused)
    const CUtensorMap& xm = FULL ? m.x : m.xm;
    const CUtensorMap& xml = FULL ? m.x_l : NP == 2 ? m.xm_l : m.xm;
    const CUtensorMap& xd = FULL ? m.x : m.xd;
    const CUtensorMap& xdl = FULL ? m.x_l : NP == 2 ? m.xd_l : m.xd;
    const CUtensorMap& yl = NP == 2 ? m.y_l : m.y;
    k<<<grid, P1_THREADS, smem, st>>>(a, nch, U, slots, xm, xml, xd, xdl, m.y, yl, m.v);
    return after_launch();
}

}  // namespace tc

int TcBf16::pass1_split(const TcOperands& op, const TcMaps& maps, float* Apart, float* Bpart,
                        int splits, int64_t s_per, bool with_b, int* status, cudaStream_t st) {
    tc::P1Args a{};
    a.S = op.S; a.O = op.O; a.R = op.R; a.s_per = s_per;
    a.Apart = Apart; a.Bpart = Bpart; a.status = status;
    a.V = op.V; a.vs = op.vs; a.X = op.Xk; a.rp = rank_pad(op.R);
    if (a.rp == 64)
        return tc::launch_pass1s<64>(a, with_b, maps, op.O_pad, splits, op.ctas, st);
    if (a.rp == 128)
        return tc::launch_pass1s<128>(a, with_b, maps, op.O_pad, splits, op.ctas, st);
    if (a.rp == 256 || a.rp == 512)   // ratios + contraction kernels (tc_mats.cu)
        return pass1_mats(op, maps, Apart, Bpart, splits, s_per, with_b, status, st);
    return DNA_ERR_UNSUPPORTED;
}

int TcBf16::pass2_split(const TcOperands& op, const TcMaps& maps, double* dpart, int slots,
                        int* status, cudaStream_t st) {
    tc::P2Args a{};
    a.S = op.S; a.O = op.O; a.R = op.R; a.s_per = 0;
    a.dpart = dpart; a.status = status;
    a.V = op.V; a.vs = op.vs; a.Xm = op.Xmk; a.Xd = op.Xdk; a.rp = rank_pad(op.R);
    if (slots != pass2_split_slots(op.O_pad, op.S, op.ctas)) return DNA_ERR_ARG;
    const int64_t Op = op.O_pad;
    if (op.plane) {   // split FP32 form
        if (a.rp == 64) return tc::launch_pass2s<64, 2, false>(a, maps, Op, slots, op.ctas, st);
        if (a.rp == 128) return tc::launch_pass2s<128, 2, false>(a, maps, Op, slots, op.ctas, st);
    } else {          // BF16 form
        if (a.rp == 64) return tc::launch_pass2s<64, 1, false>(a, maps, Op, slots, op.ctas, st);
        if (a.rp == 128) return tc::launch_pass2s<128, 1, false>(a, maps, Op, slots, op.ctas, st);
        if (a.rp == 256) return tc::launch_pass2s<256, 1, false>(a, maps, Op, slots, op.ctas, st);
    }
    return DNA_ERR_UNSUPPORTED;
}

int TcBf16::kl_split(const TcOperands& op, const TcMaps& maps, double* dpart, int slots,
                     int* status, cudaStream_t st) {
    tc::P2Args a{};
    a.S = op.S; a.O = op.O; a.R = op.R; a.s_per = 0;
    a.dpart = dpart; a.status = status;
    a.V = op.V; a.vs = op.vs; a.rp = rank_pad(op.R);
    if (slots != pass2_split_slots(op.O_pad, op.S, op.ctas)) return DNA_ERR_ARG;
    if (!op.plane) return DNA_ERR_UNSUPPORTED;
    if (a.rp == 64) return tc::launch_pass2s<64, 2, true>(a, maps, op.O_pad, slots, op.ctas, st);
    if (a.rp == 128) return tc::launch_pass2s<128, 2, true>(a, maps, op.O_pad, slots, op.ctas, st);
    return DNA_ERR_UNSUPPORTED;
}

int TcBf16::group_pass2(const TcGView* gv, const void* ctas, int n, int w, int* status,
                        cudaStream_t st) {
    if (n <= 0) return DNA_OK;
    const uint32_t smem = tc::P2SLayout<64, 1>::TOTAL + 1024;
    tc::k_tc_gpass2<64><<<n, tc::P1_THREADS, smem, st>>>(gv, static_cast<const int4*>(ctas), w,
                                                         status);
    return after_launch();
}

int TcBf16::group_prepare_pass2() {
    const int smem = (int)(tc::P2SLayout<64, 1>::TOTAL + 1024);
    return cudaFuncSetAttribute(tc::k_tc_gpass2<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem) == cudaSuccess
               ? DNA_OK
               : DNA_ERR_CUDA;
}

int TcBf16::pass2_split_slots(int64_t O_pad, int64_t S, int ctas) {
    const int64_t nch = (S + tc::SC2 - 1) / tc::SC2, nob = O_pad / tc::OBLK, U = nob * nch;
    if (U == 0) return 4;
    const int G = (int)std::min<int64_t>(ctas > 0 ? ctas : U, U);
    int most = 1;
    for (int64_t ob = 0; ob < nob; ++ob)
        most = std::max(most, tc::p2s_cta_of((ob + 1) * nch - 1, U, G) -
                                  tc::p2s_cta_of(ob * nch, U, G) + 1);
    return 4 * most;
}

}  // namespace dna
