// tcgen05 pass 1 of the FP32 form on the tensor cores (every operand split into hi + lo
// bf16 planes, three MMAs per product: hi hi + hi lo + lo hi) at padded rank RP in
// {256, 512}; Algorithm 1 steps 2-5 and 10.  Two kernels, as in the BF16 form at these
// ranks (tc_mat.cu):
//
//   ratios    Z[o, s] = sum_r X[o, r] Y[s, r] once per (o-block, chunk of 128 values of s):
//             X hi resident in tensor memory (the A operand, RP / 2 columns), X lo and Y hi,
//             Y lo streamed through a ring of 64-wide K-slices by TMA (X lo is the A operand
//             of the lo-hi product from shared memory: tensor memory holds X hi and the two
//             Z buffers, not X lo at RP = 512); the epilogue reads V from global memory a
//             half chunk ahead, forms q = v / z and qbar = q / z in float32 and writes their
//             hi and lo bf16 planes (Q[o][s], Qbar[o][s]) to a workspace through a ring of
//             three staging buffers stored by TMA;
//   contract  A[o, r] += sum_s Q[o, s] Yt[r, s] (CTAs of which = 0) and
//             B[o, r] += sum_s Qbar[o, s] Y2t[r, s] (which = 1) over (o-block, 256-wide
//             r-block, split of s) tiles, the three products per K-step into one 128 x 256
//             accumulator, written per split ([split][R][O]).  The tensor pipe's float32
//             accumulation is not round-to-nearest, so one accumulation covers at most 1024
//             values of s: a longer split runs as segments of 1024 into alternating
//             accumulators (double-buffered), and the epilogue adds each segment to the
//             split's float32 partial in order with round-to-nearest adds (the previous sums
//             read back from L2).  The splits are then only as many as the load balance
//             wants, and the host's sum over them reads a few partials instead of one per
//             1024 values of s.
//
// Every barrier wait is bounded (wait_phase) and aborts the CTA; after an abort the
// producer waits for its armed copies, each MMA-issuing thread for its MMAs, and the store
// thread for its stores, before the CTA frees its tensor memory; STATUS_TIMEOUT is then
// reported.
#include <algorithm>
#include <cfloat>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dna_internal.h"
#include "tc_common.cuh"

namespace dna {
namespace tc {
namespace mats {

constexpr int SC = 128;                       // values of s per chunk of the ratios kernel
constexpr int EPI = 16;                       // epilogue warps of the ratios kernel
constexpr int W_PROD_A = EPI, W_MMA_A = EPI + 1;
constexpr int A_THREADS = (EPI + 2) * 32;
constexpr int NSTG = 3;                       // staging buffers of the Q tiles
constexpr uint32_t TILE = 128 * 64 * 2;       // one [128 rows][64 K] bf16 tile, 16 KB

template <int RP>
struct LayoutA {
    static constexpr int KST = 2;
    // a K-slice: Y hi, Y lo [128 s][64 r] and X lo [128 o][64 r], 128-byte swizzled
    static constexpr uint32_t STAGE = 3 * TILE;
    // a staging buffer: two [128 o][64 s] tiles (Q hi and Qbar hi, Q lo and Qbar lo, or
    // Q hi and Q lo without Qbar)
    static constexpr uint32_t STG = 2 * TILE;
    static constexpr uint32_t SR = KST * STAGE;
    static constexpr uint32_t BAR = SR + NSTG * STG;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;
    static constexpr uint32_t TX = 0;          // X hi: RP / 2 columns (bf16 pairs)
    static constexpr uint32_t TZ = 256;        // two Z buffers of 128 columns
    static_assert(RP / 2 <= TZ, "X hi fits below the Z buffers");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};
enum { A_KFULL = 0, A_KEMPTY = 2, A_XFULL = 4, A_ZFULL = 5, A_ZEMPTY = 7, A_DRAIN = 9,
       A_COUNT = 10 };

struct RatioArgs {
    int64_t S, O, s_per;      // s_per: a multiple of SC
    const float* V;           // V_so, element (s, o) at V[s * vs + o]
    int64_t vs;
    const bf16* X;            // hi plane [O_pad][rp]
    int64_t rp;
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

// 16 values of s (two 16-byte chunks, 2 cg and 2 cg + 1) of row `row` of a [128][64]
// bf16 tile in the 128-byte swizzled layout
__device__ __forceinline__ void put_row16(uint32_t tile, int row, int cg, const uint32_t (&w)[8]) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const uint32_t off =
            (uint32_t)row * 128u + ((((uint32_t)(2 * cg + c)) ^ ((uint32_t)row & 7u)) << 4);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(tile + off),
                     "r"(w[4 * c]), "r"(w[4 * c + 1]), "r"(w[4 * c + 2]), "r"(w[4 * c + 3])
                     : "memory");
    }
}

constexpr int B_EPI = 8;                      // epilogue warps of the contract kernel
constexpr int W_PROD_B = B_EPI, W_MMA_B = B_EPI + 1;
constexpr int B_THREADS = (B_EPI + 2) * 32;
constexpr int RB = 256;                       // r per tile of the contract kernel
// K-slices of 64 values of s that one accumulation in tensor memory takes at most (1024
// values: the tensor pipe's float32 accumulation stays short); a longer tile adds its
// segments into the float32 partial in order with round-to-nearest adds
constexpr int SEG_SL = 16;

struct LayoutB {
    static constexpr int KST = 2;
    static constexpr uint32_t Q_TILE = OBLK * 64 * 2;    // [128 o][64 s]
    static constexpr uint32_t Y_TILE = RB * 64 * 2;      // [256 r][64 s]
    // Q hi, Q lo, Yt hi, Yt lo (which = 0) or Qbar hi, Qbar lo, Y2t hi, Y2t lo (which = 1)
    static constexpr uint32_t STAGE = 2 * Q_TILE + 2 * Y_TILE;
    static constexpr uint32_t BAR = KST * STAGE;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;               // two accumulators of 256 columns
    static_assert(STAGE % 1024 == 0, "alignment");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};
enum { C_KFULL = 0, C_KEMPTY = 2, C_ACCFULL = 4, C_ACCEMPTY = 6, C_DRAIN = 8, C_COUNT = 9 };

struct ContractArgs {
    int64_t S, O, R, s_per;   // s_per: a multiple of 64
    float* Apart;             // [splits][R][O]
    float* Bpart;
};

struct BTile {
    int64_t o0, s_begin;
    int nsl, rb, split, which;
};
// tiles: which slowest, then the split, then the o-block, r-block fastest.  CTA i of G
// takes tiles i, i + G, i + 2 G, ..., so with G even the r-blocks of one (o-block, split)
// run at the same time on CTAs i and i + 1 and the second read of the Q planes comes from
// L2 (CTAs running together also share the Yt slices of one split).
__device__ __forceinline__ BTile b_tile(int t, int nob, int nrb, int nsplit,
                                        const ContractArgs& a) {
    BTile x;
    const int per_which = nrb * nob * nsplit;
    x.which = t / per_which;
    const int u = t % per_which;
    x.rb = u % nrb;
    const int rest = u / nrb;
    x.o0 = (int64_t)(rest % nob) * OBLK;
    x.split = rest / nob;
    x.s_begin = (int64_t)x.split * a.s_per;
    const int64_t s_end = min(a.S, x.s_begin + a.s_per);
    x.nsl = s_end > x.s_begin ? (int)((s_end - x.s_begin + 63) / 64) : 0;
    return x;
}

}  // namespace mats

// ---------------------------------------------------------------- ratios kernel
template <int RP, bool WITH_B>
__global__ void __launch_bounds__(mats::A_THREADS, 1)
    k_tcs_ratios(mats::RatioArgs a, int nsplit, int ntiles,
                 const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmYl,
                 const __grid_constant__ CUtensorMap tmXl,
                 const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmQl,
                 const __grid_constant__ CUtensorMap tmQb,
                 const __grid_constant__ CUtensorMap tmQbl) {
    using namespace mats;
    using L = LayoutA<RP>;
    constexpr int KST = L::KST, KS = RP / 64;
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
        // K-slices of every chunk in the MMA thread's order: Y hi, Y lo [128 s][64 r] and
        // X lo [128 o][64 r]
        if (lane == 0 && t_begin < t_end) {
            tma_prefetch_desc(&tmY);
            tma_prefetch_desc(&tmYl);
            tma_prefetch_desc(&tmXl);
            int kk = 0;
            bool ok = true;
            for (int t = t_begin; ok && t < t_end; ++t) {
                const ATile x = a_tile(t, nsplit, a);
                for (int k = 0; ok && k < x.nch; ++k) {
                    const int32_t s0 = (int32_t)(x.s_begin + (int64_t)k * SC);
                    for (int ks = 0; ks < KS; ++ks, ++kk) {
                        const int st = kk % KST;
                        if (!(ok = wait_phase(&bar[A_KEMPTY + st], ((kk / KST) & 1) ^ 1, abort)))
                            break;
                        const uint32_t dst = sbase + st * L::STAGE;
                        const int32_t r0 = 64 * ks;
                        uint64_t* fb = &bar[A_KFULL + st];
                        mbar_arrive_expect_tx(fb, L::STAGE);
                        tma_load_2d(dst, &tmY, r0, s0, fb);
                        tma_load_2d(dst + TILE, &tmYl, r0, s0, fb);
                        tma_load_2d(dst + 2 * TILE, &tmXl, r0, (int32_t)x.o0, fb);
                    }
                }
            }
            if (*abort)   // let the copies already issued land before the CTA exits
                for (int k = max(0, kk - KST); k < kk; ++k)
                    drain_phase(&bar[A_KFULL + k % KST], (k / KST) & 1);
        }
    } else if (warp == W_MMA_A) {
        // Z(m) = X Y(m)^t into buffer m & 1: per K-slice the three products, each over the
        // slice's four K-steps (no two consecutive MMAs share a K-step's operands)
        if (lane == 0) {
            bool ok = true;
            int m = 0, j = 0, nx = 0;
            constexpr uint32_t idesc = idesc_bf16(OBLK, SC);
            for (int t = t_begin; ok && t < t_end; ++t) {
                const ATile x = a_tile(t, nsplit, a);
                if (t == t_begin || a_tile(t - 1, nsplit, a).o0 != x.o0) {
                    // a new o-block: the epilogue has written its X hi
                    if (!(ok = wait_phase(&bar[A_XFULL], nx & 1, abort))) break;
                    ++nx;
                }
                tc_fence_after();
                for (int k = 0; ok && k < x.nch; ++k, ++m) {
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
                        const uint32_t yh = sbase + (j % KST) * L::STAGE;
                        const uint32_t yl = yh + TILE, xl = yh + 2 * TILE;
                        const uint32_t xh = tmem + L::TX + (uint32_t)(32 * ks);
#pragma unroll
                        for (int kq = 0; kq < 4; ++kq)   // X hi (tensor memory) Y hi
                            mma_bf16_tmem_a(tz, xh + 8u * kq, desc_sw128(yh + 32u * kq), idesc,
                                            (ks > 0 || kq > 0) ? 1u : 0u);
#pragma unroll
                        for (int kq = 0; kq < 4; ++kq)   // X hi Y lo
                            mma_bf16_tmem_a(tz, xh + 8u * kq, desc_sw128(yl + 32u * kq), idesc, 1u);
#pragma unroll
                        for (int kq = 0; kq < 4; ++kq)   // X lo (shared memory) Y hi
                            mma_bf16(tz, desc_sw128(xl + 32u * kq), desc_sw128(yh + 32u * kq),
                                     idesc, 1u);
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
        // s = 64 h + 16 cg .. + 15 of Z buffer columns 64 h + 16 cg .., their v read from
        // global memory one half chunk ahead (lanes read consecutive o).  Per half chunk
        // one or two store groups of two [128 o][64 s] tiles go through staging buffer
        // g % NSTG; thread 0 stores them by TMA, and before group g is written it waits
        // until at most NSTG - 1 groups are still reading shared memory (so group g - NSTG,
        // the last one out of that buffer, has read it).  The waits' outcomes are OR-ed
        // over the epilogue warps at a named barrier, so all of them leave together on an
        // abort.
        constexpr uint32_t NB = 1, NT_EPI = EPI * 32;
        constexpr int GPH = WITH_B ? 2 : 1;
        const int qd = warp & 3, cg = warp >> 2;
        const int row = 32 * qd + lane;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        const bool leader = tid == 0;
        auto v_src = [&](const ATile& x, int k, int h, const float*& p, int& n) {
            const int64_t o = x.o0 + row;
            const int64_t s0 = x.s_begin + (int64_t)k * SC + 64 * h + 16 * cg;
            const int64_t left = a.S - s0;
            p = a.V + s0 * a.vs + o;
            n = (o < a.O && left > 0) ? (left < 16 ? (int)left : 16) : 0;
        };
        float vn[16];   // v of the next half chunk
        if (t_begin < t_end) {
            const float* p;
            int n;
            v_src(a_tile(t_begin, nsplit, a), 0, 0, p, n);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) vn[jj] = jj < n ? __ldg(p + jj * a.vs) : 0.f;
        }
        float qbmax = 0.f;   // an infinite qbar: z = 0 where v > 0 (infinite cost)
        bool ok = true;
        int m = 0, g = 0;
        for (int t = t_begin; ok && t < t_end; ++t) {
            const ATile x = a_tile(t, nsplit, a);
            const int64_t o = x.o0 + row;
            if (t == t_begin || a_tile(t - 1, nsplit, a).o0 != x.o0) {
                // a new o-block: its X hi rows into tensor memory (every GEMM of the previous
                // tile has completed: its last Z was read below)
#pragma unroll 1
                for (int unit = cg; unit < RP / 32; unit += 4)
                    x_to_tmem(a.X, a.rp, o, unit, tmem + L::TX + lane_off);
                tmem_st_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[A_XFULL]);
            }
            for (int k = 0; ok && k < x.nch; ++k, ++m) {
                const int b = m & 1;
                const bool w_ok = wait_phase(&bar[A_ZFULL + b], (m >> 1) & 1, abort);
                if (named_any(NB, NT_EPI, !w_ok)) { ok = false; break; }
                tc_fence_after();
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    uint32_t zr[16];
                    tmem_ld16(tmem + L::TZ + b * SC + 64 * h + 16 * cg + lane_off, zr);
                    float vv[16];
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) vv[jj] = vn[jj];
                    {   // the next half chunk's v
                        const float* pn = a.V;
                        int nn = 0;
                        if (h == 0)
                            v_src(x, k, 1, pn, nn);
                        else if (k + 1 < x.nch)
                            v_src(x, k + 1, 0, pn, nn);
                        else if (t + 1 < t_end)
                            v_src(a_tile(t + 1, nsplit, a), 0, 0, pn, nn);
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj) vn[jj] = jj < nn ? __ldg(pn + jj * a.vs) : 0.f;
                    }
                    tmem_ld_wait();
                    if (h == 1) {   // both halves read: the buffer is free for chunk m + 2
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&bar[A_ZEMPTY + b]);
                    }
                    // z >= 0; with v' = max(v, 0) and z' = max(z, FLT_MIN), q = v' / z' and
                    // qbar = q / z' are 0 where v = 0 and v / z, v / z^2 elsewhere, unless
                    // z = 0 where v > 0, which makes qbar infinite
                    uint32_t qh[8], ql[8], bh[8], bl[8];
#pragma unroll
                    for (int jj = 0; jj < 16; jj += 2) {
                        float q[2], qb[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const float v = fmaxf(vv[jj + u], 0.f);
                            const float z = fmaxf(__uint_as_float(zr[jj + u]), FLT_MIN);
                            const float rz = rcp_ftz(z);
                            q[u] = v * rz;
                            qb[u] = q[u] * rz;
                            qbmax = fmaxf(qbmax, qb[u]);
                        }
                        split2(q[0], q[1], qh[jj / 2], ql[jj / 2]);
                        if (WITH_B) split2(qb[0], qb[1], bh[jj / 2], bl[jj / 2]);
                    }
                    const int32_t s0 = (int32_t)(x.s_begin + (int64_t)k * SC + 64 * h);
#pragma unroll
                    for (int gi = 0; gi < GPH; ++gi, ++g) {
                        const uint32_t buf = sbase + L::SR + (uint32_t)(g % NSTG) * L::STG;
                        if (leader) bulk_wait_read<NSTG - 1>();
                        named_sync(NB, NT_EPI);   // buffer g % NSTG is free
                        if (!WITH_B) {
                            put_row16(buf, row, cg, qh);
                            put_row16(buf + TILE, row, cg, ql);
                        } else if (gi == 0) {
                            put_row16(buf, row, cg, qh);
                            put_row16(buf + TILE, row, cg, bh);
                        } else {
                            put_row16(buf, row, cg, ql);
                            put_row16(buf + TILE, row, cg, bl);
                        }
                        fence_proxy_async_smem();   // visible to the TMA (async proxy)
                        named_sync(NB, NT_EPI);     // every row of both tiles is written
                        if (leader) {
                            const int32_t o0 = (int32_t)x.o0;
                            if (!WITH_B) {
                                tma_store_2d(&tmQ, buf, s0, o0);
                                tma_store_2d(&tmQl, buf + TILE, s0, o0);
                            } else {
                                tma_store_2d(gi ? &tmQl : &tmQ, buf, s0, o0);
                                tma_store_2d(gi ? &tmQbl : &tmQb, buf + TILE, s0, o0);
                            }
                            bulk_commit();
                        }
                    }
                }
                if (!ok) break;
            }
        }
        if (leader) bulk_wait_all();   // the Q stores are complete before the CTA exits
        if (!(qbmax <= FLT_MAX)) atomicOr(a.status, STATUS_NONFINITE);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(a.status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

// ---------------------------------------------------------------- contract kernel
template <bool WITH_B>
__global__ void __launch_bounds__(mats::B_THREADS, 1)
    k_tcs_contract(mats::ContractArgs a, int nob, int nrb, int nsplit, int ntiles, int* status,
                   const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmQl,
                   const __grid_constant__ CUtensorMap tmQb,
                   const __grid_constant__ CUtensorMap tmQbl,
                   const __grid_constant__ CUtensorMap tmYt,
                   const __grid_constant__ CUtensorMap tmYtl,
                   const __grid_constant__ CUtensorMap tmY2t,
                   const __grid_constant__ CUtensorMap tmY2tl) {
    using namespace mats;
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
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar[C_ACCFULL + i], 1);
            mbar_init(&bar[C_ACCEMPTY + i], B_EPI);
        }
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
            tma_prefetch_desc(&tmQ); tma_prefetch_desc(&tmQl);
            tma_prefetch_desc(&tmYt); tma_prefetch_desc(&tmYtl);
            if (WITH_B) {
                tma_prefetch_desc(&tmQb); tma_prefetch_desc(&tmQbl);
                tma_prefetch_desc(&tmY2t); tma_prefetch_desc(&tmY2tl);
            }
            int kk = 0;
            bool ok = true;
            for (int t = t_first; ok && t < ntiles; t += t_step) {
                const BTile x = b_tile(t, nob, nrb, nsplit, a);
                const CUtensorMap* mq = x.which ? &tmQb : &tmQ;
                const CUtensorMap* mql = x.which ? &tmQbl : &tmQl;
                const CUtensorMap* my = x.which ? &tmY2t : &tmYt;
                const CUtensorMap* myl = x.which ? &tmY2tl : &tmYtl;
                for (int sl = 0; sl < x.nsl; ++sl, ++kk) {
                    const int st = kk % KST;
                    if (!(ok = wait_phase(&bar[C_KEMPTY + st], ((kk / KST) & 1) ^ 1, abort)))
                        break;
                    const uint32_t dst = sbase + st * L::STAGE;
                    const int32_t s0 = (int32_t)(x.s_begin + 64 * (int64_t)sl);
                    const int32_t r0 = RB * x.rb, o0 = (int32_t)x.o0;
                    uint64_t* fb = &bar[C_KFULL + st];
                    mbar_arrive_expect_tx(fb, L::STAGE);
                    tma_load_2d(dst, mq, s0, o0, fb);                             // [128 o][64 s]
                    tma_load_2d(dst + L::Q_TILE, mql, s0, o0, fb);
                    tma_load_2d(dst + 2 * L::Q_TILE, my, s0, r0, fb);             // [256 r][64 s]
                    tma_load_2d(dst + 2 * L::Q_TILE + L::Y_TILE, myl, s0, r0, fb);
                }
            }
            if (*abort)
                for (int k = max(0, kk - KST); k < kk; ++k)
                    drain_phase(&bar[C_KFULL + k % KST], (k / KST) & 1);
        }
    } else if (warp == W_MMA_B) {
        if (lane == 0) {
            bool ok = true;
            int j = 0, sg = 0;
            constexpr uint32_t idesc = idesc_bf16(OBLK, RB);
            for (int t = t_first; ok && t < ntiles; t += t_step) {
                const int nsl = b_tile(t, nob, nrb, nsplit, a).nsl;
                // segments of at most SEG_SL K-slices, each into the next accumulator
                for (int sl0 = 0; ok && sl0 < nsl; sl0 += SEG_SL, ++sg) {
                    const int ab = sg & 1, sl1 = min(nsl, sl0 + SEG_SL);
                    // the epilogue has copied segment sg - 2 out of this accumulator
                    if (sg >= 2 &&
                        !(ok = wait_phase(&bar[C_ACCEMPTY + ab], ((sg - 2) >> 1) & 1, abort)))
                        break;
                    tc_fence_after();
                    const uint32_t acc = tmem + (uint32_t)(ab * RB);
#pragma unroll 1
                    for (int sl = sl0; sl < sl1; ++sl, ++j) {
                        if (!(ok = wait_phase(&bar[C_KFULL + j % KST], (j / KST) & 1, abort)))
                            break;
                        tc_fence_after();
                        const uint32_t qh = sbase + (j % KST) * L::STAGE, ql = qh + L::Q_TILE;
                        const uint32_t yh = qh + 2 * L::Q_TILE, yl = yh + L::Y_TILE;
#pragma unroll
                        for (int kq = 0; kq < 4; ++kq)   // Q hi Yt hi
                            mma_bf16(acc, desc_sw128(qh + 32u * kq), desc_sw128(yh + 32u * kq),
                                     idesc, (sl > sl0 || kq > 0) ? 1u : 0u);
#pragma unroll
                        for (int kq = 0; kq < 4; ++kq)   // Q hi Yt lo
                            mma_bf16(acc, desc_sw128(qh + 32u * kq), desc_sw128(yl + 32u * kq),
                                     idesc, 1u);
#pragma unroll
                        for (int kq = 0; kq < 4; ++kq)   // Q lo Yt hi
                            mma_bf16(acc, desc_sw128(ql + 32u * kq), desc_sw128(yh + 32u * kq),
                                     idesc, 1u);
                        mma_commit(&bar[C_KEMPTY + j % KST]);
                    }
                    if (ok) mma_commit(&bar[C_ACCFULL + ab]);
                }
            }
            if (!ok) {
                mma_commit(&bar[C_DRAIN]);
                drain_phase(&bar[C_DRAIN], 0);
            }
        }
    } else {
        // epilogue warps: lane quadrant qd, column half hf of the 256-wide accumulator;
        // rows o = o0 + 32 qd + lane
        const int qd = warp & 3, hf = warp >> 2;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        int sg = 0;
        bool live = true;
        for (int t = t_first; live && t < ntiles; t += t_step) {
            const BTile x = b_tile(t, nob, nrb, nsplit, a);
            const int64_t o = x.o0 + 32 * qd + lane;
            float* dst = x.which ? a.Bpart : a.Apart;
            const int64_t base = (int64_t)x.split * a.R;
            for (int sl0 = 0; sl0 < x.nsl; sl0 += SEG_SL, ++sg) {
                const int ab = sg & 1;
                bool ok = wait_phase(&bar[C_ACCFULL + ab], (sg >> 1) & 1, abort);
                if (!__all_sync(0xffffffffu, ok)) {
                    live = false;
                    break;
                }
                tc_fence_after();
#pragma unroll 1
                for (int c = 0; c < 4; ++c) {
                    uint32_t r32[32];
                    tmem_ld32(tmem + (uint32_t)(ab * RB + 128 * hf + 32 * c) + lane_off, r32);
                    tmem_ld_wait();
                    if (o < a.O) {
                        // the tile's segments in order: the first writes, the later ones add
                        // (the previous sums' loads all issued before any store)
                        const int64_t r0 = (int64_t)RB * x.rb + 128 * hf + 32 * c;
                        float* col = dst + (base + r0) * a.O + o;
                        const int64_t left = a.R - r0;
                        const int nr = left < 32 ? (int)left : 32;
                        float prev[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            prev[i] = (sl0 > 0 && i < nr) ? col[(int64_t)i * a.O] : 0.f;
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (i < nr) col[(int64_t)i * a.O] = prev[i] + __uint_as_float(r32[i]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar[C_ACCEMPTY + ab]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

// ---------------------------------------------------------------- launch
template <int RP, bool WITH_B>
int launch_mats(const TcOperands& op, const TcMaps& m, float* Apart, float* Bpart, int splits,
                int64_t s_per, int* status, cudaStream_t st) {
    using namespace mats;
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
    ra.status = status;
    {
        const uint32_t smem = LayoutA<RP>::TOTAL + 1024;
        auto k = k_tcs_ratios<RP, WITH_B>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return DNA_ERR_CUDA;
        const int ntiles = nob * splits_a;
        const int grid = op.ctas > 0 ? std::min(op.ctas, ntiles) : ntiles;
        k<<<grid, A_THREADS, smem, st>>>(ra, splits_a, ntiles, m.y128, m.y128_l, m.x_l, m.q,
                                         m.q_l, m.qb, m.qb_l);
        if (int e = after_launch()) return e;
    }
    ContractArgs ca{};
    ca.S = op.S; ca.O = op.O; ca.R = op.R; ca.s_per = s_per;
    ca.Apart = Apart; ca.Bpart = Bpart;
    const uint32_t smem = LayoutB::TOTAL + 1024;
    auto k = k_tcs_contract<WITH_B>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    const int nrb = RP / RB;
    const int ntiles = (WITH_B ? 2 : 1) * nrb * nob * splits;
    const int grid = op.ctas > 0 ? std::min(op.ctas, ntiles) : ntiles;
    k<<<grid, B_THREADS, smem, st>>>(ca, nob, nrb, splits, ntiles, status, m.q, m.q_l, m.qb,
                                     m.qb_l, m.yt256, m.yt256_l, m.y2t256, m.y2t256_l);
    return after_launch();
}

}  // namespace tc

int TcBf16::pass1_mats(const TcOperands& op, const TcMaps& maps, float* Apart, float* Bpart,
                       int splits, int64_t s_per, bool with_b, int* status, cudaStream_t st) {
    const int rp = rank_pad(op.R);
    if (!op.Qg || !op.Qbg || !op.plane || !op.qplane || op.ldq % tc::mats::SC != 0 ||
        s_per % 64 != 0)
        return DNA_ERR_ARG;
    if (splits != (int)((op.S + s_per - 1) / s_per)) return DNA_ERR_ARG;
    if (rp == 256)
        return with_b ? tc::launch_mats<256, true>(op, maps, Apart, Bpart, splits, s_per, status, st)
                      : tc::launch_mats<256, false>(op, maps, Apart, Bpart, splits, s_per, status, st);
    if (rp == 512)
        return with_b ? tc::launch_mats<512, true>(op, maps, Apart, Bpart, splits, s_per, status, st)
                      : tc::launch_mats<512, false>(op, maps, Apart, Bpart, splits, s_per, status, st);
    return DNA_ERR_UNSUPPORTED;
}

}  // namespace dna
