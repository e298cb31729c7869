// tcgen05 passes of the BF16 form at large padded rank: pass 1 for RP in {256, 512}
// (Algorithm 1 steps 2-5 and 10) and pass 2 for RP = 512 (after it in this file).
//
// Pass 1.  Tensor memory cannot hold X (the A operand of GEMM1) beside Z and both
// accumulators at these ranks, so
//   * GEMM1 Z[o, s] = sum_r X[o, r] Y[s, r] takes both operands from shared memory: X and
//     Y stream together through a ring of 64-wide K-slices (M = 128, N = 128, K = 16 per
//     MMA, RP / 16 MMAs per chunk of 128 values of s);
//   * A and B are split into r-blocks of 128: a tile is one (r-block, o-block, split of s)
//     and accumulates A[o, r] and B[o, r] for its 128 values of r, recomputing Z;
//   * Q and Qbar (bf16 pairs) overwrite Z in tensor memory, each epilogue warp writing the
//     8 + 8 columns of the 16 values of s whose Z it read: tensor memory = two ZQ buffers
//     of 128 columns, A and B of the r-block (512 columns);
//   * GEMM2 / GEMM3 A[o, r] += sum_s Q[o, s] Yt[r, s], B[o, r] += sum_s Qbar[o, s] Y2t[r, s]
//     take Q from tensor memory and the r-block's rows of Y^t and (Y o Y)^t from a ring of
//     half chunks (64 values of s);
//   * the epilogue reads V straight from global memory into registers, a half chunk ahead
//     of its use, so shared memory carries only the MMA operands: per chunk RP / 2 KB of X
//     and Y slices (written by TMA, read by GEMM1; five K-slice stages) and 64 KB of the
//     r-block's Y^t and (Y o Y)^t rows.  That traffic and the chain GEMM1(m) -> epilogue(m)
//     -> GEMM2/3(m) -> GEMM1(m + 2) through the two ZQ buffers bound the kernel.
// Warp roles as in the split FP32 kernels (tc_split.cu): sixteen epilogue warps, a TMA
// producer warp, one MMA-issuing warp for GEMM1 and one for GEMM2 / GEMM3.  Persistent:
// CTA i takes the tiles [i T / G, (i + 1) T / G), numbered r-block-major so that the
// r-block CTAs of one (split, o-block) stream the same V, X and Y tiles at the same time.
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

namespace ks {

constexpr int SC = 128;   // values of s per chunk

struct Layout {
    static constexpr int KST = 5, HST = 2;
    // K-slice stage: X [128 o][64 r] and Y [128 s][64 r], bf16, K-major 128-byte swizzled
    static constexpr uint32_t X_SLICE = OBLK * 64 * 2;
    static constexpr uint32_t Y_SLICE = SC * 64 * 2;
    static constexpr uint32_t K_STAGE = X_SLICE + Y_SLICE;
    // H stage: the r-block's rows of Y^t and (Y o Y)^t for 64 values of s, [128 r][64 s]
    static constexpr uint32_t H_PLANE = 128 * SCH * 2;
    static constexpr uint32_t H_STAGE = 2 * H_PLANE;
    static constexpr uint32_t KR = 0;
    static constexpr uint32_t HR = KR + KST * K_STAGE;
    static constexpr uint32_t BAR = HR + HST * H_STAGE;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;
    // tensor memory: ZQ x 2 | A of the r-block | B of the r-block
    static constexpr uint32_t TA = 2 * SC, TB = TA + 128;
    static_assert(TB + 128 <= NCOLS, "tensor memory budget");
    static_assert(K_STAGE % 1024 == 0 && HR % 1024 == 0, "alignment");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};

enum { B_KFULL = 0, B_KEMPTY = 5, B_HFULL = 10, B_HEMPTY = 12, B_ZFULL = 14, B_QFULL = 16,
       B_QEMPTY = 20, B_DRAIN = 22, B_COUNT = 24 };

// One tile: the 128 values of r of r-block rb, one o-block, one split of s.
struct Tile {
    int64_t o0, s_begin;
    int nch, rb, split;
};
template <typename Args>
__device__ __forceinline__ Tile tile_of(int t, int nob, int nsplit, const Args& a) {
    Tile x;
    const int per_rb = nob * nsplit;
    x.rb = t / per_rb;
    const int rest = t % per_rb;
    x.o0 = (int64_t)(rest % nob) * OBLK;
    x.split = rest / nob;
    x.s_begin = (int64_t)x.split * a.s_per;
    const int64_t s_end = min(a.S, x.s_begin + a.s_per);
    x.nch = s_end > x.s_begin ? (int)((s_end - x.s_begin + SC - 1) / SC) : 0;
    return x;
}

// A walk over (tile, chunk, sub) units of one CTA, sub < per_chunk (every tile has at
// least one chunk: the host plans ceil(S / s_per) splits).
struct Cursor {
    int t, k, sub;
    Tile x;
    template <typename Args>
    __device__ __forceinline__ void start(int t0, int nob, int nsplit, const Args& a) {
        t = t0; k = 0; sub = 0;
        x = tile_of(t, nob, nsplit, a);
    }
    template <typename Args>
    __device__ __forceinline__ void next(int per_chunk, int nob, int nsplit, const Args& a) {
        if (++sub < per_chunk) return;
        sub = 0;
        if (++k < x.nch) return;
        k = 0;
        ++t;
        x = tile_of(t, nob, nsplit, a);
    }
};

}  // namespace ks

template <int RP, bool WITH_B>
__global__ void __launch_bounds__(P1_THREADS, 1)
    k_tc_pass1_kt(P1Args a, int nob, int nsplit, int ntiles,
                  const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                  const __grid_constant__ CUtensorMap tmYt,
                  const __grid_constant__ CUtensorMap tmY2t) {
    using L = ks::Layout;
    using namespace ks;
    constexpr int KST = L::KST, HST = L::HST, KS = RP / 64;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + B_COUNT * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L::BAR + B_COUNT * 8 + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t_begin = (int)((int64_t)blockIdx.x * ntiles / gridDim.x);
    const int t_end = (int)((int64_t)(blockIdx.x + 1) * ntiles / gridDim.x);

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == W_PRODUCER * 32) {
        for (int i = 0; i < KST; ++i) {
            mbar_init(&bar[B_KFULL + i], 1);
            mbar_init(&bar[B_KEMPTY + i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar[B_HFULL + i], 1);
            mbar_init(&bar[B_HEMPTY + i], 1);
            mbar_init(&bar[B_ZFULL + i], 1);
            mbar_init(&bar[B_QEMPTY + i], 1);
            mbar_init(&bar[B_DRAIN + i], 1);
        }
        for (int i = 0; i < 4; ++i) mbar_init(&bar[B_QFULL + i], W_EPI);
        *abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == W_PRODUCER) {
        // one thread services both rings in whatever order their slots free up
        if (lane == 0 && t_begin < t_end) {
            tma_prefetch_desc(&tmX); tma_prefetch_desc(&tmY); tma_prefetch_desc(&tmYt);
            if (WITH_B) tma_prefetch_desc(&tmY2t);
            Cursor ck_, ch_;
            ck_.start(t_begin, nob, nsplit, a);
            ch_.start(t_begin, nob, nsplit, a);
            int kk_ = 0, kh = 0;   // units issued per ring
            long long t0 = clock64();
            while (ck_.t < t_end || ch_.t < t_end) {
                bool prog = false;
                if (ck_.t < t_end && mbar_test(&bar[B_KEMPTY + kk_ % KST], ((kk_ / KST) & 1) ^ 1)) {
                    // K-slice sub of the chunk: X [128 o][64 r] and Y [128 s][64 r]
                    const int st = kk_ % KST;
                    const uint32_t dst = sbase + L::KR + st * L::K_STAGE;
                    const int32_t r0 = 64 * ck_.sub;
                    const int32_t s0 = (int32_t)(ck_.x.s_begin + (int64_t)ck_.k * SC);
                    mbar_arrive_expect_tx(&bar[B_KFULL + st], L::K_STAGE);
                    tma_load_2d(dst, &tmX, r0, (int32_t)ck_.x.o0, &bar[B_KFULL + st]);
                    tma_load_2d(dst + L::X_SLICE, &tmY, r0, s0, &bar[B_KFULL + st]);
                    tma_load_2d(dst + L::X_SLICE + SCH * 128, &tmY, r0, s0 + SCH,
                                &bar[B_KFULL + st]);
                    ++kk_;
                    ck_.next(KS, nob, nsplit, a);
                    prog = true;
                }
                if (ch_.t < t_end && mbar_test(&bar[B_HEMPTY + kh % HST], ((kh / HST) & 1) ^ 1)) {
                    const int st = kh % HST;
                    const uint32_t dst = sbase + L::HR + st * L::H_STAGE;
                    const int32_t s0 =
                        (int32_t)(ch_.x.s_begin + (int64_t)ch_.k * SC + SCH * ch_.sub);
                    mbar_arrive_expect_tx(&bar[B_HFULL + st], (WITH_B ? 2 : 1) * L::H_PLANE);
                    tma_load_2d(dst, &tmYt, s0, 128 * ch_.x.rb, &bar[B_HFULL + st]);
                    if (WITH_B)
                        tma_load_2d(dst + L::H_PLANE, &tmY2t, s0, 128 * ch_.x.rb,
                                    &bar[B_HFULL + st]);
                    ++kh;
                    ch_.next(2, nob, nsplit, a);
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
                for (int k = max(0, kk_ - KST); k < kk_; ++k)
                    drain_phase(&bar[B_KFULL + k % KST], (k / KST) & 1);
                for (int k = max(0, kh - HST); k < kh; ++k)
                    drain_phase(&bar[B_HFULL + k % HST], (k / HST) & 1);
            }
        }
    } else if (warp == W_MMA_Z) {
        // GEMM1 of chunk m into ZQ buffer m & 1, both operands from the K-slice ring
        if (lane == 0) {
            bool ok = true;
            int m = 0, j = 0;
            constexpr uint32_t idesc = idesc_bf16(OBLK, SC);
            for (int t = t_begin; ok && t < t_end; ++t) {
                const int nch = tile_of(t, nob, nsplit, a).nch;
                for (int k = 0; ok && k < nch; ++k, ++m) {
                    const int b = m & 1;
                    // GEMM2 / GEMM3 of chunk m - 2 have read their Q from this buffer
                    if (m >= 2 &&
                        !(ok = wait_phase(&bar[B_QEMPTY + b], ((m - 2) >> 1) & 1, abort)))
                        break;
                    const uint32_t tz = tmem + b * SC;
#pragma unroll 1
                    for (int ks = 0; ks < KS; ++ks, ++j) {
                        if (!(ok = wait_phase(&bar[B_KFULL + j % KST], (j / KST) & 1, abort)))
                            break;
                        tc_fence_after();
                        const uint32_t xs = sbase + L::KR + (j % KST) * L::K_STAGE;
                        const uint32_t ys = xs + L::X_SLICE;
#pragma unroll
                        for (int kq = 0; kq < 4; ++kq)
                            mma_bf16(tz, desc_sw128(xs + 32u * kq), desc_sw128(ys + 32u * kq),
                                     idesc, (ks > 0 || kq > 0) ? 1u : 0u);
                        mma_commit(&bar[B_KEMPTY + j % KST]);
                    }
                    if (ok) mma_commit(&bar[B_ZFULL + b]);
                }
            }
            if (!ok) {
                mma_commit(&bar[B_DRAIN + 0]);
                drain_phase(&bar[B_DRAIN + 0], 0);
            }
        }
    } else if (warp == W_MMA_AB) {
        // A += Q(m) Yt(m), B += Qbar(m) Y2t(m) for the r-block, one half chunk at a time;
        // the first MMAs of a tile overwrite the accumulators, which the epilogue has
        // copied out before it signals the tile's first Q
        if (lane == 0) {
            bool ok = true;
            int m = 0;
            constexpr uint32_t idesc = idesc_bf16(OBLK, 128);
            for (int t = t_begin; ok && t < t_end; ++t) {
                const int nch = tile_of(t, nob, nsplit, a).nch;
                for (int k = 0; ok && k < nch; ++k, ++m) {
                    const int b = m & 1;
#pragma unroll 1
                    for (int h = 0; ok && h < 2; ++h) {
                        const int jh = 2 * m + h;
                        if (!(ok = wait_phase(&bar[B_QFULL + 2 * b + h], (m >> 1) & 1, abort)))
                            break;
                        if (!(ok = wait_phase(&bar[B_HFULL + jh % HST], (jh / HST) & 1, abort)))
                            break;
                        tc_fence_after();
                        const uint32_t hs = sbase + L::HR + (jh % HST) * L::H_STAGE;
                        const uint32_t q0 = tmem + b * SC + 64 * h;
#pragma unroll
                        for (int kq = 0; kq < SCH / 16; ++kq) {
                            const uint32_t acc = (k > 0 || h > 0 || kq > 0) ? 1u : 0u;
                            mma_bf16_tmem_a(tmem + L::TA, q0 + 16 * kq, desc_sw128(hs + 32u * kq),
                                            idesc, acc);
                            if (WITH_B)
                                mma_bf16_tmem_a(tmem + L::TB, q0 + 16 * kq + 8,
                                                desc_sw128(hs + L::H_PLANE + 32u * kq), idesc,
                                                acc);
                        }
                        mma_commit(&bar[B_HEMPTY + jh % HST]);
                    }
                    if (ok) mma_commit(&bar[B_QEMPTY + b]);
                }
            }
            if (!ok) {
                mma_commit(&bar[B_DRAIN + 1]);
                drain_phase(&bar[B_DRAIN + 1], 0);
            }
        }
    } else {
        // epilogue warps 0-15: lane quadrant qd = warp % 4 (o = o0 + 32 qd + lane); in half h
        // of a chunk the warp takes the K-step kk = 4 h + cg (cg = warp / 4): the 16 values
        // s = 64 h + 16 cg .. + 15 and the ZQ columns 16 kk .. 16 kk + 15 (Q pairs in the
        // first 8, Qbar pairs in the last 8)
        const int qd = warp & 3, cg = warp >> 2;
        const int row = 32 * qd + lane;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        // this thread's 16 values of v for half h of chunk k of tile x are p[j * vs] for
        // j < n (0 for j >= n, outside the problem); each load instruction of the warp
        // reads 128 contiguous bytes of a row of V
        auto v_src = [&](const Tile& x, int k, int h, const float*& p, int& n) {
            const int64_t o = x.o0 + row;
            const int64_t s0 = x.s_begin + (int64_t)k * SC + 64 * h + 16 * cg;
            const int64_t left = a.S - s0;
            p = a.V + s0 * a.vs + o;
            n = o < a.O ? (left < 16 ? (int)left : 16) : 0;
        };
        // v of the half chunk being processed; each value is replaced by the next half
        // chunk's as soon as it has been used, so the loads fly for a whole half chunk
        float vn[16];
        if (t_begin < t_end) {
            const float* p;
            int n;
            v_src(tile_of(t_begin, nob, nsplit, a), 0, 0, p, n);
#pragma unroll
            for (int j = 0; j < 16; ++j) vn[j] = j < n ? __ldg(p + j * a.vs) : 0.f;
        }
        float qbmax = 0.f;   // an infinite qbar: z = 0 where v > 0 (infinite cost)
        bool ok = true;
        int m = 0;
        for (int t = t_begin; ok && t < t_end; ++t) {
            const Tile x = tile_of(t, nob, nsplit, a);
            for (int k = 0; k < x.nch; ++k, ++m) {
                const int b = m & 1;
                ok = wait_phase(&bar[B_ZFULL + b], (m >> 1) & 1, abort);
                if (!(ok = __all_sync(0xffffffffu, ok))) break;   // keep the warp converged
                tc_fence_after();
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    const uint32_t col = tmem + b * SC + 64 * h + 16 * cg + lane_off;
                    uint32_t zr[16];
                    tmem_ld16(col, zr);
                    const float* pn = a.V;   // the next half chunk's v
                    int nn = 0;
                    if (h == 0)
                        v_src(x, k, 1, pn, nn);
                    else if (k + 1 < x.nch)
                        v_src(x, k + 1, 0, pn, nn);
                    else if (t + 1 < t_end)
                        v_src(tile_of(t + 1, nob, nsplit, a), 0, 0, pn, nn);
                    tmem_ld_wait();
                    // z >= 0 (a sum of products of non-negative operands); with v' = max(v, 0)
                    // and z' = max(z, FLT_MIN), q = v' / z' and qbar = q / z' are 0 where
                    // v = 0 (z = 0 there too) and equal v / z, v / z^2 elsewhere, unless
                    // z = 0 where v > 0, which makes qbar infinite
                    uint32_t qp[8], qbp[8];
                    auto make_q = [&](auto all_in) {
#pragma unroll
                        for (int j = 0; j < 16; j += 2) {
                            float q[2], qb[2];
#pragma unroll
                            for (int tt = 0; tt < 2; ++tt) {
                                const float v = fmaxf(vn[j + tt], 0.f);
                                if (decltype(all_in)::value)
                                    vn[j + tt] = __ldg(pn + (j + tt) * a.vs);
                                else
                                    vn[j + tt] =
                                        j + tt < nn ? __ldg(pn + (j + tt) * a.vs) : 0.f;
                                const float z = fmaxf(__uint_as_float(zr[j + tt]), FLT_MIN);
                                const float rz = __fdividef(1.0f, z);
                                q[tt] = v * rz;
                                qb[tt] = q[tt] * rz;
                                qbmax = fmaxf(qbmax, qb[tt]);
                            }
                            qp[j / 2] = pack_bf16x2(q[0], q[1]);
                            qbp[j / 2] = pack_bf16x2(qb[0], qb[1]);
                        }
                    };
                    if (nn == 16)
                        make_q(std::true_type{});
                    else
                        make_q(std::false_type{});
                    tmem_st8(col, qp);
                    if (WITH_B) tmem_st8(col + 8, qbp);
                    tmem_st_wait();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar[B_QFULL + 2 * b + h]);
                }
            }
            if (!ok) break;
            // GEMM2 / GEMM3 of the tile's last chunk done: its A and B rows of the r-block
            const int ml = m - 1;
            ok = __all_sync(0xffffffffu,
                            wait_phase(&bar[B_QEMPTY + (ml & 1)], (ml >> 1) & 1, abort));
            if (!ok) break;
            tc_fence_after();
            const int64_t o = x.o0 + row;
            const int64_t base = (int64_t)x.split * a.R;
#pragma unroll 1
            for (int mat = 0; mat < (WITH_B ? 2 : 1); ++mat) {
                uint32_t r32[32];
                tmem_ld32(tmem + (mat ? L::TB : L::TA) + lane_off + 32 * cg, r32);
                tmem_ld_wait();
                float* dst = mat ? a.Bpart : a.Apart;
                if (o < a.O)
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int64_t r = 128 * x.rb + 32 * cg + i;
                        if (r < a.R) dst[(base + r) * a.O + o] = __uint_as_float(r32[i]);
                    }
            }
            tc_fence_before();
        }
        if (!(qbmax <= FLT_MAX)) atomicOr(a.status, STATUS_NONFINITE);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(a.status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

template <int RP, bool WITH_B>
int launch_pass1_kt(const P1Args& a, const TcMaps& m, int64_t O_pad, int splits, int ctas,
                    cudaStream_t st) {
    const uint32_t smem = ks::Layout::TOTAL + 1024;
    auto k = k_tc_pass1_kt<RP, WITH_B>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    const int nob = (int)(O_pad / OBLK);
    const int ntiles = (RP / 128) * nob * splits;
    if (ntiles == 0) return DNA_OK;
    const int grid = ctas > 0 ? std::min(ctas, ntiles) : ntiles;
    k<<<grid, P1_THREADS, smem, st>>>(a, nob, splits, ntiles, m.x, m.y, m.yt, m.y2t);
    return after_launch();
}

// ---------------------------------------------------------------- pass 2, RP = 512
// Candidate costs (Algorithm 1 steps 6-9 and 19-22): Z_mu = X_mu Y^t and Z_dna = X_dna
// Y^t per chunk of 128 values of s, both operands from shared memory (tensor memory holds
// two Z pairs, 4 x 128 columns, and no X), X_mu, X_dna and Y streaming together through a
// ring of 64-wide K-slices (eight MMAs per slice, alternating between the candidates);
// the epilogue reads V from global memory a half chunk ahead, as in pass 1, and sums
// d' = sum_s (z - v log z) (v > 0; z where v = 0) per column and candidate in float32
// over a chunk, then in float64.  Persistent over (o-block, split) tiles, o-block fastest,
// so CTAs that run at the same time share the Y slices in L2.  Each epilogue warp writes
// its own sums: cost slot 4 split + w / 4 of dpart[slot][2][O].
namespace ks {
struct Layout2 {
    static constexpr int KST = 4;
    static constexpr uint32_t X_SLICE = OBLK * 64 * 2;   // [128 o][64 r]
    static constexpr uint32_t Y_SLICE = SC * 64 * 2;     // [128 s][64 r]
    static constexpr uint32_t K_STAGE = 2 * X_SLICE + Y_SLICE;
    static constexpr uint32_t BAR = KST * K_STAGE;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;   // (Z_mu, Z_dna) x 2, 128 columns each
    static_assert(K_STAGE % 1024 == 0, "alignment");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};
enum { C_KFULL = 0, C_KEMPTY = 4, C_ZFULL = 8, C_ZEMPTY = 10, C_DRAIN = 12, C_COUNT = 14 };
constexpr int P2K_THREADS = (W_EPI + 2) * 32;   // epilogue warps, producer, MMA issuer
}  // namespace ks

template <int RP>
__global__ void __launch_bounds__(ks::P2K_THREADS, 1)
    k_tc_pass2_kt(P2Args a, int nob, int nsplit, int ntiles,
                  const __grid_constant__ CUtensorMap tmXm, const __grid_constant__ CUtensorMap tmXd,
                  const __grid_constant__ CUtensorMap tmY) {
    using L = ks::Layout2;
    using namespace ks;
    constexpr int KST = L::KST, KS = RP / 64;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + C_COUNT * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L::BAR + C_COUNT * 8 + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t_begin = (int)((int64_t)blockIdx.x * ntiles / gridDim.x);
    const int t_end = (int)((int64_t)(blockIdx.x + 1) * ntiles / gridDim.x);

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == W_PRODUCER * 32) {
        for (int i = 0; i < KST; ++i) {
            mbar_init(&bar[C_KFULL + i], 1);
            mbar_init(&bar[C_KEMPTY + i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar[C_ZFULL + i], 1);
            mbar_init(&bar[C_ZEMPTY + i], W_EPI);
            mbar_init(&bar[C_DRAIN + i], 1);
        }
        *abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == W_PRODUCER) {
        if (lane == 0 && t_begin < t_end) {
            tma_prefetch_desc(&tmXm); tma_prefetch_desc(&tmXd); tma_prefetch_desc(&tmY);
            Cursor ck_;
            ck_.start(t_begin, nob, nsplit, a);
            int kk_ = 0;
            bool ok = true;
            for (; ok && ck_.t < t_end; ++kk_, ck_.next(KS, nob, nsplit, a)) {
                const int st = kk_ % KST;
                if (!(ok = wait_phase(&bar[C_KEMPTY + st], ((kk_ / KST) & 1) ^ 1, abort))) break;
                // K-slice sub of the chunk: X_mu, X_dna [128 o][64 r], Y [128 s][64 r]
                const uint32_t dst = sbase + st * L::K_STAGE;
                const int32_t r0 = 64 * ck_.sub;
                const int32_t s0 = (int32_t)(ck_.x.s_begin + (int64_t)ck_.k * SC);
                mbar_arrive_expect_tx(&bar[C_KFULL + st], L::K_STAGE);
                tma_load_2d(dst, &tmXm, r0, (int32_t)ck_.x.o0, &bar[C_KFULL + st]);
                tma_load_2d(dst + L::X_SLICE, &tmXd, r0, (int32_t)ck_.x.o0, &bar[C_KFULL + st]);
                tma_load_2d(dst + 2 * L::X_SLICE, &tmY, r0, s0, &bar[C_KFULL + st]);
                tma_load_2d(dst + 2 * L::X_SLICE + SCH * 128, &tmY, r0, s0 + SCH,
                            &bar[C_KFULL + st]);
            }
            if (*abort)   // let the copies already issued land before the CTA exits
                for (int k = max(0, kk_ - KST); k < kk_; ++k)
                    drain_phase(&bar[C_KFULL + k % KST], (k / KST) & 1);
        }
    } else if (warp == W_EPI + 1) {
        // Z_mu(m), Z_dna(m) into pair buffer m & 1, K-slice by K-slice
        if (lane == 0) {
            bool ok = true;
            int m = 0, j = 0;
            constexpr uint32_t idesc = idesc_bf16(OBLK, SC);
            for (int t = t_begin; ok && t < t_end; ++t) {
                const int nch = tile_of(t, nob, nsplit, a).nch;
                for (int k = 0; ok && k < nch; ++k, ++m) {
                    const int b = m & 1;
                    // the epilogue has read chunk m - 2 out of this buffer pair
                    if (m >= 2 &&
                        !(ok = wait_phase(&bar[C_ZEMPTY + b], ((m - 2) >> 1) & 1, abort)))
                        break;
                    tc_fence_after();
                    const uint32_t zm = tmem + b * 2 * SC, zd = zm + SC;
#pragma unroll 1
                    for (int ks = 0; ks < KS; ++ks, ++j) {
                        if (!(ok = wait_phase(&bar[C_KFULL + j % KST], (j / KST) & 1, abort)))
                            break;
                        const uint32_t xs = sbase + (j % KST) * L::K_STAGE;
                        const uint32_t ys = xs + 2 * L::X_SLICE;
#pragma unroll
                        for (int kq = 0; kq < 4; ++kq) {
                            const uint64_t yd = desc_sw128(ys + 32u * kq);
                            const uint32_t acc = (ks > 0 || kq > 0) ? 1u : 0u;
                            mma_bf16(zm, desc_sw128(xs + 32u * kq), yd, idesc, acc);
                            mma_bf16(zd, desc_sw128(xs + L::X_SLICE + 32u * kq), yd, idesc, acc);
                        }
                        mma_commit(&bar[C_KEMPTY + j % KST]);
                    }
                    if (ok) mma_commit(&bar[C_ZFULL + b]);
                }
            }
            if (!ok) {
                mma_commit(&bar[C_DRAIN + 0]);
                drain_phase(&bar[C_DRAIN + 0], 0);
            }
        }
    } else if (warp < W_EPI) {
        // epilogue warp: lanes o = o0 + 32 qd + lane; in half h of a chunk the 16 values
        // s = 64 h + 16 cg .. + 15
        const int qd = warp & 3, cg = warp >> 2;
        const int row = 32 * qd + lane;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        auto v_src = [&](const Tile& x, int k, int h, const float*& p, int& n) {
            const int64_t o = x.o0 + row;
            const int64_t s0 = x.s_begin + (int64_t)k * SC + 64 * h + 16 * cg;
            const int64_t left = a.S - s0;
            p = a.V + s0 * a.vs + o;
            n = o < a.O ? (left < 16 ? (int)left : 16) : 0;
        };
        float vn[16];   // v of the half chunk being processed, then of the next one
        if (t_begin < t_end) {
            const float* p;
            int n;
            v_src(tile_of(t_begin, nob, nsplit, a), 0, 0, p, n);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) vn[jj] = jj < n ? __ldg(p + jj * a.vs) : 0.f;
        }
        bool ok = true, bad = false;
        int m = 0;
        for (int t = t_begin; ok && t < t_end; ++t) {
            const Tile x = tile_of(t, nob, nsplit, a);
            double acc_m = 0.0, acc_d = 0.0;
            for (int k = 0; k < x.nch; ++k, ++m) {
                const int b = m & 1;
                ok = wait_phase(&bar[C_ZFULL + b], (m >> 1) & 1, abort);
                if (!(ok = __all_sync(0xffffffffu, ok))) break;   // keep the warp converged
                tc_fence_after();
                float run_m = 0.f, run_d = 0.f;
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    const uint32_t col = tmem + b * 2 * SC + 64 * h + 16 * cg + lane_off;
                    uint32_t zm[16], zd[16];
                    tmem_ld16(col, zm);
                    tmem_ld16(col + SC, zd);
                    const float* pn = a.V;   // the next half chunk's v
                    int nn = 0;
                    if (h == 0)
                        v_src(x, k, 1, pn, nn);
                    else if (k + 1 < x.nch)
                        v_src(x, k + 1, 0, pn, nn);
                    else if (t + 1 < t_end)
                        v_src(tile_of(t + 1, nob, nsplit, a), 0, 0, pn, nn);
                    tmem_ld_wait();
                    if (h == 1) {   // both halves of the pair read: buffer free for chunk m + 2
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&bar[C_ZEMPTY + b]);
                    }
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const float v = vn[jj];
                        vn[jj] = jj < nn ? __ldg(pn + jj * a.vs) : 0.f;
                        const float z1 = __uint_as_float(zm[jj]), z2 = __uint_as_float(zd[jj]);
                        const bool pos = v > 0.f;
                        bad |= pos && !(z1 > 0.f && z2 > 0.f);
                        // the hardware logarithm (absolute error near 2^-21 around 1,
                        // relative 2^-21 elsewhere), far below the bf16 operand rounding
                        run_m += pos ? z1 - v * __logf(z1) : z1;
                        run_d += pos ? z2 - v * __logf(z2) : z2;
                    }
                }
                acc_m += (double)run_m;
                acc_d += (double)run_d;
            }
            if (!ok) break;
            const int64_t o = x.o0 + row;
            if (o < a.O) {
                const int64_t slot = 4 * (int64_t)x.split + cg;
                a.dpart[(slot * 2 + 0) * a.O + o] = acc_m;
                a.dpart[(slot * 2 + 1) * a.O + o] = acc_d;
            }
        }
        if (bad) atomicOr(a.status, STATUS_NONFINITE);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(a.status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

template <int RP>
int launch_pass2_kt(const P2Args& a, const TcMaps& m, int64_t O_pad, int splits, int ctas,
                    cudaStream_t st) {
    const uint32_t smem = ks::Layout2::TOTAL + 1024;
    auto k = k_tc_pass2_kt<RP>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    const int nob = (int)(O_pad / OBLK);
    const int ntiles = nob * splits;
    if (ntiles == 0) return DNA_OK;
    const int grid = ctas > 0 ? std::min(ctas, ntiles) : ntiles;
    k<<<grid, ks::P2K_THREADS, smem, st>>>(a, nob, splits, ntiles, m.xm, m.xd, m.y);
    return after_launch();
}

}  // namespace tc

int TcBf16::pass1_large(const TcOperands& op, const TcMaps& maps, float* Apart, float* Bpart,
                        int splits, int64_t s_per, bool with_b, int* status, cudaStream_t st) {
    tc::P1Args a{};
    a.S = op.S; a.O = op.O; a.R = op.R; a.s_per = s_per;
    a.Apart = Apart; a.Bpart = Bpart; a.status = status;
    a.V = op.V; a.vs = op.vs; a.X = op.Xk; a.rp = rank_pad(op.R);
    if (s_per % tc::ks::SC != 0) return DNA_ERR_ARG;
    if (a.rp == 256)
        return with_b ? tc::launch_pass1_kt<256, true>(a, maps, op.O_pad, splits, op.ctas, st)
                      : tc::launch_pass1_kt<256, false>(a, maps, op.O_pad, splits, op.ctas, st);
    if (a.rp == 512)
        return with_b ? tc::launch_pass1_kt<512, true>(a, maps, op.O_pad, splits, op.ctas, st)
                      : tc::launch_pass1_kt<512, false>(a, maps, op.O_pad, splits, op.ctas, st);
    return DNA_ERR_UNSUPPORTED;
}

int TcBf16::pass2_large(const TcOperands& op, const TcMaps& maps, double* dpart, int slots,
                        int64_t s_per, int* status, cudaStream_t st) {
    tc::P2Args a{};
    a.S = op.S; a.O = op.O; a.R = op.R; a.s_per = s_per;
    a.dpart = dpart; a.status = status;
    a.V = op.V; a.vs = op.vs; a.Xm = op.Xmk; a.Xd = op.Xdk; a.rp = rank_pad(op.R);
    if (s_per % tc::ks::SC != 0 || slots % 4 != 0) return DNA_ERR_ARG;
    const int splits = slots / 4;
    if (splits != (int)((op.S + s_per - 1) / s_per)) return DNA_ERR_ARG;
    if (a.rp == 512) return tc::launch_pass2_kt<512>(a, maps, op.O_pad, splits, op.ctas, st);
    return DNA_ERR_UNSUPPORTED;
}

}  // namespace dna
