// tcgen05 pass 2 at padded rank RP = 512 (Algorithm 1 steps 6-9 and 12-14; pass 1 at these
// ranks is in tc_mat.cu): the K-sliced kernel of the split FP32 form (RP 256, 512) and the
// Y-resident kernel of the BF16 form, and the tile walk they share.
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

// One tile: one o-block and one split of s (rb: the r-block, 0 for pass 2).
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

// ---------------------------------------------------------------- pass 2, RP = 512 (and split)
// Candidate costs (Algorithm 1 steps 6-9 and 19-22): Z_mu = X_mu Y^t and Z_dna = X_dna
// Y^t per chunk of 128 values of s, both operands from shared memory (tensor memory holds
// two Z pairs, 4 x 128 columns, and no X), X_mu, X_dna and Y streaming together through a
// ring of 64-wide K-slices (eight MMAs per slice, alternating between the candidates);
// the epilogue reads V from global memory a half chunk ahead, as in pass 1, and sums
// d' = sum_s (z - v log z) (v > 0; z where v = 0) per column and candidate in float32
// over a chunk, then in float64.  Persistent over (o-block, split) tiles, o-block fastest,
// so CTAs that run at the same time share the Y slices in L2.  Each epilogue warp writes
// its own sums: cost slot 4 split + w / 4 of dpart[slot][2][O].
//
// SPLIT: the FP32 form on the tensor cores (RP in {256, 512}): every operand as hi and lo
// bf16 planes, a K-slice holds X_mu, X_dna hi / lo and Y hi / lo (96 KB, two stages), and
// each Z takes the three products hi hi, hi lo, lo hi.
namespace ks {
template <bool SPLIT>
struct Layout2 {
    static constexpr int NP = SPLIT ? 2 : 1;               // planes per operand
    static constexpr int KST = SPLIT ? 2 : 4;
    static constexpr uint32_t X_SLICE = OBLK * 64 * 2;   // [128 o][64 r]
    static constexpr uint32_t Y_SLICE = SC * 64 * 2;     // [128 s][64 r]
    // X_mu hi (lo), X_dna hi (lo), Y hi (lo)
    static constexpr uint32_t K_STAGE = NP * (2 * X_SLICE + Y_SLICE);
    static constexpr uint32_t BAR = KST * K_STAGE;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;   // (Z_mu, Z_dna) x 2, 128 columns each
    static_assert(K_STAGE % 1024 == 0, "alignment");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};
enum { C_KFULL = 0, C_KEMPTY = 4, C_ZFULL = 8, C_ZEMPTY = 10, C_DRAIN = 12, C_COUNT = 14 };
constexpr int P2K_THREADS = (W_EPI + 2) * 32;   // epilogue warps, producer, MMA issuer
}  // namespace ks

template <int RP, bool SPLIT>
__global__ void __launch_bounds__(ks::P2K_THREADS, 1)
    k_tc_pass2_kt(P2Args a, int nob, int nsplit, int ntiles,
                  const __grid_constant__ CUtensorMap tmXm, const __grid_constant__ CUtensorMap tmXd,
                  const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmXml,
                  const __grid_constant__ CUtensorMap tmXdl, const __grid_constant__ CUtensorMap tmYl) {
    using L = ks::Layout2<SPLIT>;
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
            if (SPLIT) {
                tma_prefetch_desc(&tmXml); tma_prefetch_desc(&tmXdl); tma_prefetch_desc(&tmYl);
            }
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
                // plane p of the stage: X_mu, X_dna, Y (p = 1: the lo planes)
#pragma unroll
                for (int p = 0; p < L::NP; ++p) {
                    const uint32_t d = dst + (uint32_t)p * (2 * L::X_SLICE + L::Y_SLICE);
                    const CUtensorMap* mxm = p ? &tmXml : &tmXm;
                    const CUtensorMap* mxd = p ? &tmXdl : &tmXd;
                    const CUtensorMap* my = p ? &tmYl : &tmY;
                    tma_load_2d(d, mxm, r0, (int32_t)ck_.x.o0, &bar[C_KFULL + st]);
                    tma_load_2d(d + L::X_SLICE, mxd, r0, (int32_t)ck_.x.o0, &bar[C_KFULL + st]);
                    tma_load_2d(d + 2 * L::X_SLICE, my, r0, s0, &bar[C_KFULL + st]);
                    tma_load_2d(d + 2 * L::X_SLICE + SCH * 128, my, r0, s0 + SCH,
                                &bar[C_KFULL + st]);
                }
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
                        // product p: (X hi, Y hi), (X hi, Y lo), (X lo, Y hi); one in BF16
                        constexpr uint32_t PL = 2 * L::X_SLICE + L::Y_SLICE;
#pragma unroll
                        for (int p = 0; p < (SPLIT ? 3 : 1); ++p) {
                            const uint32_t xp = xs + (p == 2 ? PL : 0u);
                            const uint32_t ys = xs + (p == 1 ? PL : 0u) + 2 * L::X_SLICE;
#pragma unroll
                            for (int kq = 0; kq < 4; ++kq) {
                                const uint64_t yd = desc_sw128(ys + 32u * kq);
                                const uint32_t acc = (ks > 0 || p > 0 || kq > 0) ? 1u : 0u;
                                mma_bf16(zm, desc_sw128(xp + 32u * kq), yd, idesc, acc);
                                mma_bf16(zd, desc_sw128(xp + L::X_SLICE + 32u * kq), yd, idesc,
                                         acc);
                            }
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
                        // ln z = ln 2 log2 z with the hardware log2 (relative error
                        // about 2^-22), far below the bf16 operand rounding
                        run_m += pos ? z1 - v * (LN2F * lg2_ftz(z1)) : z1;
                        run_d += pos ? z2 - v * (LN2F * lg2_ftz(z2)) : z2;
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

template <int RP, bool SPLIT>
int launch_pass2_kt(const P2Args& a, const TcMaps& m, int64_t O_pad, int splits, int ctas,
                    cudaStream_t st) {
    const uint32_t smem = ks::Layout2<SPLIT>::TOTAL + 1024;
    auto k = k_tc_pass2_kt<RP, SPLIT>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    const int nob = (int)(O_pad / OBLK);
    const int ntiles = nob * splits;
    if (ntiles == 0) return DNA_OK;
    const int grid = ctas > 0 ? std::min(ctas, ntiles) : ntiles;
    if (SPLIT)
        k<<<grid, ks::P2K_THREADS, smem, st>>>(a, nob, splits, ntiles, m.xm, m.xd, m.y, m.xm_l,
                                               m.xd_l, m.y_l);
    else   // the lo maps are not read
        k<<<grid, ks::P2K_THREADS, smem, st>>>(a, nob, splits, ntiles, m.xm, m.xd, m.y, m.xm,
                                               m.xd, m.y);
    return after_launch();
}


// ---------------------------------------------------------------- pass 2, BF16, RP = 512
// Candidate costs with Y resident: a CTA walks units (s-block of 128 values of s, o-block),
// s-block-major, holding the s-block's Y ([128 s][512 r], 128 KB in eight 64-wide K-slices)
// in shared memory while the two candidates' K-slices ([128 o][64 r] each) stream through
// a ring of three stages.  Per unit only the candidates come in (256 KB against 384 KB when
// Y streams too), which is what bounds this pass: the copy rate into the SM.  Z_mu and
// Z_dna of a unit take 256 tensor-memory columns; two units are in flight.  Each of the 16
// epilogue warps sums d' = sum_s (z - v log z) (v > 0; z where v = 0) over 32 values of s
// for its 32 columns o in float32; the four partials of a column meet in tensor memory
// (each warp stores its pair into the first two Z columns it has read), and the warp with
// the first 32 values of s adds them in order in float64, so each (s-block, column) cost
// slot has one writer: dpart[sb][2][O].
namespace ks {
struct LayoutY {
    static constexpr int KS = 8;                        // 64-wide K-slices of r
    static constexpr int KST = 3;
    static constexpr uint32_t X_SLICE = OBLK * 64 * 2;  // [128 o][64 r]
    static constexpr uint32_t Y_SLICE = SC * 64 * 2;    // [128 s][64 r]
    static constexpr uint32_t K_STAGE = 2 * X_SLICE;    // X_mu, X_dna
    static constexpr uint32_t YR = 0;
    static constexpr uint32_t XR = YR + KS * Y_SLICE;
    static constexpr uint32_t BAR = XR + KST * K_STAGE;
    static constexpr uint32_t TOTAL = BAR + 256;
    static constexpr uint32_t NCOLS = 512;              // two (Z_mu, Z_dna) buffers
    static_assert(K_STAGE % 1024 == 0 && XR % 1024 == 0, "alignment");
    static_assert(TOTAL + 1024 <= 232448, "shared memory budget");
};
enum { Y_KFULL = 0, Y_KEMPTY = 3, Y_ZFULL = 6, Y_ZEMPTY = 8, Y_YFULL = 10, Y_YEMPTY = 11,
       Y_DRAIN = 12, Y_COUNT = 13 };
}  // namespace ks

__global__ void __launch_bounds__(ks::P2K_THREADS, 1)
    k_tc_pass2_yr(P2Args a, int nob, int nunits, const __grid_constant__ CUtensorMap tmXm,
                  const __grid_constant__ CUtensorMap tmXd, const __grid_constant__ CUtensorMap tmY) {
    using L = ks::LayoutY;
    using namespace ks;
    constexpr int KST = L::KST, KS = L::KS;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + Y_COUNT * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + L::BAR + Y_COUNT * 8 + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int u_begin = (int)((int64_t)blockIdx.x * nunits / gridDim.x);
    const int u_end = (int)((int64_t)(blockIdx.x + 1) * nunits / gridDim.x);
    const int nloc = u_end - u_begin;

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == W_PRODUCER * 32) {
        for (int i = 0; i < KST; ++i) {
            mbar_init(&bar[Y_KFULL + i], 1);
            mbar_init(&bar[Y_KEMPTY + i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar[Y_ZFULL + b], 1);
            mbar_init(&bar[Y_ZEMPTY + b], W_EPI);
        }
        mbar_init(&bar[Y_YFULL], 1);
        mbar_init(&bar[Y_YEMPTY], 1);
        mbar_init(&bar[Y_DRAIN], 1);
        *abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == W_PRODUCER) {
        if (lane == 0 && nloc > 0) {
            tma_prefetch_desc(&tmXm); tma_prefetch_desc(&tmXd); tma_prefetch_desc(&tmY);
            bool ok = true;
            int j = 0, yl = 0, prev = -1;
            for (int m = 0; ok && m < nloc; ++m) {
                const int u = u_begin + m, sb = u / nob, ob = u % nob;
                if (sb != prev) {   // the s-block's Y, once every MMA on the previous one is done
                    if (yl > 0 && !(ok = wait_phase(&bar[Y_YEMPTY], (yl - 1) & 1, abort))) break;
                    mbar_arrive_expect_tx(&bar[Y_YFULL], KS * L::Y_SLICE);
                    const int32_t s0 = 128 * sb;
                    for (int k = 0; k < KS; ++k) {
                        const uint32_t d = sbase + L::YR + k * L::Y_SLICE;
                        tma_load_2d(d, &tmY, 64 * k, s0, &bar[Y_YFULL]);
                        tma_load_2d(d + SCH * 128, &tmY, 64 * k, s0 + SCH, &bar[Y_YFULL]);
                    }
                    ++yl;
                    prev = sb;
                }
                for (int k = 0; k < KS; ++k, ++j) {
                    const int st = j % KST;
                    if (!(ok = wait_phase(&bar[Y_KEMPTY + st], ((j / KST) & 1) ^ 1, abort))) break;
                    const uint32_t d = sbase + L::XR + st * L::K_STAGE;
                    mbar_arrive_expect_tx(&bar[Y_KFULL + st], L::K_STAGE);
                    tma_load_2d(d, &tmXm, 64 * k, OBLK * ob, &bar[Y_KFULL + st]);
                    tma_load_2d(d + L::X_SLICE, &tmXd, 64 * k, OBLK * ob, &bar[Y_KFULL + st]);
                }
            }
            if (*abort) {   // let the copies already issued land before the CTA exits
                for (int k = max(0, j - KST); k < j; ++k)
                    drain_phase(&bar[Y_KFULL + k % KST], (k / KST) & 1);
                if (yl > 0) drain_phase(&bar[Y_YFULL], (yl - 1) & 1);
            }
        }
    } else if (warp == W_EPI + 1) {
        // Z_mu(m), Z_dna(m) into buffer m & 1, K-slice by K-slice against the resident Y
        if (lane == 0) {
            bool ok = true;
            int j = 0, yl = 0, prev = -1;
            constexpr uint32_t idesc = idesc_bf16(OBLK, SC);
            for (int m = 0; ok && m < nloc; ++m) {
                const int sb = (u_begin + m) / nob, b = m & 1;
                if (sb != prev) {
                    if (!(ok = wait_phase(&bar[Y_YFULL], yl & 1, abort))) break;
                    ++yl;
                    prev = sb;
                }
                // the epilogue has read unit m - 2 out of this buffer
                if (m >= 2 && !(ok = wait_phase(&bar[Y_ZEMPTY + b], ((m - 2) >> 1) & 1, abort)))
                    break;
                tc_fence_after();
                const uint32_t zm = tmem + b * 2 * SC, zd = zm + SC;
#pragma unroll 1
                for (int k = 0; k < KS; ++k, ++j) {
                    if (!(ok = wait_phase(&bar[Y_KFULL + j % KST], (j / KST) & 1, abort))) break;
                    const uint32_t xs = sbase + L::XR + (j % KST) * L::K_STAGE;
                    const uint32_t ys = sbase + L::YR + k * L::Y_SLICE;
#pragma unroll
                    for (int kq = 0; kq < 4; ++kq) {
                        const uint64_t yd = desc_sw128(ys + 32u * kq);
                        const uint32_t acc = (k > 0 || kq > 0) ? 1u : 0u;
                        mma_bf16(zm, desc_sw128(xs + 32u * kq), yd, idesc, acc);
                        mma_bf16(zd, desc_sw128(xs + L::X_SLICE + 32u * kq), yd, idesc, acc);
                    }
                    mma_commit(&bar[Y_KEMPTY + j % KST]);
                }
                if (!ok) break;
                mma_commit(&bar[Y_ZFULL + b]);
                const int nsb = m + 1 < nloc ? (u_begin + m + 1) / nob : -1;
                if (nsb != sb) mma_commit(&bar[Y_YEMPTY]);   // Y free once these MMAs finish
            }
            if (!ok) {
                mma_commit(&bar[Y_DRAIN]);
                drain_phase(&bar[Y_DRAIN], 0);
            }
        }
    } else if (warp < W_EPI) {
        // epilogue warp: lanes o = o0 + 32 qd + lane, values s = 32 cg .. 32 cg + 31 of the
        // unit's s-block, in two halves of 16
        const int qd = warp & 3, cg = warp >> 2;
        const int row = 32 * qd + lane;
        const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
        auto v_src = [&](int m, int h, const float*& p, int& n) {
            const int u = u_begin + m;
            const int64_t o = (int64_t)(u % nob) * OBLK + row;
            const int64_t s0 = (int64_t)(u / nob) * SC + 32 * cg + 16 * h;
            const int64_t left = a.S - s0;
            p = a.V + s0 * a.vs + o;
            n = o < a.O ? (left < 16 ? (left > 0 ? (int)left : 0) : 16) : 0;
        };
        float vn[16];   // v of the half being processed, then of the next one
        if (nloc > 0) {
            const float* p;
            int n;
            v_src(0, 0, p, n);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) vn[jj] = jj < n ? __ldg(p + jj * a.vs) : 0.f;
        }
        bool bad = false;
        for (int m = 0; m < nloc; ++m) {
            const int b = m & 1;
            bool ok = wait_phase(&bar[Y_ZFULL + b], (m >> 1) & 1, abort);
            ok = __all_sync(0xffffffffu, ok);   // keep the warp converged
            tc_fence_after();
            const uint32_t zbase = tmem + b * 2 * SC + lane_off;
            float run_m = 0.f, run_d = 0.f;
#pragma unroll 1
            for (int h = 0; ok && h < 2; ++h) {
                const uint32_t col = zbase + 32 * cg + 16 * h;
                uint32_t zm[16], zd[16];
                tmem_ld16(col, zm);
                tmem_ld16(col + SC, zd);
                const float* pn = a.V;   // the next half's v
                int nn = 0;
                if (h == 0)
                    v_src(m, 1, pn, nn);
                else if (m + 1 < nloc)
                    v_src(m + 1, 0, pn, nn);
                tmem_ld_wait();
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const float v = vn[jj];
                    vn[jj] = jj < nn ? __ldg(pn + jj * a.vs) : 0.f;
                    const float z1 = __uint_as_float(zm[jj]), z2 = __uint_as_float(zd[jj]);
                    const bool pos = v > 0.f;
                    bad |= pos && !(z1 > 0.f && z2 > 0.f);
                    run_m += pos ? z1 - v * (LN2F * lg2_ftz(z1)) : z1;
                    run_d += pos ? z2 - v * (LN2F * lg2_ftz(z2)) : z2;
                }
            }
            // the four partials of each column meet in the first two columns each warp read;
            // every epilogue warp reaches the barrier of every unit, and all of them leave
            // together if any one gave up waiting
            if (ok) {
                tmem_st2(zbase + 32 * cg, __float_as_uint(run_m), __float_as_uint(run_d));
                tmem_st_wait();
            }
            tc_fence_before();
            const bool fail = named_any(1, 32 * W_EPI, !ok);
            tc_fence_after();
            if (fail) break;
            if (cg == 0) {
                uint32_t pm[4], pd[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) tmem_ld2(zbase + 32 * k, pm[k], pd[k]);
                tmem_ld_wait();
                double acc_m = 0.0, acc_d = 0.0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    acc_m += (double)__uint_as_float(pm[k]);
                    acc_d += (double)__uint_as_float(pd[k]);
                }
                const int u = u_begin + m;
                const int64_t o = (int64_t)(u % nob) * OBLK + row, sb = u / nob;
                if (o < a.O) {
                    a.dpart[(sb * 2 + 0) * a.O + o] = acc_m;
                    a.dpart[(sb * 2 + 1) * a.O + o] = acc_d;
                }
            }
            // the unit is read: buffer free for unit m + 2
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[Y_ZEMPTY + b]);
        }
        if (bad) atomicOr(a.status, STATUS_NONFINITE);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(a.status, STATUS_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

int launch_pass2_yr(const P2Args& a, const TcMaps& m, int64_t O_pad, int ctas, cudaStream_t st) {
    const uint32_t smem = ks::LayoutY::TOTAL + 1024;
    if (cudaFuncSetAttribute(k_tc_pass2_yr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return DNA_ERR_CUDA;
    const int nob = (int)(O_pad / OBLK);
    const int64_t nsb = (a.S + ks::SC - 1) / ks::SC;
    const int64_t nunits = nsb * nob;
    if (nunits == 0) return DNA_OK;
    if (nunits > INT32_MAX) return DNA_ERR_ARG;
    const int grid = (int)std::min<int64_t>(ctas > 0 ? ctas : nunits, nunits);
    k_tc_pass2_yr<<<grid, ks::P2K_THREADS, smem, st>>>(a, nob, (int)nunits, m.xm, m.xd, m.y);
    return after_launch();
}

}  // namespace tc

int TcBf16::pass2_large(const TcOperands& op, const TcMaps& maps, double* dpart, int slots,
                        int64_t s_per, int* status, cudaStream_t st) {
    tc::P2Args a{};
    a.S = op.S; a.O = op.O; a.R = op.R; a.s_per = s_per;
    a.dpart = dpart; a.status = status;
    a.V = op.V; a.vs = op.vs; a.Xm = op.Xmk; a.Xd = op.Xdk; a.rp = rank_pad(op.R);
    if (!op.plane && a.rp == 512) {   // BF16: Y resident, one cost slot per 128 values of s
        if (s_per != tc::ks::SC || slots != (op.S + tc::ks::SC - 1) / tc::ks::SC)
            return DNA_ERR_ARG;
        return tc::launch_pass2_yr(a, maps, op.O_pad, op.ctas, st);
    }
    if (s_per % tc::ks::SC != 0 || slots % 4 != 0) return DNA_ERR_ARG;
    const int splits = slots / 4;
    if (splits != (int)((op.S + s_per - 1) / s_per)) return DNA_ERR_ARG;
    if (op.plane) {   // the FP32 form on the tensor cores
        if (a.rp == 256) return tc::launch_pass2_kt<256, true>(a, maps, op.O_pad, splits, op.ctas, st);
        if (a.rp == 512) return tc::launch_pass2_kt<512, true>(a, maps, op.O_pad, splits, op.ctas, st);
        return DNA_ERR_UNSUPPORTED;
    }
    return DNA_ERR_UNSUPPORTED;
}

}  // namespace dna
