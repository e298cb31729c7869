// tcgen05 tensor-core kernels of the DNA half-step, BF16 operands with FP32 accumulation
// in TMEM (the precision form), for padded rank RP in {64, 128}.
//
// Pass 1 (Algorithm 1 steps 2-5 and 10), per CTA = 128 values of o (the TMEM lanes) and
// an s-range:
//   GEMM1  Z[o, s]  = sum_r X[o, r] Y[s, r]            M = 128, N = 64 (one s-chunk), K = RP
//   epilogue (4 warps, thread = lane = o): z from TMEM, v from shared memory,
//          q = v / z, qbar = q / z (0 where v = 0), rounded to bf16 into shared memory
//   GEMM2  A[o, r] += sum_s Q[o, s] Yt[r, s]           M = 128, N = RP, K = 64
//   GEMM3  B[o, r] += sum_s Qbar[o, s] Y2t[r, s]       (Y2t = (Y o Y)^t)
// A and B stay in TMEM for the whole s-range; Z and Q never reach global memory.
// Pass 2 (steps 7-9, 12-14): Zmu = Xmu Y^t and Zdna = Xdna Y^t into TMEM, then per lane
// (= column o) the cost terms -v log z + z, summed in float32 over a chunk and in float64
// across chunks.
// Operands are K-major tiles in the 128-byte swizzled layout, staged with cp.async; one
// thread issues the MMAs; completion is tracked by an mbarrier with a bounded wait.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dna_internal.h"
#include "tc_ptx.cuh"

namespace dna {
namespace tc {

constexpr int OBLK = 128;  // o per CTA (MMA M, TMEM lanes)
constexpr int SCH = 64;    // s per chunk (GEMM1 N, GEMM2 K)
constexpr int NTH = 128;   // 4 warps: thread i owns TMEM lane i
constexpr long long WAIT_LIMIT = 4000000000LL;  // SM cycles (about 2 s) per wait

using bf16 = __nv_bfloat16;

// Load a ROWS x KE (bf16) K-major tile from row-major global memory (leading dimension
// ld elements) into the swizzled layout at shared address sbase.  The global tile must be
// fully inside the (padded) allocation.
template <int ROWS, int KE>
__device__ __forceinline__ void load_kmajor(uint32_t sbase, const bf16* __restrict__ g,
                                            int64_t ld) {
    constexpr int CPR = KE / 8;  // 16-byte chunks per row
    for (int c = threadIdx.x; c < ROWS * CPR; c += NTH) {
        const int row = c / CPR, kc = c % CPR;
        cp_async16(sbase + sw128_offset(row, kc, ROWS), g + (int64_t)row * ld + kc * 8, 16);
    }
}

// V tile: SCH rows (s) x 128 columns (o) of float32, row-major in shared memory.  Rows at
// or beyond s_end and 4-column groups starting at or beyond O are zero-filled.
__device__ __forceinline__ void load_v_tile(uint32_t sbase, const float* __restrict__ V,
                                            int64_t vs, int64_t s0, int64_t s_end, int64_t o0,
                                            int64_t O) {
    for (int c = threadIdx.x; c < SCH * (OBLK / 4); c += NTH) {
        const int row = c / (OBLK / 4), cc = c % (OBLK / 4);
        const int64_t s = s0 + row, o = o0 + cc * 4;
        const bool ok = s < s_end && o < O;
        const float* src = ok ? V + s * vs + o : V;
        cp_async16(sbase + (uint32_t)(row * OBLK + cc * 4) * 4u, src, ok ? 16u : 0u);
    }
}

struct P1Args {
    int64_t S, O, R, S_pad, s_per;
    const bf16* Xk;    // [O_pad][RP]
    const bf16* Yk;    // [S_pad][RP]
    const bf16* Ytk;   // [RP][S_pad]
    const bf16* Y2tk;  // [RP][S_pad]
    const float* V;    // V_so, leading dimension vs (multiple of 4), 16-byte aligned
    int64_t vs;
    float* Apart;      // [splits][R][O]
    float* Bpart;
    int* status;
};

template <int RP>
struct P1Smem {
    static constexpr uint32_t X = 0;
    static constexpr uint32_t Y = X + OBLK * RP * 2;
    static constexpr uint32_t YT = Y + SCH * RP * 2;
    static constexpr uint32_t Y2T = YT + RP * SCH * 2;
    static constexpr uint32_t Q = Y2T + RP * SCH * 2;
    static constexpr uint32_t QB = Q + OBLK * SCH * 2;
    static constexpr uint32_t VT = QB + OBLK * SCH * 2;
    static constexpr uint32_t BAR = VT + SCH * OBLK * 4;
    static constexpr uint32_t TOTAL = BAR + 64;
    static constexpr uint32_t NCOLS = (SCH + 2 * RP) <= 256 ? 256 : 512;
};

template <int RP, bool WITH_B>
__global__ void __launch_bounds__(NTH, 1) k_tc_pass1(P1Args a) {
    using L = P1Smem<RP>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + 16);
    const float* Vs = reinterpret_cast<const float*>(sm + L::VT);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t o0 = (int64_t)blockIdx.x * OBLK;
    const int64_t o = o0 + tid;
    const int64_t s_begin = (int64_t)blockIdx.y * a.s_per;
    const int64_t s_end = min(a.S, s_begin + a.s_per);
    const int nchunks = s_end > s_begin ? (int)((s_end - s_begin + SCH - 1) / SCH) : 0;

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == 0) { mbar_init(bar, 1); fence_mbar_init(); }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tZ = tmem, tA = tmem + SCH, tB = tmem + SCH + RP;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;

    load_kmajor<OBLK, RP>(sbase + L::X, a.Xk + o0 * RP, RP);
    uint32_t phase = 0;
    bool ok = true;
    int bad = 0;
    for (int ci = 0; ci < nchunks && ok; ++ci) {
        const int64_t s0 = s_begin + (int64_t)ci * SCH;
        load_kmajor<SCH, RP>(sbase + L::Y, a.Yk + s0 * RP, RP);
        load_kmajor<RP, SCH>(sbase + L::YT, a.Ytk + s0, a.S_pad);
        if (WITH_B) load_kmajor<RP, SCH>(sbase + L::Y2T, a.Y2tk + s0, a.S_pad);
        load_v_tile(sbase + L::VT, a.V, a.vs, s0, s_end, o0, a.O);
        cp_async_commit();
        cp_async_wait_all();
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {  // GEMM1: Z = X Y^t over K = RP
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < RP / 16; ++k) {
                const uint32_t kb = 32u * k, atom = kb >> 7, within = kb & 127u;
                mma_bf16(tZ, desc_sw128(sbase + L::X + atom * OBLK * 128 + within),
                         desc_sw128(sbase + L::Y + atom * SCH * 128 + within),
                         idesc_bf16(OBLK, SCH), k > 0);
            }
            mma_commit(bar);
        }
        ok = mbar_wait_bounded(bar, phase, WAIT_LIMIT);
        phase ^= 1;
        ok = __syncthreads_and(ok);
        if (!ok) break;
        tc_fence_after();
        // epilogue: q and qbar for row o, s = s0 .. s0 + 63
#pragma unroll
        for (int h = 0; h < SCH / 32; ++h) {
            uint32_t zr[32];
            tmem_ld32(tZ + lane_off + 32 * h, zr);
            tmem_ld_wait();
            uint32_t qp[16], qbp[16];
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
                float q[2], qb[2];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int sl = 32 * h + j + t;
                    float v = Vs[sl * OBLK + tid];
                    if (o >= a.O) v = 0.f;
                    const float z = __uint_as_float(zr[j + t]);
                    q[t] = 0.f;
                    qb[t] = 0.f;
                    if (v > 0.f) {
                        if (z > 0.f) { q[t] = __fdividef(v, z); qb[t] = __fdividef(q[t], z); }
                        else bad = 1;
                    }
                }
                qp[j / 2] = pack_bf16x2(q[0], q[1]);
                qbp[j / 2] = pack_bf16x2(qb[0], qb[1]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t off = sw128_offset(tid, 4 * h + c, OBLK);
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sbase + L::Q + off),
                             "r"(qp[4 * c]), "r"(qp[4 * c + 1]), "r"(qp[4 * c + 2]),
                             "r"(qp[4 * c + 3])
                             : "memory");
                if (WITH_B)
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                                     sbase + L::QB + off),
                                 "r"(qbp[4 * c]), "r"(qbp[4 * c + 1]), "r"(qbp[4 * c + 2]),
                                 "r"(qbp[4 * c + 3])
                                 : "memory");
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {  // GEMM2 / GEMM3 over K = 64 (this chunk)
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < SCH / 16; ++k) {
                const uint32_t kb = 32u * k;
                mma_bf16(tA, desc_sw128(sbase + L::Q + kb), desc_sw128(sbase + L::YT + kb),
                         idesc_bf16(OBLK, RP), (ci > 0 || k > 0) ? 1u : 0u);
                if (WITH_B)
                    mma_bf16(tB, desc_sw128(sbase + L::QB + kb), desc_sw128(sbase + L::Y2T + kb),
                             idesc_bf16(OBLK, RP), (ci > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(bar);
        }
        ok = mbar_wait_bounded(bar, phase, WAIT_LIMIT);
        phase ^= 1;
        ok = __syncthreads_and(ok);
    }
    if (bad) atomicOr(a.status, STATUS_NONFINITE);
    if (!ok) {
        if (tid == 0) atomicOr(a.status, STATUS_TIMEOUT);
    } else if (nchunks > 0) {
        tc_fence_after();
        const int64_t base = (int64_t)blockIdx.y * a.R;
#pragma unroll
        for (int g = 0; g < RP / 32; ++g) {
            uint32_t r32[32];
            tmem_ld32(tA + lane_off + 32 * g, r32);
            tmem_ld_wait();
            if (o < a.O)
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int64_t r = 32 * g + i;
                    if (r < a.R) a.Apart[(base + r) * a.O + o] = __uint_as_float(r32[i]);
                }
            if (WITH_B) {
                tmem_ld32(tB + lane_off + 32 * g, r32);
                tmem_ld_wait();
                if (o < a.O)
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int64_t r = 32 * g + i;
                        if (r < a.R) a.Bpart[(base + r) * a.O + o] = __uint_as_float(r32[i]);
                    }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

struct P2Args {
    int64_t S, O, R, s_per;
    const bf16* Xmk;   // [O_pad][RP] MU candidate
    const bf16* Xdk;   // [O_pad][RP] Newton candidate
    const bf16* Yk;    // [S_pad][RP]
    const float* V;
    int64_t vs;
    double* dpart;     // [splits][2][O]
    int* status;
};

template <int RP>
struct P2Smem {
    static constexpr uint32_t XM = 0;
    static constexpr uint32_t XD = XM + OBLK * RP * 2;
    static constexpr uint32_t Y = XD + OBLK * RP * 2;
    static constexpr uint32_t VT = Y + SCH * RP * 2;
    static constexpr uint32_t BAR = VT + SCH * OBLK * 4;
    static constexpr uint32_t TOTAL = BAR + 64;
    static constexpr uint32_t NCOLS = 2 * SCH;
};

template <int RP>
__global__ void __launch_bounds__(NTH, 1) k_tc_pass2(P2Args a) {
    using L = P2Smem<RP>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(sm);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + 16);
    const float* Vs = reinterpret_cast<const float*>(sm + L::VT);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t o0 = (int64_t)blockIdx.x * OBLK;
    const int64_t o = o0 + tid;
    const int64_t s_begin = (int64_t)blockIdx.y * a.s_per;
    const int64_t s_end = min(a.S, s_begin + a.s_per);
    const int nchunks = s_end > s_begin ? (int)((s_end - s_begin + SCH - 1) / SCH) : 0;

    if (warp == 0) { tmem_alloc(tslot, L::NCOLS); tmem_relinquish(); }
    if (tid == 0) { mbar_init(bar, 1); fence_mbar_init(); }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tM = tmem, tD = tmem + SCH;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;

    load_kmajor<OBLK, RP>(sbase + L::XM, a.Xmk + o0 * RP, RP);
    load_kmajor<OBLK, RP>(sbase + L::XD, a.Xdk + o0 * RP, RP);
    double acc_m = 0.0, acc_d = 0.0;
    uint32_t phase = 0;
    bool ok = true;
    int bad = 0;
    for (int ci = 0; ci < nchunks && ok; ++ci) {
        const int64_t s0 = s_begin + (int64_t)ci * SCH;
        load_kmajor<SCH, RP>(sbase + L::Y, a.Yk + s0 * RP, RP);
        load_v_tile(sbase + L::VT, a.V, a.vs, s0, s_end, o0, a.O);
        cp_async_commit();
        cp_async_wait_all();
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < RP / 16; ++k) {
                const uint32_t kb = 32u * k, atom = kb >> 7, within = kb & 127u;
                const uint64_t yd = desc_sw128(sbase + L::Y + atom * SCH * 128 + within);
                mma_bf16(tM, desc_sw128(sbase + L::XM + atom * OBLK * 128 + within), yd,
                         idesc_bf16(OBLK, SCH), k > 0);
                mma_bf16(tD, desc_sw128(sbase + L::XD + atom * OBLK * 128 + within), yd,
                         idesc_bf16(OBLK, SCH), k > 0);
            }
            mma_commit(bar);
        }
        ok = mbar_wait_bounded(bar, phase, WAIT_LIMIT);
        phase ^= 1;
        ok = __syncthreads_and(ok);
        if (!ok) break;
        tc_fence_after();
        float run_m = 0.f, run_d = 0.f;
#pragma unroll
        for (int h = 0; h < SCH / 32; ++h) {
            uint32_t zm[32], zd[32];
            tmem_ld32(tM + lane_off + 32 * h, zm);
            tmem_ld32(tD + lane_off + 32 * h, zd);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float v = Vs[(32 * h + j) * OBLK + tid];
                if (o >= a.O) v = 0.f;
                const float z1 = __uint_as_float(zm[j]), z2 = __uint_as_float(zd[j]);
                float t1 = z1, t2 = z2;
                if (v > 0.f) {
                    if (z1 > 0.f && z2 > 0.f) {
                        t1 -= v * __logf(z1);
                        t2 -= v * __logf(z2);
                    } else {
                        bad = 1;
                    }
                }
                run_m += t1;
                run_d += t2;
            }
        }
        acc_m += (double)run_m;
        acc_d += (double)run_d;
        tc_fence_before();
        __syncthreads();  // the next chunk overwrites Y and V in shared memory
    }
    if (bad) atomicOr(a.status, STATUS_NONFINITE);
    if (!ok) {
        if (tid == 0) atomicOr(a.status, STATUS_TIMEOUT);
    } else if (o < a.O) {
        a.dpart[((int64_t)blockIdx.y * 2 + 0) * a.O + o] = acc_m;
        a.dpart[((int64_t)blockIdx.y * 2 + 1) * a.O + o] = acc_d;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, L::NCOLS);
}

// dst[i][j] (leading dimension ld, padded to rows_pad x cols_pad with zeros) =
// bf16(src(i, j)) (squared first when `square`), where src(i, j) = src[i * si + j * sj]
// for i < rows, j < cols, and one of si, sj is 1.  32 x 32 tiles through shared memory.
__global__ void k_to_bf16(const float* __restrict__ src, int64_t si, int64_t sj, int64_t rows,
                          int64_t cols, bf16* __restrict__ dst, int64_t ld, bool square) {
    __shared__ float tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
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

template <int RP, bool WITH_B>
int launch_pass1(const P1Args& a, int64_t O_pad, int splits, cudaStream_t st) {
    const uint32_t smem = P1Smem<RP>::TOTAL + 1024;
    auto k = k_tc_pass1<RP, WITH_B>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    dim3 grid((unsigned)(O_pad / OBLK), (unsigned)splits);
    k<<<grid, NTH, smem, st>>>(a);
    return after_launch();
}

template <int RP>
int launch_pass2(const P2Args& a, int64_t O_pad, int splits, cudaStream_t st) {
    const uint32_t smem = P2Smem<RP>::TOTAL + 1024;
    auto k = k_tc_pass2<RP>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    dim3 grid((unsigned)(O_pad / OBLK), (unsigned)splits);
    k<<<grid, NTH, smem, st>>>(a);
    return after_launch();
}

}  // namespace tc

int TcBf16::rank_pad(int64_t R) { return R <= 64 ? 64 : (R <= 128 ? 128 : 0); }

int TcBf16::to_bf16(const float* src, int64_t si, int64_t sj, int64_t rows, int64_t cols,
                    void* dst, int64_t ld, int64_t rows_pad, int64_t cols_pad, bool square,
                    cudaStream_t st) {
    dim3 blk(32, 8);
    dim3 grid((unsigned)((cols_pad + 31) / 32), (unsigned)((rows_pad + 31) / 32));
    tc::k_to_bf16<<<grid, blk, 0, st>>>(src, si, sj, rows, cols, static_cast<tc::bf16*>(dst), ld,
                                         square);
    return after_launch();
}

int TcBf16::pass1(const TcOperands& op, const float* V, int64_t vs, float* Apart, float* Bpart,
                  int splits, int64_t s_per, bool with_b, int* status, cudaStream_t st) {
    tc::P1Args a{};
    a.S = op.S; a.O = op.O; a.R = op.R; a.S_pad = op.S_pad; a.s_per = s_per;
    a.Xk = static_cast<const tc::bf16*>(op.Xk);
    a.Yk = static_cast<const tc::bf16*>(op.Yk);
    a.Ytk = static_cast<const tc::bf16*>(op.Ytk);
    a.Y2tk = static_cast<const tc::bf16*>(op.Y2tk);
    a.V = V; a.vs = vs; a.Apart = Apart; a.Bpart = Bpart; a.status = status;
    const int rp = rank_pad(op.R);
    if (rp == 64)
        return with_b ? tc::launch_pass1<64, true>(a, op.O_pad, splits, st)
                      : tc::launch_pass1<64, false>(a, op.O_pad, splits, st);
    if (rp == 128)
        return with_b ? tc::launch_pass1<128, true>(a, op.O_pad, splits, st)
                      : tc::launch_pass1<128, false>(a, op.O_pad, splits, st);
    return DNA_ERR_UNSUPPORTED;
}

int TcBf16::pass2(const TcOperands& op, const void* Xmk, const void* Xdk, const float* V,
                  int64_t vs, double* dpart, int splits, int64_t s_per, int* status,
                  cudaStream_t st) {
    tc::P2Args a{};
    a.S = op.S; a.O = op.O; a.R = op.R; a.s_per = s_per;
    a.Xmk = static_cast<const tc::bf16*>(Xmk);
    a.Xdk = static_cast<const tc::bf16*>(Xdk);
    a.Yk = static_cast<const tc::bf16*>(op.Yk);
    a.V = V; a.vs = vs; a.dpart = dpart; a.status = status;
    const int rp = rank_pad(op.R);
    if (rp == 64) return tc::launch_pass2<64>(a, op.O_pad, splits, st);
    if (rp == 128) return tc::launch_pass2<128>(a, op.O_pad, splits, st);
    return DNA_ERR_UNSUPPORTED;
}

int TcBf16::chunk() { return tc::SCH; }
int TcBf16::oblock() { return tc::OBLK; }

}  // namespace dna
