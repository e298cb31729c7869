// Device-side pieces shared by the tcgen05 kernels (tc_bf16.cu, tc_split.cu): tile
// constants, bounded barrier waits, kernel argument blocks, and the copy of an operand
// row block into tensor memory.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "dna_internal.h"
#include "tc_ptx.cuh"

namespace dna {
namespace tc {

constexpr int OBLK = 128;      // o per CTA (MMA M, TMEM lanes)
constexpr int SCH = 64;        // s per chunk (GEMM1 N, GEMM2 K)
constexpr long long WAIT_LIMIT = 4000000000LL;  // SM cycles (about 2 s) per wait

using bf16 = __nv_bfloat16;

// Wait for a barrier phase; give up when another thread of the CTA has aborted or after
// WAIT_LIMIT cycles (then abort the CTA).
// A phase that has already completed costs only the non-blocking test: the suspending
// try_wait costs a couple of hundred cycles even then.
__device__ __forceinline__ bool wait_phase_limit(uint64_t* bar, uint32_t parity,
                                                 volatile int* abort, long long limit) {
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > limit) {
            *abort = 1;
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort) {
    return wait_phase_limit(bar, parity, abort, WAIT_LIMIT);
}

// After an abort: wait (bounded, ignoring the abort flag) for a phase that was armed, so
// that no TMA copy or MMA is still writing when the CTA releases its memory.
__device__ __forceinline__ void drain_phase(uint64_t* bar, uint32_t parity) {
    mbar_wait_bounded(bar, parity, WAIT_LIMIT / 4);
}

struct P1Args {
    int64_t S, O, R, s_per;
    float* Apart;   // [splits][R][O]
    float* Bpart;
    int* status;
    const float* V;   // V_so, element (s, o) at V[s * vs + o]
    int64_t vs;
    const void* X;    // bf16 X operand [O_pad][rp]
    int64_t rp;
};

struct P2Args {
    int64_t S, O, R, s_per;
    double* dpart;  // [splits][2][O]
    int* status;
    const float* V;
    int64_t vs;
    const void* Xm;   // bf16 candidates [O_pad][rp]
    const void* Xd;
    int64_t rp;
};

// ---------------------------------------------------------------- RP in {64, 128}
// Sixteen epilogue warps (four per TMEM lane quadrant, each taking 16 of the 64 chunk
// columns), then the TMA producer warp and the MMA-issuing warps.
//
// Three costs shape these kernels.  Shared-memory bandwidth: the o-block's X (X_mu,
// X_dna) is copied once into tensor memory and read by the MMAs from there, and Q, Qbar
// are written by the epilogue straight into tensor memory, so only V and the per-chunk B
// operands (Y, Y^t, (Y o Y)^t) pass through shared memory, all by TMA.  Group boundaries:
// each wait, fence or commit of an MMA-issuing thread costs the tensor pipe a few hundred
// cycles, so each issuing thread waits on at most two barriers and commits once per chunk.
// Issue concurrency: two issuing threads (one per independent GEMM chain) keep the tensor
// pipe busy while the other one is at a boundary.
constexpr int W_EPI = 16;
constexpr int W_PRODUCER = W_EPI;
constexpr int P1_THREADS = (W_EPI + 3) * 32;      // producer + two MMA warps
constexpr int W_MMA_Z = W_EPI + 1, W_MMA_AB = W_EPI + 2;

// v -> (hi, lo) bf16 pairs of two values: hi = bf16(v), lo = bf16(v - hi) (the operand
// split of the FP32 form on the tensor cores).
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
    hi = pack_bf16x2(v0, v1);
    const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
    lo = pack_bf16x2(v0 - h0, v1 - h1);
}

// X rows [o][rp] (bf16, global) -> tensor memory, 16-column unit `unit` (32 values of r)
// of the lane quadrant addressed by taddr.
__device__ __forceinline__ void x_to_tmem(const bf16* __restrict__ X, int64_t rp, int64_t o,
                                          int unit, uint32_t taddr) {
    const uint4* src = reinterpret_cast<const uint4*>(X + o * rp + 32 * unit);
    uint32_t w[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint4 q = src[i];
        w[4 * i] = q.x; w[4 * i + 1] = q.y; w[4 * i + 2] = q.z; w[4 * i + 3] = q.w;
    }
    tmem_st16(taddr + 16 * unit, w);
}

}  // namespace tc
}  // namespace dna
