// Kernels of the sparse-V form (a DNA half-step that touches only the non-zeros of V).
//
// A half-step over the (s, o) view of Section 2 (H-step: o = column t, s = row n; W-step:
// o = row n, s = column t) needs z = (W H)_so only where v_so != 0: the ratios q = v/z and
// qbar = v/z^2 (steps 3, 10) are 0 elsewhere (the note after Algorithm 1), so A and B
// (eq. 7, 14) are sums over the non-zeros of the column, and so is the -v log z part of the
// candidates' costs (steps 9, 14).  The sum z part needs no zeros either:
// sum_s z_so = sum_r (sum_s y_sr) x_ro = sum_r c0_r x_ro with c0 the column sums of Y.
//
// Storage: the non-zeros of view column o are k in [ptr[o], ptr[o + 1]), at s = idx[k] with
// value val[k] (CSC of V for the H-step, CSR of V for the W-step); Yg is the fixed factor
// as an S x R row-major array (W for the H-step, a transposed copy of H for the W-step),
// so the R values of y(s, .) are one contiguous, coalesced row.
//
// Work is split into segments of at most SEG non-zeros of one view column (term rows of
// count data follow a Zipf law: one row can hold thousands of non-zeros), one warp per
// segment; lane l holds r = l + 32 j (j < RPL).  Each segment writes its partial sums
// [seg][R], and a warp per view column then adds its segments in order.  Dot products over
// r are reduced with a fixed xor butterfly, so every result is bit-reproducible.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dna_internal.h"

namespace dna {
namespace sparse {

constexpr int WARPS = 8;   // warps (segments or view columns) per CTA
constexpr int U = 8;       // non-zeros whose loads are issued together
constexpr int SEG = SPARSE_SEG;

template <typename Tp>
__device__ __forceinline__ Tp warp_sum(Tp x) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) x += __shfl_xor_sync(0xffffffffu, x, m);
    return x;
}

// The non-zeros of a segment are read 32 at a time with one coalesced load (lane l holds
// the index and value of non-zero k + l) and handed to the whole warp by shuffles; the
// next 32 are loaded while the current ones are used, so each batch of U non-zeros waits
// only for its gathered rows y(s, .).
template <typename Tp>
struct Chunk {
    int32_t s;
    Tp v;
};

template <typename Tp>
__device__ __forceinline__ Chunk<Tp> load_chunk(int64_t k, int64_t k1, int lane,
                                                const int32_t* __restrict__ idx,
                                                const Tp* __restrict__ val) {
    Chunk<Tp> c;
    const bool in = k + lane < k1;
    c.s = in ? idx[k + lane] : 0;
    c.v = in ? val[k + lane] : Tp(0);
    return c;
}

// The rows y(s, .) gathered by the U non-zeros base .. base + U - 1 of chunk c (row 0 past
// the segment's end, where the chunk holds s = 0 and v = 0).
template <typename Tp, int RPL>
__device__ __forceinline__ void gather_batch(const Chunk<Tp>& c, int base, int lane, int64_t R,
                                             const Tp* __restrict__ Yg, Tp (&y)[U][RPL]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t s = __shfl_sync(0xffffffffu, c.s, base + u);
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int64_t r = lane + 32 * j;
            y[u][j] = r < R ? Yg[s * R + r] : Tp(0);
        }
    }
}

// Sums each of the NV per-lane values p[i] over the warp (NV a power of two <= 32) with a
// fixed reduce-scatter: at the step with xor mask m the lanes with bit m set keep the upper
// half of the remaining values and the others the lower half, each adding its partner's
// copy of the half it keeps; after log2(NV) steps a lane holds one value, index
// lane >> (5 - log2(NV)), and the remaining xor steps complete its sum over all 32 lanes.
// NV + 5 - log2(NV) - 1 shuffles for NV values instead of 5 NV.
template <typename Tp, int NV>
__device__ __forceinline__ Tp scatter_sum(Tp (&p)[NV], int lane) {
    static_assert(NV >= 1 && NV <= 32 && (NV & (NV - 1)) == 0, "NV: a power of two <= 32");
    int m = 16;
#pragma unroll
    for (int cnt = NV; cnt > 1; cnt >>= 1, m >>= 1) {
        const bool hi = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < cnt / 2; ++i) {
            const Tp keep = hi ? p[i + cnt / 2] : p[i];
            const Tp send = hi ? p[i] : p[i + cnt / 2];
            p[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
    Tp t = p[0];
#pragma unroll
    for (; m > 0; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
    return t;
}

// Runs body(chunk, base, y) over the non-zeros [k0, k1) in batches of U.
template <typename Tp, int RPL, class F>
__device__ __forceinline__ void for_nonzeros(int64_t k0, int64_t k1, int lane, int64_t R,
                                             const int32_t* __restrict__ idx,
                                             const Tp* __restrict__ val,
                                             const Tp* __restrict__ Yg, F&& body) {
    Chunk<Tp> cur = load_chunk<Tp>(k0, k1, lane, idx, val);
    for (int64_t k = k0; k < k1; k += 32) {
        const Chunk<Tp> nxt = load_chunk<Tp>(k + 32, k1, lane, idx, val);
        const int n = (int)(k1 - k < 32 ? k1 - k : 32);
        for (int base = 0; base < n; base += U) {
            Tp y[U][RPL];
            gather_batch<Tp, RPL>(cur, base, lane, R, Yg, y);
            body(cur, base, y);
        }
        cur = nxt;
    }
}

using Segs = SparseSegs;

// Pass 1 (Algorithm 1 steps 2-5 and 10 on the non-zeros of one segment): partial raw sums
// Aseg[g][r] = sum_k y(s_k, r) q_k and Bseg[g][r] = sum_k y(s_k, r)^2 qbar_k with q = v / z,
// qbar = q / z.  Sets STATUS_NONFINITE when z <= 0 (or is not a number) at a positive v.
template <typename Tp, int RPL>
__global__ void __launch_bounds__(WARPS * 32)
    k_sp_pass1(View v, Segs sg, const int32_t* __restrict__ idx, const Tp* __restrict__ val,
               const Tp* __restrict__ Yg, Tp* __restrict__ Aseg, Tp* __restrict__ Bseg,
               bool with_b, int* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (g >= sg.n) return;
    const int64_t R = v.R, o = sg.col[g];
    const Tp* __restrict__ X = static_cast<const Tp*>(v.X);
    Tp x[RPL], a[RPL], b[RPL];
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int64_t r = lane + 32 * j;
        x[j] = r < R ? X[r * v.xr + o * v.xo] : Tp(0);
        a[j] = Tp(0);
        b[j] = Tp(0);
    }
    bool bad = false;
    constexpr int LOGU = U == 8 ? 3 : (U == 4 ? 2 : (U == 16 ? 4 : -1));
    static_assert(LOGU > 0, "U: 4, 8 or 16");
    const int ul = lane >> (5 - LOGU);   // the non-zero of the batch this lane finishes
    for_nonzeros<Tp, RPL>(sg.k0[g], sg.k1[g], lane, R, idx, val, Yg,
                          [&](const Chunk<Tp>& c, int base, Tp (&y)[U][RPL]) {
        Tp p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            p[u] = Tp(0);
#pragma unroll
            for (int j = 0; j < RPL; ++j) p[u] += y[u][j] * x[j];
        }
        const Tp z = scatter_sum<Tp, U>(p, lane);             // z of non-zero ul
        const Tp vl = __shfl_sync(0xffffffffu, c.v, base + ul);
        Tp q = Tp(0), qb = Tp(0);
        if (vl > Tp(0)) {                                      // v = 0: q = qbar = 0
            if (z > Tp(0)) {
                const Tp rz = Tp(1) / z;                       // q = v / z, qbar = q / z
                q = vl * rz;
                qb = q * rz;
            } else {
                bad = true;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const Tp qu = __shfl_sync(0xffffffffu, q, u << (5 - LOGU));
            const Tp qbu = __shfl_sync(0xffffffffu, qb, u << (5 - LOGU));
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                a[j] += y[u][j] * qu;
                b[j] += y[u][j] * y[u][j] * qbu;
            }
        }
    });
    bad = __any_sync(0xffffffffu, bad);
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int64_t r = lane + 32 * j;
        if (r < R) {
            Aseg[g * R + r] = a[j];
            if (with_b) Bseg[g * R + r] = b[j];
        }
    }
    if (bad && status) atomicOr(status, STATUS_NONFINITE);
}

// A(r, o) = sum over the segments of column o of Aseg (in segment order), written [R][O]
// (split 0 of the dense layout); the same for B.  A warp per view column.
template <typename Tp, int RPL>
__global__ void __launch_bounds__(WARPS * 32)
    k_sp_reduce_ab(int64_t O, int64_t R, const int64_t* __restrict__ sptr,
                   const Tp* __restrict__ Aseg, const Tp* __restrict__ Bseg, Tp* __restrict__ A,
                   Tp* __restrict__ B, bool with_b) {
    const int lane = threadIdx.x & 31;
    const int64_t o = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (o >= O) return;
    Tp a[RPL], b[RPL];
#pragma unroll
    for (int j = 0; j < RPL; ++j) { a[j] = Tp(0); b[j] = Tp(0); }
    for (int64_t g = sptr[o]; g < sptr[o + 1]; ++g) {
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int64_t r = lane + 32 * j;
            if (r < R) {
                a[j] += Aseg[g * R + r];
                if (with_b) b[j] += Bseg[g * R + r];
            }
        }
    }
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int64_t r = lane + 32 * j;
        if (r < R) {
            A[r * O + o] = a[j];
            if (with_b) B[r * O + o] = b[j];
        }
    }
}

// Pass 2 (steps 7-9, 12-14 on the non-zeros of one segment): the partial sums
// dseg[2 g] = sum_{v>0} -v log z_MU and dseg[2 g + 1] = sum_{v>0} -v log z_DNA.  The term
// of non-zero k is added by lane (k - k0) mod U in the element type (at most SEG / U terms
// per lane: float64 arithmetic is slow on this GPU), then the lanes' sums are added in
// float64 by the fixed butterfly.
template <typename Tp, int RPL>
__global__ void __launch_bounds__(WARPS * 32)
    k_sp_pass2(View v, Segs sg, const int32_t* __restrict__ idx, const Tp* __restrict__ val,
               const Tp* __restrict__ Yg, const Tp* __restrict__ Xmu,
               const Tp* __restrict__ Xdna, double* __restrict__ dseg) {
    const int lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (g >= sg.n) return;
    const int64_t R = v.R, O = v.O, o = sg.col[g];
    Tp xm[RPL], xd[RPL];
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int64_t r = lane + 32 * j;
        xm[j] = r < R ? Xmu[r * O + o] : Tp(0);
        xd[j] = r < R ? Xdna[r * O + o] : Tp(0);
    }
    Tp lm_t = Tp(0), ld_t = Tp(0);
    constexpr int LOG2U = U == 8 ? 4 : (U == 4 ? 3 : (U == 16 ? 5 : -1));
    static_assert(LOG2U > 0, "U: 4, 8 or 16");
    // lane l finishes value l >> (5 - LOG2U) of the 2U: the MU z of non-zero u (values
    // 0 .. U - 1) or the Newton z (U .. 2U - 1); one lane of each value adds its term
    const int vi = lane >> (5 - LOG2U), ul = vi & (U - 1);
    const bool adds = (lane & ((1 << (5 - LOG2U)) - 1)) == 0;
    for_nonzeros<Tp, RPL>(sg.k0[g], sg.k1[g], lane, R, idx, val, Yg,
                          [&](const Chunk<Tp>& c, int base, Tp (&y)[U][RPL]) {
        Tp p[2 * U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            p[u] = Tp(0);
            p[U + u] = Tp(0);
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                p[u] += y[u][j] * xm[j];
                p[U + u] += y[u][j] * xd[j];
            }
        }
        const Tp z = scatter_sum<Tp, 2 * U>(p, lane);
        const Tp vl = __shfl_sync(0xffffffffu, c.v, base + ul);
        if (adds && vl > Tp(0)) {   // log of a non-positive z gives NaN / -inf
            const Tp t = vl * log(z);
            if (vi < U) lm_t -= t; else ld_t -= t;
        }
    });
    const double lm = warp_sum((double)lm_t);
    const double ld = warp_sum((double)ld_t);
    if (lane == 0) {
        dseg[2 * g] = lm;
        dseg[2 * g + 1] = ld;
    }
}

// Per view column o: the segments' partial costs in order, plus sum_s z = sum_r c0_r x(r, o)
// of each candidate, into dpart[o] (MU) and dpart[O + o] (Newton).
template <typename Tp, int RPL>
__global__ void __launch_bounds__(WARPS * 32)
    k_sp_reduce_cost(int64_t O, int64_t R, const int64_t* __restrict__ sptr,
                     const double* __restrict__ dseg, const Tp* __restrict__ Xmu,
                     const Tp* __restrict__ Xdna, const double* __restrict__ c0,
                     double* __restrict__ dpart, int* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t o = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (o >= O) return;
    double zm = 0.0, zd = 0.0;
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int64_t r = lane + 32 * j;
        if (r < R) {
            zm += c0[r] * (double)Xmu[r * O + o];
            zd += c0[r] * (double)Xdna[r * O + o];
        }
    }
    zm = warp_sum(zm);
    zd = warp_sum(zd);
    if (lane == 0) {
        double lm = 0.0, ld = 0.0;
        for (int64_t g = sptr[o]; g < sptr[o + 1]; ++g) {
            lm += dseg[2 * g];
            ld += dseg[2 * g + 1];
        }
        const double dm = lm + zm, dd = ld + zd;
        dpart[o] = dm;
        dpart[O + o] = dd;
        if (!isfinite(dm) || !isfinite(dd)) atomicOr(status, STATUS_NONFINITE);
    }
}

// d_KL (eq. 1) of the H view, per segment: sum over its non-zeros of v log(v / z) - v into
// dseg[g] (float64).
template <typename Tp, int RPL>
__global__ void __launch_bounds__(WARPS * 32)
    k_sp_kl(View v, Segs sg, const int32_t* __restrict__ idx, const Tp* __restrict__ val,
            const Tp* __restrict__ Yg, double* __restrict__ dseg) {
    const int lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (g >= sg.n) return;
    const int64_t R = v.R, o = sg.col[g];
    const Tp* __restrict__ X = static_cast<const Tp*>(v.X);
    Tp x[RPL];
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int64_t r = lane + 32 * j;
        x[j] = r < R ? X[r * v.xr + o * v.xo] : Tp(0);
    }
    Tp acc_t = Tp(0);   // the element type within the segment, float64 across lanes
    constexpr int LOGU = U == 8 ? 3 : (U == 4 ? 2 : (U == 16 ? 4 : -1));
    const int ul = lane >> (5 - LOGU);
    const bool adds = (lane & ((1 << (5 - LOGU)) - 1)) == 0;
    for_nonzeros<Tp, RPL>(sg.k0[g], sg.k1[g], lane, R, idx, val, Yg,
                          [&](const Chunk<Tp>& c, int base, Tp (&y)[U][RPL]) {
        Tp p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            p[u] = Tp(0);
#pragma unroll
            for (int j = 0; j < RPL; ++j) p[u] += y[u][j] * x[j];
        }
        const Tp z = scatter_sum<Tp, U>(p, lane);
        const Tp vl = __shfl_sync(0xffffffffu, c.v, base + ul);
        if (adds && vl > Tp(0)) acc_t += vl * log(vl / z) - vl;
    });
    const double acc = warp_sum((double)acc_t);
    if (lane == 0) dseg[g] = acc;
}

// Per column t of the H view: its segments' d_KL terms plus sum_n z_nt = sum_r c0_r h(r, t)
// into part[t].
template <typename Tp, int RPL>
__global__ void __launch_bounds__(WARPS * 32)
    k_sp_reduce_kl(View v, const int64_t* __restrict__ sptr, const double* __restrict__ dseg,
                   const double* __restrict__ c0, double* __restrict__ part,
                   int* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t o = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (o >= v.O) return;
    const Tp* __restrict__ X = static_cast<const Tp*>(v.X);
    double zs = 0.0;
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int64_t r = lane + 32 * j;
        if (r < v.R) zs += c0[r] * (double)X[r * v.xr + o * v.xo];
    }
    zs = warp_sum(zs);
    if (lane == 0) {
        double acc = 0.0;
        for (int64_t g = sptr[o]; g < sptr[o + 1]; ++g) acc += dseg[g];
        const double d = acc + zs;
        part[o] = d;
        if (!isfinite(d)) atomicOr(status, STATUS_NONFINITE);
    }
}

// Y^t: out[t * R + r] = H[r * T + t] (R x T row-major in, T x R row-major out), through
// 32 x 32 shared-memory tiles so both sides stay coalesced.  CTA (32, 8).
template <typename Tp>
__global__ void __launch_bounds__(256) k_transpose(const Tp* __restrict__ in, int64_t rows,
                                                   int64_t cols, Tp* __restrict__ out) {
    __shared__ Tp tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? in[r * cols + c] : Tp(0);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[c * rows + r] = tile[threadIdx.x][i];
    }
}

}  // namespace sparse
}  // namespace dna
