// Fused per-half-step kernels between the two O(NRT) passes, for the single-problem path:
//   k_cand_fused   candidates (steps 6 and 11, eq. 10, 11, 15, 17) and, for the tensor-core
//                  form, their bf16 operand copies;
//   k_select_fused selection (steps 15 / 28) and the per-block partial sums of the new
//                  factor that the step 16 / 29 normalisation divides by;
//   k_scale_ops    the normalisation itself (X by 1/f_r, Y by f_r) fused with the
//                  preparation of a half-step: its bf16 operand tiles and the partial sums
//                  of its eq. 7 / 14 denominators.
// Every element is independent except for the fixed-order reductions, so all loads of a
// thread are issued before their results are used, and transposed layouts go through
// shared-memory tiles so that global accesses stay coalesced.
#pragma once

#include <cuda_bf16.h>

#include "simt_kernels.cuh"

namespace dna {
namespace glue {

using bf16 = __nv_bfloat16;
constexpr int TO = 32;   // o (or s) per tile
constexpr int TY = 32;   // r groups per CTA (threadIdx.y): 1024 threads
constexpr int UNR = 8;   // r values per thread whose loads are issued together
static_assert(TY == TO, "k_cand_fused gives each r group one column of the tile");

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
// the two bf16 halves of a pack2 word as float32
__device__ __forceinline__ float lo_half(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float hi_half(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
// bf16(x) and bf16(x - bf16(x))
__device__ __forceinline__ void split1(float x, bf16& h, bf16& l) {
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(x - __bfloat162float(h));
}

// Dynamic shared memory of k_cand_fused: red [TY][TO]; cs, ics [R]; sc; xs, ms [R][TO + 1].
template <typename Tp>
constexpr size_t cand_smem(int64_t R, bool bf) {
    return sizeof(Tp) * (2 * (size_t)R + (bf ? 2 : 1) * (size_t)R * (TO + 1) + TO + TY * TO);
}

// CTA = 32 columns o (threadIdx.x) x 32 groups of r (threadIdx.y); grid covers O (or O_pad
// when bf16 copies are written: the padding rows are written as zeros).
template <typename Tp, bool BF>
__global__ void __launch_bounds__(1024) k_cand_fused(View v, const double* __restrict__ c,
                                                    const Tp* __restrict__ Apart,
                                                    const Tp* __restrict__ Bpart, int splits,
                                                    Tp* __restrict__ Xmu, Tp* __restrict__ Xdna,
                                                    Tp eps, Tp alpha, bf16* __restrict__ Xmk,
                                                    bf16* __restrict__ Xdk, int64_t rp,
                                                    int64_t plane) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t R = v.R, O = v.O;
    Tp* red = reinterpret_cast<Tp*>(smem_raw);                    // [TY][TO]
    Tp* cs = red + TY * TO;                                       // [R]
    Tp* ics = cs + R;                                             // [R]
    Tp* scl = ics + R;                                            // [TO]
    Tp* xs = scl + TO;                                            // [R][TO + 1]: x, then x_dna
    Tp* ms = xs + R * (TO + 1);                                   // [R][TO + 1]: x_mu (BF)
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int64_t o0 = (int64_t)blockIdx.x * TO, o = o0 + tx;
    const bool live = o < O;
    const Tp* __restrict__ X = static_cast<const Tp*>(v.X);

    for (int64_t r = tid; r < R; r += TY * 32) {
        cs[r] = (Tp)c[r];
        ics[r] = Tp(1) / (Tp)c[r];
    }
    if (v.xo == 1) {   // rows of X contiguous along o
#pragma unroll 8
        for (int64_t r = ty; r < R; r += TY) xs[r * (TO + 1) + tx] = live ? X[r * v.xr + o] : Tp(0);
    } else {           // columns of X contiguous along r: lanes walk r
        const int i = ty;   // TY == TO: one column per r group
        const int64_t oi = o0 + i;
#pragma unroll 8
        for (int64_t r = tx; r < R; r += 32)
            xs[r * (TO + 1) + i] = oi < O ? X[r * v.xr + oi * v.xo] : Tp(0);
    }
    __syncthreads();

    Tp den = Tp(0);
    for (int64_t r0 = ty; r0 < R; r0 += TY * UNR) {
        Tp ra[UNR], rb[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) { ra[u] = Tp(0); rb[u] = Tp(0); }
        if (live) {
#pragma unroll 4
            for (int sp = 0; sp < splits; ++sp) {
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    const int64_t r = r0 + TY * u;
                    if (r < R) {
                        ra[u] += Apart[((int64_t)sp * R + r) * O + o];
                        rb[u] += Bpart[((int64_t)sp * R + r) * O + o];
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int64_t r = r0 + TY * u;
            if (r >= R) break;
            const Tp x = xs[r * (TO + 1) + tx];
            const Tp a = ra[u] * ics[r] - Tp(1);   // eq. 7
            const Tp b = rb[u] * ics[r];           // eq. 14
            // eq. 11 as x (W^t q)_r / c_r: no cancellation where 1 + a is small
            const Tp xmu = x * (ra[u] * ics[r]);
            Tp xd;
            if (a < Tp(0)) {                       // eq. 15, gain floored at eps
                const Tp xb = x * b;
                const Tp g = simt::dev_div(xb, xb - a);
                xd = x * (g > eps ? g : eps);
            } else {                               // eq. 17, step capped at alpha x
                const Tp stp = b > Tp(0) ? simt::dev_div(a, b) : Tp(0);
                const Tp cap = alpha * x;
                xd = x + (stp < cap ? stp : cap);
            }
            if (!live) xd = Tp(0);
            if (live) Xmu[r * O + o] = xmu;
            xs[r * (TO + 1) + tx] = xd;
            if constexpr (BF) ms[r * (TO + 1) + tx] = live ? xmu : Tp(0);
            den += cs[r] * xd;
        }
    }
    red[ty * TO + tx] = den;
    __syncthreads();
    {   // warp ty sums column ty's TY partials with a fixed butterfly (in the element
        // type: float64 arithmetic is slow on this GPU)
        const int col = ty;
        Tp tot = red[tx * TO + col];
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, m);
        const int64_t oc = o0 + col;
        if (tx == 0)
            scl[col] = oc < O ? (tot > Tp(0) ? (Tp)v.vsum[oc] / tot : Tp(1)) : Tp(0);   // eq. 10
    }
    __syncthreads();
    const Tp sc = scl[tx];
#pragma unroll 4
    for (int64_t r = ty; r < R; r += TY) {
        const Tp xd = xs[r * (TO + 1) + tx] * sc;
        if (live) Xdna[r * O + o] = xd;
        if constexpr (BF) xs[r * (TO + 1) + tx] = xd;
    }
    if constexpr (BF) {
        __syncthreads();
        // K-major bf16 rows [o][rp]: lanes walk pairs of r
        {
            const int i = ty;
            const int64_t oi = o0 + i;
            for (int64_t r = 2 * tx; r < rp; r += 64) {
                float m0 = 0.f, m1 = 0.f, d0 = 0.f, d1 = 0.f;
                if (r < R) { m0 = (float)ms[r * (TO + 1) + i]; d0 = (float)xs[r * (TO + 1) + i]; }
                if (r + 1 < R) {
                    m1 = (float)ms[(r + 1) * (TO + 1) + i];
                    d1 = (float)xs[(r + 1) * (TO + 1) + i];
                }
                const uint32_t mh = pack2(m0, m1), dh = pack2(d0, d1);
                *reinterpret_cast<uint32_t*>(Xmk + oi * rp + r) = mh;
                *reinterpret_cast<uint32_t*>(Xdk + oi * rp + r) = dh;
                if (plane) {   // lo planes: x - bf16(x)
                    *reinterpret_cast<uint32_t*>(Xmk + plane + oi * rp + r) =
                        pack2(m0 - lo_half(mh), m1 - hi_half(mh));
                    *reinterpret_cast<uint32_t*>(Xdk + plane + oi * rp + r) =
                        pack2(d0 - lo_half(dh), d1 - hi_half(dh));
                }
            }
        }
    }
}

// The candidates kernel for R <= 16 RS (the usual case): CTA = 32 columns o (threadIdx.x)
// x ceil(R / RS) <= 16 groups of RS consecutive r (threadIdx.y), every thread keeping its RS
// candidates in registers, so the eq. 10 renormalisation needs one shared-memory
// reduction and no second pass over r.  The split partials of pass 1 are summed in
// ascending split order while they stream in (no separate pass over them).  With BF the grid covers O_pad and the bf16 operand rows
// [o][rp] are written with zeros in the padding; at RS = 8 they go through shared memory,
// so that the CTA's rows (32 rp contiguous values per plane) are stored 512 bytes per warp
// instruction.  The 32 columns of block bx.
template <typename Tp, bool BF, int RS>
__device__ __forceinline__ void cand_reg_tile(const View& v, const double* __restrict__ c,
                                              const Tp* __restrict__ Apart,
                                              const Tp* __restrict__ Bpart, int splits,
                                              Tp* __restrict__ Xmu, Tp* __restrict__ Xdna,
                                              Tp eps, Tp alpha, bf16* __restrict__ Xmk,
                                              bf16* __restrict__ Xdk, int64_t rp, int64_t plane,
                                              int64_t bx) {
    static_assert(RS % 8 == 0, "operand rows are written 8 values at a time");
    constexpr bool STAGE = BF && RS == 8;
    __shared__ Tp red[16][33];
    __shared__ Tp scl[32];
    // staged bf16 rows: [plane: mu hi, dna hi, mu lo, dna lo][r group][o] (16 bytes each)
    __shared__ uint4 stg[STAGE ? 4 : 1][STAGE ? 16 : 1][STAGE ? 33 : 1];
    const int64_t R = v.R, O = v.O;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t o = bx * 32 + tx;
    const bool live = o < O;
    const int64_t r0 = (int64_t)ty * RS;
    const int nr = live && r0 < R ? (int)(R - r0 < RS ? R - r0 : RS) : 0;
    const Tp* __restrict__ X = static_cast<const Tp*>(v.X);

    Tp ra[RS], rb[RS], x[RS];
#pragma unroll
    for (int i = 0; i < RS; ++i) { ra[i] = Tp(0); rb[i] = Tp(0); x[i] = Tp(0); }
    if (nr > 0) {
        {
            const Tp* xp = X + r0 * v.xr + o * v.xo;
#pragma unroll
            for (int i = 0; i < RS; ++i) {
                if (i < nr) x[i] = *xp;
                xp += v.xr;
            }
        }
        const Tp* ap = Apart + r0 * O + o;
        const Tp* bp = Bpart + r0 * O + o;
        const int64_t ss = R * O;
#pragma unroll 1
        for (int sp = 0; sp < splits; ++sp) {
            Tp a0[RS], b0[RS];
#pragma unroll
            for (int i = 0; i < RS; ++i) {
                a0[i] = i < nr ? ap[i * O] : Tp(0);
                b0[i] = i < nr ? bp[i * O] : Tp(0);
            }
#pragma unroll
            for (int i = 0; i < RS; ++i) {
                ra[i] += a0[i];
                rb[i] += b0[i];
            }
            ap += ss;
            bp += ss;
        }
    }
    Tp den = Tp(0), xd[RS], xm[RS];
#pragma unroll
    for (int i = 0; i < RS; ++i) {
        const int64_t r = r0 + i;
        xd[i] = Tp(0);
        xm[i] = Tp(0);
        if (i >= nr) continue;
        const Tp cr = (Tp)c[r], ic = Tp(1) / cr;
        const Tp a = ra[i] * ic - Tp(1);   // eq. 7
        const Tp b = rb[i] * ic;           // eq. 14
        const Tp xr = x[i];
        xm[i] = xr * (ra[i] * ic);         // eq. 11 as x (W^t q)_r / c_r (no cancellation)
        if (a < Tp(0)) {                   // eq. 15, gain floored at eps
            const Tp xb = xr * b;
            const Tp g = simt::dev_div(xb, xb - a);
            xd[i] = xr * (g > eps ? g : eps);
        } else {                           // eq. 17, step capped at alpha x
            const Tp stp = b > Tp(0) ? simt::dev_div(a, b) : Tp(0);
            const Tp cap = alpha * xr;
            xd[i] = xr + (stp < cap ? stp : cap);
        }
        Xmu[r * O + o] = xm[i];
        den += cr * xd[i];
    }
    red[ty][tx] = den;
    __syncthreads();
    if (ty == 0) {   // eq. 10 per column: the r groups' partials in ascending order
        Tp tot = red[0][tx];
        for (int g = 1; g < (int)blockDim.y; ++g) tot += red[g][tx];
        scl[tx] = live ? (tot > Tp(0) ? (Tp)v.vsum[o] / tot : Tp(1)) : Tp(0);
    }
    __syncthreads();
    const Tp sc = scl[tx];
#pragma unroll
    for (int i = 0; i < RS; ++i) {
        xd[i] *= sc;
        if (i < nr) Xdna[(r0 + i) * O + o] = xd[i];
    }
    if constexpr (BF) {   // K-major bf16 rows [o][rp], o < O_pad, r < rp (zeros beyond)
        if (r0 < rp) {
#pragma unroll
            for (int q = 0; q < RS; q += 8) {
                uint32_t mh[4], dh[4], ml[4], dl[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float m0 = (float)xm[q + 2 * k], m1 = (float)xm[q + 2 * k + 1];
                    const float d0 = (float)xd[q + 2 * k], d1 = (float)xd[q + 2 * k + 1];
                    mh[k] = pack2(m0, m1);
                    dh[k] = pack2(d0, d1);
                    ml[k] = pack2(m0 - lo_half(mh[k]), m1 - hi_half(mh[k]));   // x - bf16(x)
                    dl[k] = pack2(d0 - lo_half(dh[k]), d1 - hi_half(dh[k]));
                }
                if constexpr (STAGE) {
                    stg[0][ty][tx] = make_uint4(mh[0], mh[1], mh[2], mh[3]);
                    stg[1][ty][tx] = make_uint4(dh[0], dh[1], dh[2], dh[3]);
                    stg[2][ty][tx] = make_uint4(ml[0], ml[1], ml[2], ml[3]);
                    stg[3][ty][tx] = make_uint4(dl[0], dl[1], dl[2], dl[3]);
                } else {
                    const int64_t off = o * rp + r0 + q;
                    *reinterpret_cast<uint4*>(Xmk + off) = make_uint4(mh[0], mh[1], mh[2], mh[3]);
                    *reinterpret_cast<uint4*>(Xdk + off) = make_uint4(dh[0], dh[1], dh[2], dh[3]);
                    if (plane) {
                        *reinterpret_cast<uint4*>(Xmk + plane + off) =
                            make_uint4(ml[0], ml[1], ml[2], ml[3]);
                        *reinterpret_cast<uint4*>(Xdk + plane + off) =
                            make_uint4(dl[0], dl[1], dl[2], dl[3]);
                    }
                }
            }
        }
        if constexpr (STAGE) {
            // the CTA's rows o = 32 bx .. 32 bx + 31 are one run of 32 rp bf16 values per
            // plane: chunk k (16 bytes) of the run is group k % (rp / 8) of row k / (rp / 8)
            __syncthreads();
            const int gpr = (int)(rp / 8), nch = 32 * gpr;
            const int tid = ty * 32 + tx, nt = 32 * (int)blockDim.y;
            uint4* M = reinterpret_cast<uint4*>(Xmk + bx * 32 * rp);
            uint4* D = reinterpret_cast<uint4*>(Xdk + bx * 32 * rp);
            for (int k = tid; k < nch; k += nt) {
                const int j = k / gpr, g = k % gpr;
                M[k] = stg[0][g][j];
                D[k] = stg[1][g][j];
                if (plane) {
                    reinterpret_cast<uint4*>(Xmk + plane + bx * 32 * rp)[k] = stg[2][g][j];
                    reinterpret_cast<uint4*>(Xdk + plane + bx * 32 * rp)[k] = stg[3][g][j];
                }
            }
        }
    }
}

template <typename Tp, bool BF, int RS>
__global__ void __launch_bounds__(512) k_cand_reg(View v, const double* __restrict__ c,
                                                  const Tp* __restrict__ Apart,
                                                  const Tp* __restrict__ Bpart, int splits,
                                                  Tp* __restrict__ Xmu, Tp* __restrict__ Xdna,
                                                  Tp eps, Tp alpha, bf16* __restrict__ Xmk,
                                                  bf16* __restrict__ Xdk, int64_t rp,
                                                  int64_t plane) {
    cand_reg_tile<Tp, BF, RS>(v, c, Apart, Bpart, splits, Xmu, Xdna, eps, alpha, Xmk, Xdk, rp,
                              plane, blockIdx.x);
}

// A[0][i] = A[0][i] + A[1][i] + ... + A[splits-1][i] (ascending, the order the candidates
// kernel uses, so results are unchanged), and the same for B (may be null): the split
// partials of pass 1 streamed once with wide loads before the candidates read them.
template <typename Tp>
__global__ void __launch_bounds__(256) k_split_sum(Tp* __restrict__ A, Tp* __restrict__ B,
                                                   int64_t n, int splits) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if constexpr (sizeof(Tp) == 4) {
        if (n % 4 == 0) {   // float4 path (slots are 16-byte aligned when n % 4 == 0)
            const int64_t n4 = n / 4;
            for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    float4* M = reinterpret_cast<float4*>(m ? B : A);
                    if (!M) continue;
                    float4 acc = M[i];
#pragma unroll 4
                    for (int sp = 1; sp < splits; ++sp) {
                        const float4 t = M[(int64_t)sp * n4 + i];
                        acc.x += t.x; acc.y += t.y; acc.z += t.z; acc.w += t.w;
                    }
                    M[i] = acc;
                }
            }
            return;
        }
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            Tp* M = m ? B : A;
            if (!M) continue;
            Tp acc = M[i];
#pragma unroll 4
            for (int sp = 1; sp < splits; ++sp) acc += M[(int64_t)sp * n + i];
            M[i] = acc;
        }
    }
}

template <typename Tp>
constexpr size_t select_smem(int64_t R) {
    return sizeof(Tp) * (size_t)R * (TO + 1) + 32 * sizeof(int);
}

// Selection: x(r, o) <- Newton candidate iff d_dna < d_mu (ties keep MU), the choice and
// the final costs per column, and fpart[blk][r] = sum over this CTA's 32 columns of the
// new x(r, o) (float64), the first level of the normalisation sums.  Each cost is the
// column's eq. 5 sub-problem cost less a constant: the pass-2 slots plus
// reg * sum_r x(r, o) of that candidate (reg = lambda for H, rho for W; eq. 5 and eq. 4).
//
// Descent selection (dcur given): the Newton candidate is compared with the starting column
// instead of the MU candidate: dpart holds the Newton costs only ([splits][O]), dcur the
// starting column's ([cur_splits][O]), and the penalty of the starting column is
// reg * sum_r x(r, o) of the current X.  dfin receives (d_start, d_dna).
template <typename Tp>
__global__ void __launch_bounds__(256) k_select_fused(View v, const Tp* __restrict__ Xmu,
                                                      const Tp* __restrict__ Xdna,
                                                      const double* __restrict__ dpart,
                                                      int splits, uint8_t* __restrict__ choice,
                                                      double* __restrict__ dfin,
                                                      double* __restrict__ fpart, double reg,
                                                      const double* __restrict__ dcur,
                                                      int cur_splits) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t R = v.R, O = v.O;
    Tp* xs = reinterpret_cast<Tp*>(smem_raw);                   // [R][TO + 1]
    int* nw = reinterpret_cast<int*>(xs + R * (TO + 1));        // [TO]
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int64_t o0 = (int64_t)blockIdx.x * TO, o = o0 + tx;
    const bool live = o < O;
    // the cost slots of column o: warp ty adds the contiguous range [ty k, (ty + 1) k)
    // (k = ceil(splits / 8)), warp 0 the eight range sums in order
    __shared__ double dsum[2][8][TO];
    const Tp* __restrict__ Xcur = static_cast<const Tp*>(v.X);
    if (dcur == nullptr) {
        const int per = (splits + 7) / 8, sp0 = ty * per, sp1 = min(splits, sp0 + per);
        double dm = 0.0, dd = 0.0;
        if (live)
#pragma unroll 8
            for (int sp = sp0; sp < sp1; ++sp) {   // loads of eight slots in flight
                dm += dpart[((int64_t)sp * 2 + 0) * O + o];
                dd += dpart[((int64_t)sp * 2 + 1) * O + o];
            }
        dsum[0][ty][tx] = dm;
        dsum[1][ty][tx] = dd;
    } else {
        const int per = (splits + 7) / 8, sp0 = ty * per, sp1 = min(splits, sp0 + per);
        const int pc = (cur_splits + 7) / 8, c0 = ty * pc, c1 = min(cur_splits, c0 + pc);
        double dm = 0.0, dd = 0.0;
        if (live) {
            for (int sp = c0; sp < c1; ++sp) dm += dcur[(int64_t)sp * O + o];
            for (int sp = sp0; sp < sp1; ++sp) dd += dpart[(int64_t)sp * O + o];
        }
        dsum[0][ty][tx] = dm;
        dsum[1][ty][tx] = dd;
    }
    // the eq. 5 penalty: warp ty sums r = ty, ty + 8, ... of both candidates (float64)
    __shared__ double psum[2][8][TO];
    if (reg != 0.0) {
        double pm = 0.0, pd = 0.0;
        if (live)
            for (int64_t r = ty; r < R; r += 8) {
                pm += dcur ? (double)Xcur[r * v.xr + o * v.xo] : (double)Xmu[r * O + o];
                pd += (double)Xdna[r * O + o];
            }
        psum[0][ty][tx] = pm;
        psum[1][ty][tx] = pd;
    }
    __syncthreads();
    if (ty == 0) {
        int newton = 0;
        if (live) {
            double dm = dsum[0][0][tx], dd = dsum[1][0][tx];
            for (int g = 1; g < 8; ++g) {
                dm += dsum[0][g][tx];
                dd += dsum[1][g][tx];
            }
            if (reg != 0.0) {
                double pm = psum[0][0][tx], pd = psum[1][0][tx];
                for (int g = 1; g < 8; ++g) {
                    pm += psum[0][g][tx];
                    pd += psum[1][g][tx];
                }
                dm += reg * pm;
                dd += reg * pd;
            }
            newton = dd < dm;
            choice[o] = (uint8_t)newton;
            dfin[o] = dm;
            dfin[O + o] = dd;
        }
        nw[tx] = newton;
    }
    __syncthreads();
    const Tp* __restrict__ src = nw[tx] ? Xdna : Xmu;
    Tp* __restrict__ X = static_cast<Tp*>(v.X);
    const bool direct = v.xo == 1;
#pragma unroll 16
    for (int64_t r = ty; r < R; r += 8) {
        const Tp x = live ? src[r * O + o] : Tp(0);
        xs[r * (TO + 1) + tx] = x;
        if (direct && live) X[r * v.xr + o] = x;
    }
    __syncthreads();
    if (!direct) {   // columns of X contiguous along r: lanes walk r
        for (int i = ty; i < TO; i += 8) {
            const int64_t oi = o0 + i;
            if (oi >= O) break;
#pragma unroll 4
            for (int64_t r = tx; r < R; r += 32) X[r * v.xr + oi * v.xo] = xs[r * (TO + 1) + i];
        }
    }
    for (int64_t r = tid; r < R; r += 256) {
        Tp s = Tp(0);
#pragma unroll 8
        for (int i = 0; i < TO; ++i) s += xs[r * (TO + 1) + i];
        fpart[(int64_t)blockIdx.x * R + r] = (double)s;
    }
}

// The multiplicative update (eq. 11) fused with the first level of the step 16 / 29 sums:
// x(r, o) <- x(r, o) * (sum over splits of Apart(r, o)) / c_r, written in place, and
// fpart[blk][r] = sum over this CTA's 32 columns of the new x(r, o) (float64).  The same
// CTA shape, grid and fpart layout as k_select_fused, so the normalisation that follows is
// shared with the DNA half-step.
template <typename Tp>
__global__ void __launch_bounds__(256) k_mu_fused(View v, const double* __restrict__ c,
                                                  const Tp* __restrict__ Apart, int splits,
                                                  double* __restrict__ fpart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t R = v.R, O = v.O;
    Tp* xs = reinterpret_cast<Tp*>(smem_raw);                   // [R][TO + 1]
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int64_t o0 = (int64_t)blockIdx.x * TO, o = o0 + tx;
    const bool live = o < O;
    Tp* __restrict__ X = static_cast<Tp*>(v.X);
    const bool direct = v.xo == 1;
    if (!direct) {   // columns of X contiguous along r: read the tile with lanes along r
        for (int i = ty; i < TO; i += 8) {
            const int64_t oi = o0 + i;
#pragma unroll 4
            for (int64_t r = tx; r < R; r += 32)
                xs[r * (TO + 1) + i] = oi < O ? X[r * v.xr + oi * v.xo] : Tp(0);
        }
        __syncthreads();
    }
#pragma unroll 4
    for (int64_t r = ty; r < R; r += 8) {
        Tp ra = Tp(0);
        if (live)
            for (int sp = 0; sp < splits; ++sp) ra += Apart[((int64_t)sp * R + r) * O + o];
        const Tp x = direct ? (live ? X[r * v.xr + o] : Tp(0)) : xs[r * (TO + 1) + tx];
        const Tp xm = live ? x * (ra / (Tp)c[r]) : Tp(0);   // eq. 11
        xs[r * (TO + 1) + tx] = xm;
        if (direct && live) X[r * v.xr + o] = xm;
    }
    __syncthreads();
    if (!direct) {
        for (int i = ty; i < TO; i += 8) {
            const int64_t oi = o0 + i;
            if (oi >= O) break;
#pragma unroll 4
            for (int64_t r = tx; r < R; r += 32) X[r * v.xr + oi * v.xo] = xs[r * (TO + 1) + i];
        }
    }
    for (int64_t r = tid; r < R; r += 256) {
        Tp s = Tp(0);
#pragma unroll 8
        for (int i = 0; i < TO; ++i) s += xs[r * (TO + 1) + i];
        fpart[(int64_t)blockIdx.x * R + r] = (double)s;
    }
}

// out[r] = in[r] + reg, an exact zero replaced by 1 (the factor sums of Algorithm 1 from
// sums that other ranks helped form).
template <int UNUSED = 0>
__global__ void k_add_reg(const double* __restrict__ in, int64_t R, double reg,
                          double* __restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) {
        const double s = in[r] + reg;
        out[r] = s == 0.0 ? 1.0 : s;
    }
}

// One tile job of k_scale_ops.
struct OpsArgs {
    // the target half-step's X (element (r, o) at X[r * xr + o * xo]) and Y ((s, r) at
    // Y[s * ys + r * yr])
    void* X;
    int64_t xr, xo, O;
    void* Y;
    int64_t ys, yr, S;
    int64_t R;
    const double* f;   // normaliser f_r, or null (no scaling, nothing written back)
    bool xmul;         // X *= f_r and Y /= f_r (else X /= f_r and Y *= f_r)
    // bf16 operands of the target half-step (tensor-core form), or null
    bf16* Xk;          // [O_pad][rp]
    bf16* Yk;          // [S_pad][rp]
    bf16* Ytk;         // [rp][S_pad]
    bf16* Y2tk;        // [rp][S_pad], or null
    int64_t rp, O_pad, S_pad;
    int64_t plane;     // > 0: also write lo planes (x - bf16(x)) `plane` elements after each
    double* cpart;     // [ceil(S / 32)][R] partial sums over s of the (scaled) y(s, r), or null
    int64_t xtiles_o, tiles_r, xtiles;   // X tiles: xtiles_o x tiles_r; then the Y tiles
};

// Tiles of 32 values of i (o of X, s of Y) x RT values of r: blocks [0, xtiles) cover X as
// (o-tile, r-tile), the rest cover Y as (s-tile, r-tile).  Every thread issues its RT / 8
// loads before any store.  Extents are the padded ones when bf16 operands are written, so
// the padding of the operand buffers is rewritten as zeros.
template <typename Tp, int RT>
__global__ void __launch_bounds__(256, 4) k_scale_ops(OpsArgs a) {
    constexpr int NL = RT / 8;                 // elements per thread
    __shared__ Tp tile[RT][TO + 1];            // [r][i]
    __shared__ Tp fr[RT];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const bool isx = (int64_t)blockIdx.x < a.xtiles;
    const int64_t b = isx ? (int64_t)blockIdx.x : (int64_t)blockIdx.x - a.xtiles;
    const int64_t it = b / a.tiles_r, rt = b % a.tiles_r;
    const int64_t r0 = rt * RT, i0 = it * TO;   // i = o (X tiles) or s (Y tiles)
    const int64_t n = isx ? a.O : a.S;
    for (int k = tid; k < RT; k += 256) {
        const int64_t r = r0 + k;
        Tp s = Tp(1);
        if (a.f && r < a.R) {
            const Tp f = (Tp)a.f[r];
            s = (isx == a.xmul) ? f : Tp(1) / f;
        }
        fr[k] = s;
    }
    __syncthreads();
    Tp* M = static_cast<Tp*>(isx ? a.X : a.Y);
    // element (r, i): X[r * xr + i * xo] or Y[i * ys + r * yr]
    const int64_t sr = isx ? a.xr : a.yr, si = isx ? a.xo : a.ys;
    Tp x[NL];
    if (si == 1) {   // contiguous along i: lanes walk i, thread rows walk r
        const int64_t i = i0 + tx;
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int64_t r = r0 + ty + 8 * k;
            x[k] = (r < a.R && i < n) ? M[r * sr + i] : Tp(0);
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int rl = ty + 8 * k;
            const int64_t r = r0 + rl, i = i0 + tx;
            x[k] *= fr[rl];
            if (a.f && r < a.R && i < n) M[r * sr + i] = x[k];
            tile[rl][tx] = x[k];
        }
    } else {         // contiguous along r: lanes walk 32 values of r, thread rows walk i
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int il = ty + 8 * (k % 4), rl = tx + 32 * (k / 4);
            const int64_t i = i0 + il, r = r0 + rl;
            x[k] = (r < a.R && i < n) ? M[i * si + r * sr] : Tp(0);
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int il = ty + 8 * (k % 4), rl = tx + 32 * (k / 4);
            const int64_t i = i0 + il, r = r0 + rl;
            x[k] *= fr[rl];
            if (a.f && r < a.R && i < n) M[i * si + r * sr] = x[k];
            tile[rl][il] = x[k];
        }
    }
    __syncthreads();
    if (!isx && a.cpart && i0 < a.S)
        for (int k = tid; k < RT; k += 256)
            if (r0 + k < a.R) {
                Tp s = Tp(0);
#pragma unroll 8
                for (int j = 0; j < TO; ++j) s += tile[k][j];
                a.cpart[it * a.R + r0 + k] = (double)s;
            }
    if (a.Xk == nullptr) return;
    if constexpr (sizeof(Tp) == 4) {
        // rows [i][rp] with r contiguous (Xk of X tiles, Yk of Y tiles): pairs of r, a warp
        // storing one row's RT values of r (or two rows' when RT = 32)
        bf16* RM = isx ? a.Xk : a.Yk;
        const int64_t ipad = isx ? a.O_pad : a.S_pad;
        for (int p = tid; p < TO * RT / 2; p += 256) {
            const int il = p / (RT / 2), rl = 2 * (p % (RT / 2));
            const int64_t i = i0 + il, r = r0 + rl;
            if (i < ipad && r < a.rp) {   // rp is even, so r + 1 < rp too
                const float y0 = tile[rl][il], y1 = tile[rl + 1][il];
                const uint32_t h = pack2(y0, y1);
                *reinterpret_cast<uint32_t*>(RM + i * a.rp + r) = h;
                if (a.plane)
                    *reinterpret_cast<uint32_t*>(RM + a.plane + i * a.rp + r) =
                        pack2(y0 - lo_half(h), y1 - hi_half(h));
            }
        }
        if (isx) return;
        // Ytk, Y2tk [r][S_pad] with s contiguous: pairs of s (S_pad is a multiple of 64)
        for (int p = tid; p < RT * TO / 2; p += 256) {
            const int rl = p / (TO / 2), il = 2 * (p % (TO / 2));
            const int64_t r = r0 + rl, i = i0 + il;
            if (r < a.rp && i < a.S_pad) {
                const float y0 = tile[rl][il], y1 = tile[rl][il + 1];
                const int64_t at = r * a.S_pad + i;
                const uint32_t h = pack2(y0, y1);
                *reinterpret_cast<uint32_t*>(a.Ytk + at) = h;
                if (a.plane)
                    *reinterpret_cast<uint32_t*>(a.Ytk + a.plane + at) =
                        pack2(y0 - lo_half(h), y1 - hi_half(h));
                if (a.Y2tk) {
                    const float q0 = y0 * y0, q1 = y1 * y1;
                    const uint32_t h2 = pack2(q0, q1);
                    *reinterpret_cast<uint32_t*>(a.Y2tk + at) = h2;
                    if (a.plane)
                        *reinterpret_cast<uint32_t*>(a.Y2tk + a.plane + at) =
                            pack2(q0 - lo_half(h2), q1 - hi_half(h2));
                }
            }
        }
    }
}

}  // namespace glue
}  // namespace dna
