// CUDA-core (SIMT) kernels of the DNA half-step, templated on the element type.
//
// One half-step, in the (s, o, r) terms of dna::View, Algorithm 1 steps 2-15:
//   z(s,o) = sum_r y(s,r) x(r,o)                                   (step 2 / 7 / 12)
//   q = v / z, qbar = v / z^2 (0 where v = 0)                      (step 3, 10)
//   A(r,o) = sum_s y(s,r) q(s,o),  B(r,o) = sum_s y(s,r)^2 qbar(s,o)   (steps 5, 10)
//   candidates per (r, o) (steps 6, 11), per-column costs (steps 9, 14), selection
//   (step 15).
// Pass 1 never writes Z or Q to memory: each CTA owns a block of o and streams s in
// chunks, computing the z tile in registers, q and qbar into shared memory, and
// accumulating A and B for its r-block in registers (the structure of a fused
// back-to-back GEMM).  Pass 2 recomputes z for both candidates the same way and reduces
// the cost terms per column.  The reduction over s may be split across CTAs (grid z);
// partial sums are combined later in a fixed order, so results are deterministic.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dna_internal.h"

namespace dna {
namespace simt {

constexpr int NT = 256;   // threads per CTA in passes 1 and 2
constexpr int OB = 64;    // o-block
constexpr int SB = 64;    // s-chunk
constexpr int LD = 68;    // padded leading dimension of the [*][64] shared tiles

__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    double2 a = *reinterpret_cast<const double2*>(p);
    double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ float dev_log(float x) { return logf(x); }
__device__ __forceinline__ double dev_log(double x) { return log(x); }
// a / b: the fast-division intrinsic in float32 (a few ulp), exact division in float64
__device__ __forceinline__ float dev_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double dev_div(double a, double b) { return a / b; }

// Load a ROWS x COLS tile into shared memory (leading dimension LD):
//   sm[i][j] = g[(i0 + i) * si + (j0 + j) * sj] when i0 + i < ni and j0 + j < nj, else 0.
// Consecutive threads walk the unit-stride global dimension so that reads coalesce.
template <typename Tp, int ROWS, int COLS>
__device__ __forceinline__ void load_tile(Tp* __restrict__ sm, const Tp* __restrict__ g,
                                          int64_t si, int64_t sj, int64_t i0, int64_t j0,
                                          int64_t ni, int64_t nj) {
    if (sj == 1) {
        for (int e = threadIdx.x; e < ROWS * COLS; e += NT) {
            const int i = e / COLS, j = e % COLS;
            const int64_t gi = i0 + i, gj = j0 + j;
            sm[i * LD + j] = (gi < ni && gj < nj) ? __ldg(g + gi * si + gj) : Tp(0);
        }
    } else {
        for (int e = threadIdx.x; e < ROWS * COLS; e += NT) {
            const int j = e / ROWS, i = e % ROWS;
            const int64_t gi = i0 + i, gj = j0 + j;
            sm[i * LD + j] = (gi < ni && gj < nj) ? __ldg(g + gi * si + gj * sj) : Tp(0);
        }
    }
}

// Accumulate the 4 x 4 register tile z[s][o] += sum_{r < RB} Yt[r][zs + s] * Xs[r][zo + o].
template <typename Tp, int RB>
__device__ __forceinline__ void z_tile(const Tp* __restrict__ Yt, const Tp* __restrict__ Xs,
                                       int zs, int zo, Tp (&z)[4][4]) {
#pragma unroll 4
    for (int r = 0; r < RB; ++r) {
        Tp xa[4], ya[4];
        ld4(Xs + r * LD + zo, xa);
        ld4(Yt + r * LD + zs, ya);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) z[i][j] = fma(ya[i], xa[j], z[i][j]);
    }
}

template <typename Tp, int RB>
struct Pass1Cfg {
    static constexpr int RPT = RB / 16;  // r rows per thread in the A/B accumulators
    static constexpr size_t smem = (size_t)(2 * RB * LD + 2 * SB * LD) * sizeof(Tp);
};

// Pass 1: raw A and B sums for one (o-block, r-block, s-split).
// grid = (ceil(O / OB), ceil(R / RB), splits); Apart/Bpart are [splits][R][O].
// dcur (may be null): the r-block-0 tiles also write the starting factor's per-column cost
// d'(o) = sum_{v>0} (-v log z) + sum z over their split of s into dcur[split][O] (float64;
// the terms summed in the element type within a chunk), for descent selection.
template <typename Tp, int RB, bool WITH_B>
__device__ __forceinline__ void pass1_tile(const View& v, Tp* __restrict__ Apart,
                                           Tp* __restrict__ Bpart, int64_t s_per,
                                           int* __restrict__ status, int64_t tile_o, int64_t tile_r,
                                           int64_t tile_s, unsigned char* smem_raw,
                                           double* __restrict__ dcur = nullptr) {
    using C = Pass1Cfg<Tp, RB>;
    Tp* Xs = reinterpret_cast<Tp*>(smem_raw);  // [RB][LD]  x(r, o) of the current r-piece
    Tp* Yt = Xs + RB * LD;                     // [RB][LD]  y(s, r) transposed: Yt[r][s]
    Tp* Qs = Yt + RB * LD;                     // [SB][LD]  q(s, o)
    Tp* Qb = Qs + SB * LD;                     // [SB][LD]  qbar(s, o)

    const Tp* __restrict__ V = static_cast<const Tp*>(v.V);
    const Tp* __restrict__ X = static_cast<const Tp*>(v.X);
    const Tp* __restrict__ Y = static_cast<const Tp*>(v.Y);
    const int tid = threadIdx.x;
    const int64_t o0 = tile_o * OB;
    const int64_t rown0 = tile_r * RB;
    const int64_t s_begin = tile_s * s_per;
    const int64_t s_end = min(v.S, s_begin + s_per);
    const int npieces = (int)((v.R + RB - 1) / RB);

    const int zo = (tid % 16) * 4, zs = (tid / 16) * 4;  // z tile of this thread
    const int go = (tid % 16) * 4, gr = tid / 16;        // A/B rows gr + 16 i

    Tp accA[C::RPT][4], accB[C::RPT][4];
#pragma unroll
    for (int i = 0; i < C::RPT; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { accA[i][j] = Tp(0); accB[i][j] = Tp(0); }

    if (npieces == 1) load_tile<Tp, RB, OB>(Xs, X, v.xr, v.xo, 0, o0, v.R, v.O);
    int bad = 0;
    const bool want_cur = dcur != nullptr && tile_r == 0;
    double dsum[4] = {0.0, 0.0, 0.0, 0.0};   // this thread's columns zo .. zo + 3

    for (int64_t s0 = s_begin; s0 < s_end; s0 += SB) {
        Tp z[4][4], vpre[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                z[i][j] = Tp(0);
                // issue this chunk's V loads now; they complete behind the z-tile FMAs
                const int64_t s = s0 + zs + i, o = o0 + zo + j;
                vpre[i][j] = (s < s_end && o < v.O) ? __ldg(V + s * v.vs + o) : Tp(0);
            }
        for (int p = 0; p < npieces; ++p) {
            if (npieces > 1) load_tile<Tp, RB, OB>(Xs, X, v.xr, v.xo, (int64_t)p * RB, o0, v.R, v.O);
            load_tile<Tp, RB, SB>(Yt, Y, v.yr, v.ys, (int64_t)p * RB, s0, v.R, v.S);
            __syncthreads();
            z_tile<Tp, RB>(Yt, Xs, zs, zo, z);
            __syncthreads();
        }
        if (want_cur) {   // the starting column's cost terms (steps 9 / 14 at the current x)
            Tp t[4] = {Tp(0), Tp(0), Tp(0), Tp(0)};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const Tp vv = vpre[i][j], zz = z[i][j];
                    if (s0 + zs + i < s_end)
                        t[j] += vv > Tp(0) ? zz - vv * dev_log(zz) : zz;
                }
#pragma unroll
            for (int j = 0; j < 4; ++j) dsum[j] += (double)t[j];
        }
        // q = v / z and qbar = v / z^2, zero where v = 0 (note after Algorithm 1): one
        // reciprocal per element, branch-free, rows stored as vectors (no bank conflicts)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            Tp q[4], qb[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const Tp vv = vpre[i][j], zz = z[i][j];
                const bool pos = vv > Tp(0);
                bad |= (pos && !(zz > Tp(0))) ? 1 : 0;
                const Tp rz = dev_div(Tp(1), zz);
                q[j] = pos ? vv * rz : Tp(0);
                qb[j] = pos ? q[j] * rz : Tp(0);
            }
            st4(Qs + (zs + i) * LD + zo, q);
            st4(Qb + (zs + i) * LD + zo, qb);
        }
        if (npieces > 1)
            load_tile<Tp, RB, SB>(Yt, Y, v.yr, v.ys, rown0, s0, v.R, v.S);
        __syncthreads();
        // A += Y^t Q and B += (Y o Y)^t Qbar over this chunk
#pragma unroll 2
        for (int s = 0; s < SB; ++s) {
            Tp qv[4], qbv[4];
            ld4(Qs + s * LD + go, qv);
            if (WITH_B) ld4(Qb + s * LD + go, qbv);
#pragma unroll
            for (int i = 0; i < C::RPT; ++i) {
                const Tp y = Yt[(gr + 16 * i) * LD + s];
#pragma unroll
                for (int j = 0; j < 4; ++j) accA[i][j] = fma(y, qv[j], accA[i][j]);
                if (WITH_B) {
                    const Tp y2 = y * y;
#pragma unroll
                    for (int j = 0; j < 4; ++j) accB[i][j] = fma(y2, qbv[j], accB[i][j]);
                }
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(status, STATUS_NONFINITE);
    if (want_cur) {   // the 16 threads of each column group, added in a fixed order
        double* red = reinterpret_cast<double*>(smem_raw);   // [16][OB], over Xs / Yt
#pragma unroll
        for (int j = 0; j < 4; ++j) red[(tid / 16) * OB + zo + j] = dsum[j];
        __syncthreads();
        if (tid < OB) {
            double d = 0.0;
            for (int g = 0; g < 16; ++g) d += red[g * OB + tid];
            const int64_t o = o0 + tid;
            if (o < v.O) {
                dcur[tile_s * v.O + o] = d;
                if (!isfinite(d)) atomicOr(status, STATUS_NONFINITE);
            }
        }
    }

    const int64_t base = tile_s * v.R;
#pragma unroll
    for (int i = 0; i < C::RPT; ++i) {
        const int64_t r = rown0 + gr + 16 * i;
        if (r >= v.R) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t o = o0 + go + j;
            if (o < v.O) {
                Apart[(base + r) * v.O + o] = accA[i][j];
                if (WITH_B) Bpart[(base + r) * v.O + o] = accB[i][j];
            }
        }
    }
}

// Pass 1 for one problem: grid = (ceil(O / OB), ceil(R / RB), splits).
template <typename Tp, int RB, bool WITH_B>
__global__ void __launch_bounds__(NT, sizeof(Tp) == 4 ? 2 : 1)
    k_pass1(View v, Tp* __restrict__ Apart, Tp* __restrict__ Bpart, int64_t s_per,
            int* __restrict__ status, double* __restrict__ dcur) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pass1_tile<Tp, RB, WITH_B>(v, Apart, Bpart, s_per, status, blockIdx.x, blockIdx.y, blockIdx.z,
                               smem_raw, dcur);
}

template <typename Tp, int RB, int NC>
struct Pass2Cfg {
    static constexpr size_t tiles = (size_t)((NC + 1) * RB * LD) * sizeof(Tp);
    static constexpr size_t red = (size_t)16 * NC * OB * sizeof(double);
    static constexpr size_t smem = tiles > red ? tiles : red;
};

// Pass 2: per-column cost partials for NC candidates (Algorithm 1 steps 7-9, 12-14).
// FULL = false: d'(o) = sum_{v>0} (-v log z) + sum z (the candidate comparison).
// FULL = true:  sum_{v>0} v log(v / z) - sum v + sum z (eq. 1, for dna_kl).
// X_c(r, o) at Xc[r * xr + o * xo].  dpart is [splits][NC][O] float64.
template <typename Tp, int RB, int NC, bool FULL>
__device__ __forceinline__ void pass2_tile(const View& v, const Tp* __restrict__ X0,
                                           const Tp* __restrict__ X1, int64_t xr, int64_t xo,
                                           double* __restrict__ dpart, int64_t s_per,
                                           int* __restrict__ status, int64_t tile_o,
                                           int64_t tile_s, unsigned char* smem_raw) {
    Tp* Yt = reinterpret_cast<Tp*>(smem_raw);  // [RB][LD]
    Tp* Xs = Yt + RB * LD;                     // [NC][RB][LD]
    const Tp* __restrict__ V = static_cast<const Tp*>(v.V);
    const Tp* __restrict__ Y = static_cast<const Tp*>(v.Y);
    const int tid = threadIdx.x;
    const int64_t o0 = tile_o * OB;
    const int64_t s_begin = tile_s * s_per;
    const int64_t s_end = min(v.S, s_begin + s_per);
    const int npieces = (int)((v.R + RB - 1) / RB);
    const int zo = (tid % 16) * 4, zs = (tid / 16) * 4;

    double dacc[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) dacc[c][j] = 0.0;

    if (npieces == 1) {
        load_tile<Tp, RB, OB>(Xs, X0, xr, xo, 0, o0, v.R, v.O);
        if (NC > 1) load_tile<Tp, RB, OB>(Xs + RB * LD, X1, xr, xo, 0, o0, v.R, v.O);
    }
    int bad = 0;
    for (int64_t s0 = s_begin; s0 < s_end; s0 += SB) {
        Tp z[NC][4][4], vpre[4][4];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) z[c][i][j] = Tp(0);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t s = s0 + zs + i, o = o0 + zo + j;
                vpre[i][j] = (s < s_end && o < v.O) ? __ldg(V + s * v.vs + o) : Tp(0);
            }
        for (int p = 0; p < npieces; ++p) {
            if (npieces > 1) {
                load_tile<Tp, RB, OB>(Xs, X0, xr, xo, (int64_t)p * RB, o0, v.R, v.O);
                if (NC > 1)
                    load_tile<Tp, RB, OB>(Xs + RB * LD, X1, xr, xo, (int64_t)p * RB, o0, v.R, v.O);
            }
            load_tile<Tp, RB, SB>(Yt, Y, v.yr, v.ys, (int64_t)p * RB, s0, v.R, v.S);
            __syncthreads();
#pragma unroll
            for (int c = 0; c < NC; ++c) z_tile<Tp, RB>(Yt, Xs + c * RB * LD, zs, zo, z[c]);
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            Tp run[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) run[c] = Tp(0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const Tp vv = vpre[i][j];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const Tp zz = z[c][i][j];
                    const bool pos = vv > Tp(0);
                    bad |= (pos && !(zz > Tp(0))) ? 1 : 0;
                    // branch-free: the v = 0 terms (possibly log of a non-positive z) are
                    // discarded by the select
                    const Tp t = FULL ? (vv * dev_log(vv / zz) - vv) : (-vv * dev_log(zz));
                    run[c] += pos ? zz + t : zz;
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) dacc[c][j] += (double)run[c];
        }
    }
    if (bad) atomicOr(status, STATUS_NONFINITE);

    // reduce the 16 threads that share each o (they differ in zs)
    __syncthreads();
    double* red = reinterpret_cast<double*>(smem_raw);  // [16][NC][OB]
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) red[((tid / 16) * NC + c) * OB + zo + j] = dacc[c][j];
    __syncthreads();
    if (tid < NC * OB) {
        const int c = tid / OB, oo = tid % OB;
        double sum = 0.0;
        for (int k = 0; k < 16; ++k) sum += red[(k * NC + c) * OB + oo];
        const int64_t o = o0 + oo;
        if (o < v.O) dpart[(tile_s * NC + c) * v.O + o] = sum;
    }
}

// Pass 2 for one problem: grid = (ceil(O / OB), splits).
template <typename Tp, int RB, int NC, bool FULL>
__global__ void __launch_bounds__(NT, sizeof(Tp) == 4 ? 2 : 1)
    k_pass2(View v, const Tp* __restrict__ X0, const Tp* __restrict__ X1, int64_t xr, int64_t xo,
            double* __restrict__ dpart, int64_t s_per, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pass2_tile<Tp, RB, NC, FULL>(v, X0, X1, xr, xo, dpart, s_per, status, blockIdx.x, blockIdx.y,
                                 smem_raw);
}

// Candidates (steps 6 and 11, eq. 10, 11, 15, 17).  CTA = 32 columns o (threadIdx.x) x 8
// groups of r (threadIdx.y); the eq. 10 denominator of each column is reduced over the 8
// groups in shared memory in a fixed order.
template <typename Tp>
__device__ __forceinline__ void candidates_tile(const View& v, const double* __restrict__ c,
                                                const Tp* __restrict__ Apart,
                                                const Tp* __restrict__ Bpart, int splits,
                                                Tp* __restrict__ Xmu, Tp* __restrict__ Xdna,
                                                Tp eps, Tp alpha, int64_t tile_o) {
    __shared__ double red[8][32];
    __shared__ Tp cs[512], ics[512];   // c_r and 1 / c_r in the element type (R <= 512)
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty * 32 + tx; r < v.R; r += 256) {
        cs[r] = (Tp)c[r];
        ics[r] = Tp(1) / (Tp)c[r];
    }
    __syncthreads();
    const int64_t o = tile_o * 32 + tx;
    const bool live = o < v.O;
    const Tp* __restrict__ X = static_cast<const Tp*>(v.X);
    Tp den = Tp(0);   // this thread's R / 8 terms of the eq. 10 denominator
    if (live) {
        for (int64_t r = ty; r < v.R; r += 8) {
            Tp ra = Tp(0), rb = Tp(0);
            for (int sp = 0; sp < splits; ++sp) {
                ra += Apart[((int64_t)sp * v.R + r) * v.O + o];
                rb += Bpart[((int64_t)sp * v.R + r) * v.O + o];
            }
            const Tp ic = ics[r];
            const Tp a = ra * ic - Tp(1);         // eq. 7
            const Tp b = rb * ic;                 // eq. 14
            const Tp x = X[r * v.xr + o * v.xo];
            // eq. 11 (step 6) as x (W^t q)_r / c_r: no cancellation where 1 + a is small
            const Tp xmu = x * (ra * ic);
            Tp xd;
            if (a < Tp(0)) {                      // eq. 15 with the eps floor on the gain
                const Tp xb = x * b;
                const Tp g = dev_div(xb, xb - a);
                xd = x * (g > eps ? g : eps);
            } else {                              // eq. 17, gain capped at 1 + alpha
                const Tp st = b > Tp(0) ? dev_div(a, b) : Tp(0);
                const Tp cap = alpha * x;
                xd = x + (st < cap ? st : cap);
            }
            Xmu[r * v.O + o] = xmu;
            Xdna[r * v.O + o] = xd;
            den += cs[r] * xd;
        }
    }
    red[ty][tx] = (double)den;
    __syncthreads();
    if (live) {
        double tot = 0.0;
        for (int k = 0; k < 8; ++k) tot += red[k][tx];
        const Tp sc = (Tp)(tot > 0.0 ? v.vsum[o] / tot : 1.0);   // eq. 10
        for (int64_t r = ty; r < v.R; r += 8) Xdna[r * v.O + o] *= sc;
    }
    __syncthreads();   // the shared arrays are reused by the next tile
}

template <typename Tp>
__global__ void __launch_bounds__(256) k_candidates(View v, const double* __restrict__ c,
                                                    const Tp* __restrict__ Apart,
                                                    const Tp* __restrict__ Bpart, int splits,
                                                    Tp* __restrict__ Xmu, Tp* __restrict__ Xdna,
                                                    Tp eps, Tp alpha) {
    candidates_tile<Tp>(v, c, Apart, Bpart, splits, Xmu, Xdna, eps, alpha, blockIdx.x);
}

// MU in place (eq. 11): x(r, o) <- x(r, o) * raw_a(r, o) / c_r.
template <typename Tp>
__global__ void k_mu_apply(View v, const double* __restrict__ c, const Tp* __restrict__ Apart,
                           int splits) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= v.O) return;
    Tp* __restrict__ X = static_cast<Tp*>(v.X);
    for (int64_t r = 0; r < v.R; ++r) {
        Tp ra = Tp(0);
        for (int sp = 0; sp < splits; ++sp) ra += Apart[((int64_t)sp * v.R + r) * v.O + o];
        X[r * v.xr + o * v.xo] = X[r * v.xr + o * v.xo] * (ra / (Tp)c[r]);
    }
}

// Selection (step 15 / 28): keep the Newton candidate iff d_dna < d_mu (ties keep MU),
// each cost being the column's eq. 5 sub-problem cost less a constant: the pass-2 sum
// plus reg * sum_r x(r, o) (reg = lambda for H, rho for W; eq. 5 and its mirror eq. 4).
// CTA = 32 columns o x 8 groups of r.
template <typename Tp>
__device__ __forceinline__ void select_tile(const View& v, const Tp* __restrict__ Xmu,
                                            const Tp* __restrict__ Xdna,
                                            const double* __restrict__ dpart, int splits,
                                            uint8_t* __restrict__ choice,
                                            double* __restrict__ dfin, int64_t tile_o,
                                            double reg) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t o = tile_o * 32 + tx;
    if (o >= v.O) return;
    double dm = 0.0, dd = 0.0;
    for (int sp = 0; sp < splits; ++sp) {
        dm += dpart[((int64_t)sp * 2 + 0) * v.O + o];
        dd += dpart[((int64_t)sp * 2 + 1) * v.O + o];
    }
    if (reg != 0.0) {   // the penalty of eq. 5, summed over r in ascending order
        double sm = 0.0, sd = 0.0;
        for (int64_t r = 0; r < v.R; ++r) {
            sm += (double)Xmu[r * v.O + o];
            sd += (double)Xdna[r * v.O + o];
        }
        dm += reg * sm;
        dd += reg * sd;
    }
    const bool newton = dd < dm;
    if (ty == 0) {
        choice[o] = newton ? 1 : 0;
        dfin[o] = dm;
        dfin[v.O + o] = dd;
    }
    Tp* __restrict__ X = static_cast<Tp*>(v.X);
    const Tp* __restrict__ src = newton ? Xdna : Xmu;
    for (int64_t r = ty; r < v.R; r += 8) X[r * v.xr + o * v.xo] = src[r * v.O + o];
}

template <typename Tp>
__global__ void __launch_bounds__(256) k_select(View v, const Tp* __restrict__ Xmu,
                                                const Tp* __restrict__ Xdna,
                                                const double* __restrict__ dpart, int splits,
                                                uint8_t* __restrict__ choice,
                                                double* __restrict__ dfin, double reg) {
    select_tile<Tp>(v, Xmu, Xdna, dpart, splits, choice, dfin, blockIdx.x, reg);
}

// Gradient of eq. 1 with respect to the view's X from the raw pass-1 sums:
// G(r, o) = scale * (c_r - sum over splits of Apart(r, o)) = scale * sum_s y(s, r)(1 - q(s, o)),
// written to G[r * gr + o * go].  CTA = 32 values of o x 8 groups of r.
template <typename Tp>
__global__ void __launch_bounds__(256) k_grad_x(View v, const double* __restrict__ c,
                                                const Tp* __restrict__ Apart, int splits,
                                                double scale, Tp* __restrict__ G, int64_t gr,
                                                int64_t go) {
    const int64_t o = (int64_t)blockIdx.x * 32 + threadIdx.x;
    if (o >= v.O) return;
    const Tp sc = (Tp)scale;
    for (int64_t r = threadIdx.y; r < v.R; r += 8) {
        Tp a = Tp(0);
        for (int sp = 0; sp < splits; ++sp) a += Apart[((int64_t)sp * v.R + r) * v.O + o];
        G[r * gr + o * go] = sc * ((Tp)c[r] - a);
    }
}

// Gradient of eq. 1 with respect to V: dV(s, o) = scale * log(v / z) where v > 0, else 0,
// with z(s, o) = sum_r y(s, r) x(r, o).  One CTA per 64 x 64 tile of (s, o).
template <typename Tp, int RB>
__global__ void __launch_bounds__(NT) k_grad_v(View v, double scale, Tp* __restrict__ dV,
                                               int64_t ldd, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Tp* Yt = reinterpret_cast<Tp*>(smem_raw);  // [RB][LD]
    Tp* Xs = Yt + RB * LD;                     // [RB][LD]
    const Tp* __restrict__ V = static_cast<const Tp*>(v.V);
    const Tp* __restrict__ X = static_cast<const Tp*>(v.X);
    const Tp* __restrict__ Y = static_cast<const Tp*>(v.Y);
    const int tid = threadIdx.x;
    const int64_t o0 = (int64_t)blockIdx.x * OB, s0 = (int64_t)blockIdx.y * SB;
    const int zo = (tid % 16) * 4, zs = (tid / 16) * 4;
    Tp z[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) z[i][j] = Tp(0);
    for (int64_t p = 0; p * RB < v.R; ++p) {
        load_tile<Tp, RB, OB>(Xs, X, v.xr, v.xo, p * RB, o0, v.R, v.O);
        load_tile<Tp, RB, SB>(Yt, Y, v.yr, v.ys, p * RB, s0, v.R, v.S);
        __syncthreads();
        z_tile<Tp, RB>(Yt, Xs, zs, zo, z);
        __syncthreads();
    }
    int bad = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t s = s0 + zs + i;
        if (s >= v.S) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t o = o0 + zo + j;
            if (o >= v.O) continue;
            const Tp vv = V[s * v.vs + o];
            Tp g = Tp(0);
            if (vv > Tp(0)) {
                if (z[i][j] > Tp(0)) g = (Tp)scale * dev_log(vv / z[i][j]);
                else bad = 1;
            }
            dV[s * ldd + o] = g;
        }
    }
    if (bad) atomicOr(status, STATUS_NONFINITE);
}

// ------------------------------------------------------------------ adjoint of the H step
// One H half-step at fixed W (Algorithm 1 steps 2-15, no normalisation) maps column h to
//   MU column:     h'_r = h_r A_r / c_r                                  (eq. 11)
//   Newton column: h'_r = s g_r / D,  D = sum_l c_l g_l,  s = sum_n v_n  (eq. 10)
//                  g_r = h^2 b / (h b - a) (a < 0, gain > eps), eps h (floor),
//                        h + a / b (a >= 0, below the cap), (1 + alpha) h (cap)
// with a = A / c - 1, b = B / c, A = W^t (V / Z), B = (W o W)^t (V / Z^2), Z = W H.  The
// selection (which column took which candidate) is held fixed.  Given hb' = dL/dh', this
// kernel forms, per column, the direct part of dL/dh, the adjoints Abar = dL/dA and
// Bbar = dL/dB (raw sums), and vs = dL/ds.  With cpart it also forms the part of dL/dW
// that flows through the column sums c_r = sum_n w_nr + lambda (every w_nr of column r
// receives it):
//   dL/dc_r = -(abar (a + 1) + bbar b) / c_r - [Newton] (s hg / D^2) g_r
// (a = A / c - 1 and b = B / c, so da/dc = -(a + 1) / c and db/dc = -b / c; the eq. 10
// denominator D = sum_l c_l g_l gives dD/dc_r = g_r, and dL/dD = -s hg / D^2 with
// hg = sum_r hb'_r g_r), summed over the CTA's 32 columns into cpart[blockIdx.x][r].
// CTA = 32 columns x 8 groups of r (one warp per group).
template <typename Tp>
__global__ void __launch_bounds__(256)
    k_adj_elem(View v, const double* __restrict__ c, const Tp* __restrict__ Apart,
               const Tp* __restrict__ Bpart, int splits, const uint8_t* __restrict__ choice,
               const Tp* __restrict__ Hbar1, Tp* __restrict__ Hbar0, Tp* __restrict__ Abar,
               Tp* __restrict__ Bbar, double* __restrict__ vs, Tp eps, Tp alpha,
               double* __restrict__ cpart) {
    __shared__ double red[2][8][32];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t o = (int64_t)blockIdx.x * 32 + tx;
    const bool live = o < v.O;
    const Tp* __restrict__ X = static_cast<const Tp*>(v.X);
    const bool newton = live && choice[o];
    // pass 1 over r: D = sum c g and sum hb' g (Newton columns)
    double dsum = 0.0, hg = 0.0;
    if (newton) {
        for (int64_t r = ty; r < v.R; r += 8) {
            Tp ra = Tp(0), rb = Tp(0);
            for (int sp = 0; sp < splits; ++sp) {
                ra += Apart[((int64_t)sp * v.R + r) * v.O + o];
                rb += Bpart[((int64_t)sp * v.R + r) * v.O + o];
            }
            const Tp cr = (Tp)c[r], x = X[r * v.xr + o * v.xo];
            const Tp a = ra / cr - Tp(1), b = rb / cr;
            Tp g;
            if (a < Tp(0)) {
                const Tp xb = x * b, gain = xb / (xb - a);
                g = x * (gain > eps ? gain : eps);
            } else {
                const Tp st = b > Tp(0) ? a / b : Tp(0), cap = alpha * x;
                g = x + (st < cap ? st : cap);
            }
            dsum += (double)(cr * g);
            hg += (double)(Hbar1[r * v.xr + o * v.xo] * g);
        }
    }
    red[0][ty][tx] = dsum;
    red[1][ty][tx] = hg;
    __syncthreads();
    double D = 0.0, HG = 0.0;
    for (int k = 0; k < 8; ++k) { D += red[0][k][tx]; HG += red[1][k][tx]; }
    const double s_o = live ? v.vsum[o] : 0.0;
    const bool renorm = D > 0.0;
    const Tp f1 = (Tp)(renorm ? s_o / D : 1.0);            // d h' / d g (diagonal part)
    const Tp f2 = (Tp)(renorm ? s_o * HG / (D * D) : 0.0); // weight of the D coupling
    if (ty == 0 && live) vs[o] = (newton && renorm) ? HG / D : 0.0;
    // the loop bound is uniform over the warp (one warp per ty), so every lane takes part
    // in the cpart shuffle; lanes past the last column contribute 0
    for (int64_t r = ty; r < v.R; r += 8) {
        double cb = 0.0;
        if (live) {
            Tp ra = Tp(0), rb = Tp(0);
            for (int sp = 0; sp < splits; ++sp) {
                ra += Apart[((int64_t)sp * v.R + r) * v.O + o];
                rb += Bpart[((int64_t)sp * v.R + r) * v.O + o];
            }
            const Tp cr = (Tp)c[r], x = X[r * v.xr + o * v.xo];
            const Tp hb1 = Hbar1[r * v.xr + o * v.xo];
            const Tp a = ra / cr - Tp(1), b = rb / cr;
            Tp hx, ab = Tp(0), bb = Tp(0);   // dL/dh (direct), dL/da, dL/db
            Tp g = Tp(0);                    // the Newton column's g_r (for dL/dc)
            if (!newton) {                   // h' = h (1 + a)
                hx = hb1 * (Tp(1) + a);
                ab = hb1 * x;
            } else {
                const Tp gb = f1 * hb1 - cr * f2;   // dL/dg_r
                if (a < Tp(0)) {
                    const Tp xb = x * b, den = xb - a, gain = xb / den;
                    if (gain > eps) {                // g = x^2 b / (x b - a)
                        const Tp d2 = den * den;
                        hx = gb * xb * (xb - Tp(2) * a) / d2;
                        ab = gb * x * xb / d2;
                        bb = -gb * a * x * x / d2;
                        g = x * gain;
                    } else {                         // floor: g = eps x
                        hx = gb * eps;
                        g = eps * x;
                    }
                } else {
                    const Tp st = b > Tp(0) ? a / b : Tp(0), cap = alpha * x;
                    if (st < cap) {                  // g = x + a / b
                        hx = gb;
                        if (b > Tp(0)) { ab = gb / b; bb = -gb * a / (b * b); }
                        g = x + st;
                    } else {                         // cap: g = (1 + alpha) x
                        hx = gb * (Tp(1) + alpha);
                        g = x + cap;
                    }
                }
            }
            Hbar0[r * v.xr + o * v.xo] = hx;
            Abar[r * v.O + o] = ab / cr;     // a = A / c - 1
            Bbar[r * v.O + o] = bb / cr;     // b = B / c
            cb = -(double)(ab * (a + Tp(1)) + bb * b) / (double)cr - (double)(f2 * g);
        }
        if (cpart) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) cb += __shfl_xor_sync(0xffffffffu, cb, off);
            if (tx == 0) cpart[(int64_t)blockIdx.x * v.R + r] = cb;
        }
    }
}

template <typename Tp, int RB>
struct AdjCfg {
    static constexpr int RPT = RB / 16;
    static constexpr size_t smem = (size_t)(4 * RB * LD + SB * LD) * sizeof(Tp);
};

// The GEMM-shaped part of the adjoint, per (o-block, r-block = all R <= RB, s-split):
//   P1 = Y Abar, P2 = (Y o Y) Bbar                       (z-tiles, K = R)
//   zbar = -qbar P1 - 2 (qbar / z) P2,  qbar = v / z^2    (through A and B)
//   Hpart += Y^t zbar                                    (through z = W h)
//   Vbar(s, o) += P1 / z + P2 / z^2 + vs_o               (through q, qbar and s)
// Vbar is owned element-wise by one thread per split range, so it is updated in place.
template <typename Tp, int RB>
__global__ void __launch_bounds__(NT)
    k_adj_gemm(View v, const Tp* __restrict__ Abar, const Tp* __restrict__ Bbar,
               const double* __restrict__ vs, Tp* __restrict__ Hpart, Tp* __restrict__ Vbar,
               int64_t ldvb, int64_t s_per, int* __restrict__ status) {
    using C = AdjCfg<Tp, RB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Tp* Xs = reinterpret_cast<Tp*>(smem_raw);  // [RB][LD] x(r, o)
    Tp* As = Xs + RB * LD;                     // [RB][LD] Abar(r, o)
    Tp* Bs = As + RB * LD;                     // [RB][LD] Bbar(r, o)
    Tp* Yt = Bs + RB * LD;                     // [RB][LD] y(s, r) transposed
    Tp* Zb = Yt + RB * LD;                     // [SB][LD] zbar(s, o)
    const Tp* __restrict__ V = static_cast<const Tp*>(v.V);
    const Tp* __restrict__ X = static_cast<const Tp*>(v.X);
    const Tp* __restrict__ Y = static_cast<const Tp*>(v.Y);
    const int tid = threadIdx.x;
    const int64_t o0 = (int64_t)blockIdx.x * OB;
    const int64_t s_begin = (int64_t)blockIdx.y * s_per;
    const int64_t s_end = min(v.S, s_begin + s_per);
    const int zo = (tid % 16) * 4, zs = (tid / 16) * 4;
    const int go = (tid % 16) * 4, gr = tid / 16;
    Tp acc[C::RPT][4];
#pragma unroll
    for (int i = 0; i < C::RPT; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = Tp(0);
    load_tile<Tp, RB, OB>(Xs, X, v.xr, v.xo, 0, o0, v.R, v.O);
    load_tile<Tp, RB, OB>(As, Abar, v.O, 1, 0, o0, v.R, v.O);
    load_tile<Tp, RB, OB>(Bs, Bbar, v.O, 1, 0, o0, v.R, v.O);
    int bad = 0;
    for (int64_t s0 = s_begin; s0 < s_end; s0 += SB) {
        load_tile<Tp, RB, SB>(Yt, Y, v.yr, v.ys, 0, s0, v.R, v.S);
        __syncthreads();
        Tp z[4][4], p1[4][4], p2[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) { z[i][j] = Tp(0); p1[i][j] = Tp(0); p2[i][j] = Tp(0); }
        z_tile<Tp, RB>(Yt, Xs, zs, zo, z);
        z_tile<Tp, RB>(Yt, As, zs, zo, p1);
#pragma unroll 4
        for (int r = 0; r < RB; ++r) {   // P2 = (Y o Y) Bbar
            Tp ba[4], ya[4];
            ld4(Bs + r * LD + zo, ba);
            ld4(Yt + r * LD + zs, ya);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) p2[i][j] = fma(ya[i] * ya[i], ba[j], p2[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t s = s0 + zs + i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t o = o0 + zo + j;
                Tp zb = Tp(0);
                if (s < s_end && o < v.O) {
                    const Tp vv = V[s * v.vs + o], zz = z[i][j];
                    Tp vb = (Tp)vs[o];
                    if (vv > Tp(0)) {
                        if (zz > Tp(0)) {
                            const Tp iz = Tp(1) / zz, qb = vv * iz * iz;
                            zb = -qb * p1[i][j] - Tp(2) * qb * iz * p2[i][j];
                            vb += p1[i][j] * iz + p2[i][j] * iz * iz;
                        } else {
                            bad = 1;
                        }
                    } else if (zz > Tp(0)) {
                        const Tp iz = Tp(1) / zz;
                        vb += p1[i][j] * iz + p2[i][j] * iz * iz;
                    }
                    if (Vbar) Vbar[s * ldvb + o] += vb;
                }
                Zb[(zs + i) * LD + zo + j] = zb;
            }
        }
        __syncthreads();
        // Hpart(r, o) += sum_s y(s, r) zbar(s, o)
#pragma unroll 2
        for (int s = 0; s < SB; ++s) {
            Tp zv[4];
            ld4(Zb + s * LD + go, zv);
#pragma unroll
            for (int i = 0; i < C::RPT; ++i) {
                const Tp y = Yt[(gr + 16 * i) * LD + s];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(y, zv[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(status, STATUS_NONFINITE);
    const int64_t base = (int64_t)blockIdx.y * v.R;
#pragma unroll
    for (int i = 0; i < C::RPT; ++i) {
        const int64_t r = gr + 16 * i;
        if (r >= v.R) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t o = o0 + go + j;
            if (o < v.O) Hpart[(base + r) * v.O + o] = acc[i][j];
        }
    }
}

// The part of dL/dW of one H step that flows through A, B and Z (W held as a variable):
//   A = W^t Q, B = (W o W)^t Qbar, Z = W H, Q = V / Z, Qbar = V / Z^2 give
//   dL/dw_sr = sum_o [ q(s,o) Abar(r,o) + 2 w_sr qbar(s,o) Bbar(r,o) + zbar(s,o) x(r,o) ]
// with zbar = -qbar P1 - 2 (qbar / z) P2, P1 = W Abar, P2 = (W o W) Bbar as in k_adj_gemm.
// Each CTA owns a 64-row s-block and every r <= RB, walks its split of o in 64-wide chunks
// (z, P1, P2 as 4 x 4 register tiles, then q, qbar, zbar as shared tiles [o][s]) and
// accumulates the two sums of the (r, s) tile in registers; Wpart is [splits][R][S].
// The y^t tile and the zbar tile share one region (y^t is reloaded per chunk).
template <typename Tp, int RB>
struct WgradCfg {
    static constexpr int RPT = RB / 16;            // r rows per thread of the (r, s) tile
    static constexpr int UR = RB > SB ? RB : SB;   // rows of the y^t / zbar region
    static constexpr size_t smem = (size_t)((3 * RB + UR + 2 * OB) * LD) * sizeof(Tp);
};

template <typename Tp, int RB>
__global__ void __launch_bounds__(NT)
    k_adj_wgrad(View v, const Tp* __restrict__ Abar, const Tp* __restrict__ Bbar,
                Tp* __restrict__ Wpart, int64_t o_per, int* __restrict__ status) {
    using C = WgradCfg<Tp, RB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Tp* Xs = reinterpret_cast<Tp*>(smem_raw);  // [RB][LD] x(r, o)
    Tp* As = Xs + RB * LD;                     // [RB][LD] Abar(r, o)
    Tp* Bs = As + RB * LD;                     // [RB][LD] Bbar(r, o)
    Tp* Yt = Bs + RB * LD;                     // [RB][LD] y(s, r) transposed, or
    Tp* Zb = Yt;                               // [OB][LD] zbar(s, o) transposed
    Tp* Qs = Yt + C::UR * LD;                  // [OB][LD] q(s, o) transposed
    Tp* Qb = Qs + OB * LD;                     // [OB][LD] qbar(s, o) transposed
    const Tp* __restrict__ V = static_cast<const Tp*>(v.V);
    const Tp* __restrict__ X = static_cast<const Tp*>(v.X);
    const Tp* __restrict__ Y = static_cast<const Tp*>(v.Y);
    const int tid = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * SB;
    const int64_t o_begin = (int64_t)blockIdx.y * o_per;
    const int64_t o_end = min(v.O, o_begin + o_per);
    const int zo = (tid % 16) * 4, zs = (tid / 16) * 4;   // (s, o) tile of the GEMM phase
    const int gs = (tid % 16) * 4, gr = tid / 16;         // (r, s) tile of the sums
    Tp acc1[C::RPT][4], acc2[C::RPT][4];
#pragma unroll
    for (int i = 0; i < C::RPT; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc1[i][j] = Tp(0); acc2[i][j] = Tp(0); }
    int bad = 0;
    for (int64_t oc = o_begin; oc < o_end; oc += OB) {
        load_tile<Tp, RB, SB>(Yt, Y, v.yr, v.ys, 0, s0, v.R, v.S);
        load_tile<Tp, RB, OB>(Xs, X, v.xr, v.xo, 0, oc, v.R, o_end);
        load_tile<Tp, RB, OB>(As, Abar, v.O, 1, 0, oc, v.R, o_end);
        load_tile<Tp, RB, OB>(Bs, Bbar, v.O, 1, 0, oc, v.R, o_end);
        __syncthreads();
        Tp z[4][4], p1[4][4], p2[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) { z[i][j] = Tp(0); p1[i][j] = Tp(0); p2[i][j] = Tp(0); }
        z_tile<Tp, RB>(Yt, Xs, zs, zo, z);
        z_tile<Tp, RB>(Yt, As, zs, zo, p1);
#pragma unroll 4
        for (int r = 0; r < RB; ++r) {   // P2 = (Y o Y) Bbar
            Tp ba[4], ya[4];
            ld4(Bs + r * LD + zo, ba);
            ld4(Yt + r * LD + zs, ya);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) p2[i][j] = fma(ya[i] * ya[i], ba[j], p2[i][j]);
        }
        __syncthreads();   // every read of the y^t tile is done: the region becomes zbar
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t s = s0 + zs + i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t o = oc + zo + j;
                Tp q = Tp(0), qb = Tp(0), zb = Tp(0);
                if (s < v.S && o < o_end) {
                    const Tp vv = V[s * v.vs + o], zz = z[i][j];
                    if (vv > Tp(0)) {
                        if (zz > Tp(0)) {
                            const Tp iz = Tp(1) / zz;
                            q = vv * iz;
                            qb = q * iz;
                            zb = -qb * p1[i][j] - Tp(2) * qb * iz * p2[i][j];
                        } else {
                            bad = 1;
                        }
                    }
                }
                Qs[(zo + j) * LD + zs + i] = q;
                Qb[(zo + j) * LD + zs + i] = qb;
                Zb[(zo + j) * LD + zs + i] = zb;
            }
        }
        __syncthreads();
        // acc1(r, s) += sum_o Abar(r, o) q(s, o) + x(r, o) zbar(s, o);
        // acc2(r, s) += sum_o Bbar(r, o) qbar(s, o)
#pragma unroll 2
        for (int o = 0; o < OB; ++o) {
            Tp qv[4], qbv[4], zbv[4];
            ld4(Qs + o * LD + gs, qv);
            ld4(Qb + o * LD + gs, qbv);
            ld4(Zb + o * LD + gs, zbv);
#pragma unroll
            for (int i = 0; i < C::RPT; ++i) {
                const int r = gr + 16 * i;
                const Tp a = As[r * LD + o], x = Xs[r * LD + o], b = Bs[r * LD + o];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc1[i][j] = fma(a, qv[j], fma(x, zbv[j], acc1[i][j]));
                    acc2[i][j] = fma(b, qbv[j], acc2[i][j]);
                }
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(status, STATUS_NONFINITE);
    const int64_t base = (int64_t)blockIdx.y * v.R;
#pragma unroll
    for (int i = 0; i < C::RPT; ++i) {
        const int64_t r = gr + 16 * i;
        if (r >= v.R) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t s = s0 + gs + j;
            if (s >= v.S) continue;
            const Tp w = Y[s * v.ys + r * v.yr];
            Wpart[(base + r) * v.S + s] = acc1[i][j] + Tp(2) * w * acc2[i][j];
        }
    }
}

// Wbar(s, r) += sum over splits of Wpart(r, s) + sum over parts of cpart(r) (the column-sum
// term of k_adj_elem), Wbar laid out like the view's Y.  CTA = 32 values of s x 8 of r.
template <typename Tp>
__global__ void __launch_bounds__(256)
    k_adj_wcombine(View v, const Tp* __restrict__ Wpart, int splits,
                   const double* __restrict__ cpart, int64_t nparts, Tp* __restrict__ Wbar) {
    __shared__ double cb[128];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    for (int64_t r = tid; r < v.R; r += 256) {
        double t = 0.0;
        for (int64_t k = 0; k < nparts; ++k) t += cpart[k * v.R + r];
        cb[r] = t;
    }
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * 32 + tx;
    if (s >= v.S) return;
    for (int64_t r = ty; r < v.R; r += 8) {
        double t = cb[r];
        for (int sp = 0; sp < splits; ++sp) t += (double)Wpart[((int64_t)sp * v.R + r) * v.S + s];
        Tp* w = Wbar + s * v.ys + r * v.yr;
        *w = (Tp)((double)*w + t);
    }
}

// Hbar(r, o) += sum over splits of Hpart(r, o).
template <typename Tp>
__global__ void __launch_bounds__(256) k_adj_combine(View v, const Tp* __restrict__ Hpart,
                                                     int splits, Tp* __restrict__ Hbar) {
    const int64_t o = (int64_t)blockIdx.x * 32 + threadIdx.x;
    if (o >= v.O) return;
    for (int64_t r = threadIdx.y; r < v.R; r += 8) {
        Tp t = Tp(0);
        for (int sp = 0; sp < splits; ++sp) t += Hpart[((int64_t)sp * v.R + r) * v.O + o];
        Hbar[r * v.xr + o * v.xo] += t;
    }
}

// A factor sum that is exactly zero (an all-zero column of W or row of H without
// regularisation, excluded by the assumption of Section 2) is replaced by 1.
__device__ __forceinline__ double nonzero_sum(double s, bool guard) {
    return (guard && s == 0.0) ? 1.0 : s;
}

// out[r] = sum_i M(i, r) + reg for a matrix with element (i, r) at M[i * si + r * sr],
// i < n.  One CTA of 32 x 8 threads per 32 values of r; fixed summation order.
template <typename Tp>
__global__ void k_factor_sums(const Tp* __restrict__ M, int64_t n, int64_t R, int64_t si,
                              int64_t sr, double reg, double* __restrict__ out, bool guard) {
    __shared__ double red[8][33];
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int64_t r = (int64_t)blockIdx.x * 32 + lane;
    double s = 0.0;
    if (r < R)
        for (int64_t i = ty; i < n; i += 8) s += (double)M[i * si + r * sr];
    red[ty][lane] = s;
    __syncthreads();
    if (ty == 0 && r < R) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[k][lane];
        out[r] = nonzero_sum(t + reg, guard);
    }
}

// Column sums in two levels: part[split][r] = sum over rows i of split `split` of M(i, r),
// M(i, r) at M[i * si + r * sr]; grid = (ceil(R / 32), nsplit), CTA 32 x 8.
template <typename Tp>
__global__ void k_colsum_part(const Tp* __restrict__ M, int64_t n, int64_t R, int64_t si,
                              int64_t sr, int64_t rows_per, double* __restrict__ part) {
    __shared__ double red[8][33];
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int64_t r = (int64_t)blockIdx.x * 32 + lane;
    const int64_t i0 = (int64_t)blockIdx.y * rows_per, i1 = min(n, i0 + rows_per);
    Tp s = Tp(0);
    if (r < R)
        for (int64_t i = i0 + ty; i < i1; i += 8) s += M[i * si + r * sr];
    red[ty][lane] = (double)s;
    __syncthreads();
    if (ty == 0 && r < R) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[k][lane];
        part[(int64_t)blockIdx.y * R + r] = t;
    }
}

// out[r] = sum over k of part[k][r] + reg for a few r: one CTA per r, 256 partial sums
// per thread stride, then a fixed tree (the part_sums of the glue, R small).  With `next`,
// also next[r] = d_r / out[r] + reg (d_r the sum without reg, an exact zero guarded): the
// sum over the row of the factor that the step 16 / 29 normalisation divides by out[r],
// plus reg, which is the eq. 7 / 14 denominator of the following half-step.  A template
// only so that every translation unit including this header may define it.
template <int UNUSED = 0>
__global__ void __launch_bounds__(256) k_colsum_small(const double* __restrict__ part,
                                                      int nsplit, int64_t R, double reg,
                                                      double* __restrict__ out, bool guard,
                                                      double* __restrict__ next = nullptr) {
    __shared__ double red[256];
    const int64_t r = blockIdx.x;
    double t = 0.0;
    for (int k = threadIdx.x; k < nsplit; k += 256) t += part[(int64_t)k * R + r];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double f = nonzero_sum(red[0] + reg, guard);
        out[r] = f;
        if (next) next[r] = nonzero_sum(red[0] / f + reg, true);
    }
}

// out[r] (and next[r]) as k_colsum_small for many r.  CTA = 32 values of r (lanes, so loads
// coalesce) x 32 groups of splits: group g adds splits g, g + 32, ... in order, then the 32
// group sums are added in order.
template <int UNUSED = 0>
__global__ void __launch_bounds__(1024) k_colsum_final(const double* __restrict__ part,
                                                       int nsplit, int64_t R, double reg,
                                                       double* __restrict__ out, bool guard,
                                                       double* __restrict__ next = nullptr) {
    __shared__ double red[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t r = (int64_t)blockIdx.x * 32 + tx;
    double t = 0.0;
    if (r < R) {
#pragma unroll 4
        for (int k = ty; k < nsplit; k += 32) t += part[(int64_t)k * R + r];
    }
    red[ty][tx] = t;
    __syncthreads();
    if (ty == 0 && r < R) {
        double tot = 0.0;
        for (int g = 0; g < 32; ++g) tot += red[g][tx];
        const double f = nonzero_sum(tot + reg, guard);
        out[r] = f;
        if (next) next[r] = nonzero_sum(tot / f + reg, true);
    }
}

// Row-sum variant for unit-stride rows (element (r, i) at M[r * ld + i]): one CTA of 256
// threads per r; per-thread sums, then fixed-order warp butterflies and a final pass over
// the 8 warp sums.
template <typename Tp>
__global__ void __launch_bounds__(256) k_row_sums(const Tp* __restrict__ M, int64_t n, int64_t ld,
                                                  double reg, double* __restrict__ out, bool guard) {
    __shared__ double red[8];
    const int64_t r = blockIdx.x;
    // per-thread sums in the element type (four independent chains), float64 across threads
    Tp s0 = Tp(0), s1 = Tp(0), s2 = Tp(0), s3 = Tp(0);
    const Tp* __restrict__ row = M + r * ld;
    int64_t i = threadIdx.x;
    for (; i + 768 < n; i += 1024) {
        s0 += row[i];
        s1 += row[i + 256];
        s2 += row[i + 512];
        s3 += row[i + 768];
    }
    for (; i < n; i += 256) s0 += row[i];
    double s = (double)(s0 + s1) + (double)(s2 + s3);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[k];
        out[r] = nonzero_sum(t + reg, guard);
    }
}

// X(r, o) /= f_r for all (r, o) and Y(s, r) *= f_r for all (s, r) (steps 1, 16, 29).
// blockIdx.y < ceil(R / 8) covers X, the rest covers Y; threadIdx.y picks r within a group
// of 8 and threadIdx.x walks the other index, so no element needs an integer division.
template <typename Tp>
__global__ void __launch_bounds__(256) k_rescale(View v, const double* __restrict__ f,
                                                 int64_t xblocks) {
    const int64_t rg = (int64_t)blockIdx.y;
    const bool isx = rg < xblocks;
    const int64_t r = (isx ? rg : rg - xblocks) * 8 + threadIdx.y;
    if (r >= v.R) return;
    const Tp fr = isx ? Tp(1) / (Tp)f[r] : (Tp)f[r];   // X is divided, Y multiplied
    const int64_t n = isx ? v.O : v.S;
    Tp* __restrict__ M = isx ? static_cast<Tp*>(v.X)
                             : const_cast<Tp*>(static_cast<const Tp*>(v.Y));
    const int64_t stride_r = isx ? v.xr : v.yr, stride_i = isx ? v.xo : v.ys;
    for (int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 32) {
        const int64_t idx = r * stride_r + i * stride_i;
        M[idx] *= fr;
    }
}

// Vt[t][n] = V[n][t] (32 x 32 tiles).
template <typename Tp>
__global__ void k_transpose(const Tp* __restrict__ V, int64_t N, int64_t T, int64_t ldv,
                            Tp* __restrict__ Vt, int64_t ldvt) {
    __shared__ Tp tile[32][33];
    const int64_t n0 = (int64_t)blockIdx.y * 32, t0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t n = n0 + k, t = t0 + threadIdx.x;
        tile[k][threadIdx.x] = (n < N && t < T) ? V[n * ldv + t] : Tp(0);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t t = t0 + k, n = n0 + threadIdx.x;
        if (t < T && n < N) Vt[t * ldvt + n] = tile[threadIdx.x][k];
    }
}


// k_transpose fused with the column and row sums of V: per 32 x 32 tile the sums of its
// 32 rows (colpart[n-tile][t]) and of its 32 columns (rowpart[t-tile][n]), in the element
// type (exact for counts), for k_colsum_final to add up in float64.  With Vc, also a copy
// of V into Vc (leading dimension T): V may then be pinned host memory that the kernel
// reads across the host link (the copy in of dna_run_host).
template <typename Tp>
__global__ void __launch_bounds__(256) k_transpose_sums(const Tp* __restrict__ V, int64_t N,
                                                        int64_t T, int64_t ldv,
                                                        Tp* __restrict__ Vt, int64_t ldvt,
                                                        double* __restrict__ colpart,
                                                        double* __restrict__ rowpart,
                                                        Tp* __restrict__ Vc = nullptr) {
    __shared__ Tp tile[32][33];
    const int64_t n0 = (int64_t)blockIdx.y * 32, t0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t n = n0 + k, t = t0 + threadIdx.x;
        const Tp x = (n < N && t < T) ? V[n * ldv + t] : Tp(0);
        tile[k][threadIdx.x] = x;
        if (Vc && n < N && t < T) Vc[n * T + t] = x;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t t = t0 + k, n = n0 + threadIdx.x;
        if (t < T && n < N) Vt[t * ldvt + n] = tile[threadIdx.x][k];
    }
    if (threadIdx.y == 0) {          // column t0 + lane: sum over the tile's rows
        Tp sum = Tp(0);
#pragma unroll 8
        for (int k = 0; k < 32; ++k) sum += tile[k][threadIdx.x];
        const int64_t t = t0 + threadIdx.x;
        if (t < T) colpart[(int64_t)blockIdx.y * T + t] = (double)sum;
    } else if (threadIdx.y == 1) {   // row n0 + lane: sum over the tile's columns
        Tp sum = Tp(0);
#pragma unroll 8
        for (int k = 0; k < 32; ++k) sum += tile[threadIdx.x][k];
        const int64_t n = n0 + threadIdx.x;
        if (n < N) rowpart[(int64_t)blockIdx.x * N + n] = (double)sum;
    }
}

}  // namespace simt
}  // namespace dna
