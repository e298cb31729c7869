// Internal interfaces of the DNA library (not part of the C ABI).
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the driver entry point is looked up at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "dna.h"

namespace dna {

// Kernel launches issued by this host thread (read around each phase for dna_phase_times).
inline int64_t& launch_count() {
    static thread_local int64_t n = 0;
    return n;
}
// Call right after each kernel launch: counts it and reports a launch error.
inline int after_launch() {
    ++launch_count();
    return cudaGetLastError() == cudaSuccess ? DNA_OK : DNA_ERR_CUDA;
}

// Partial-sum slots of the two-level factor sums.
constexpr int FSUM_SPLITS = 64;

// Device status bits (sticky, OR-ed by kernels, read by synchronising calls).
enum : int { STATUS_NONFINITE = 1, STATUS_TIMEOUT = 2 };

// One half-step seen as "update the owned factor X (R x O) with the fixed factor
// Y (S x R)", reducing over s (Section 2: the W half-step is the H half-step on the
// transposes).  H-step: s = n, o = t, X = H, Y = W, V_so = V.  W-step: s = t, o = n,
// X = W^t, Y = H^t, V_so = V^t (the transposed copy made at bind time).
struct View {
    int64_t S, O, R;
    const void* V;      // V_so, element (s, o) at V[s * vs + o]
    int64_t vs;
    void* X;            // element (r, o) at X[r * xr + o * xo]
    int64_t xr, xo;
    const void* Y;      // element (s, r) at Y[s * ys + r * yr]
    int64_t ys, yr;
    const double* vsum; // sum_s v(s, o), length O (the eq. 10 target)
};

// Segment table of one view of a sparse V: segment g covers the non-zeros [k0[g], k1[g])
// of view column col[g]; the segments of column o are [sptr[o], sptr[o + 1]).
constexpr int SPARSE_SEG = 128;   // non-zeros per segment at most

struct SparseSegs {
    const int32_t* col;
    const int64_t* k0;
    const int64_t* k1;
    const int64_t* sptr;
    int64_t n;
};

// Launchers, one instantiation per element type (float, double).  Each returns a
// DNA_* status (launch errors only; device-side errors go to *status).
template <typename Tp> struct Simt {
    // sum over s of y(s, r) + reg -> out[r] (the eq. 7 / 14 denominators); work holds at
    // least FSUM_SPLITS * R float64
    static int factor_sums_y(const View& v, double reg, double* out, double* work,
                             cudaStream_t st);
    // sum over o of x(r, o) + reg -> out[r] (the step 16 / 29 normalisers)
    static int factor_sums_x(const View& v, double reg, double* out, double* work,
                             cudaStream_t st);
    // x(r, o) *= f_r^-1 ... : X scaled by 1/f_r, Y scaled by f_r (steps 1, 16, 29)
    static int rescale(const View& v, const double* f, cudaStream_t st);
    // pass 1: raw sums Apart = sum_s y q, Bpart = sum_s y^2 qbar (split over s); with dcur,
    // also the starting factor's per-column costs [splits][O] (descent selection)
    static int pass1(const View& v, Tp* Apart, Tp* Bpart, int splits, int64_t s_per,
                     bool with_b, int* status, cudaStream_t st, double* dcur = nullptr);
    // candidates: MU and renormalised Newton candidates, laid out [R][O]
    static int candidates(const View& v, const double* c, const Tp* Apart, const Tp* Bpart,
                          int splits, Tp* Xmu, Tp* Xdna, double eps, double alpha,
                          cudaStream_t st);
    // MU update in place (eq. 11): x <- x * raw_a / c
    static int mu_apply(const View& v, const double* c, const Tp* Apart, int splits,
                        cudaStream_t st);
    // pass 2: per-column costs of the two candidates, float64 partials [splits][2][O]
    static int pass2(const View& v, const Tp* Xmu, const Tp* Xdna, double* dpart, int splits,
                     int64_t s_per, int* status, cudaStream_t st);
    // pass 2 for one candidate X ([R][O]): its per-column costs, dpart [splits][O]
    static int pass2_one(const View& v, const Tp* X, double* dpart, int splits, int64_t s_per,
                         int* status, cudaStream_t st);
    // selection: x(r, o) <- Newton if d_dna < d_mu else MU, each d being the pass-2 sum
    // plus reg * sum_r x (the eq. 5 penalty; reg = lambda for H, rho for W); choice and
    // final costs
    static int select(const View& v, const Tp* Xmu, const Tp* Xdna, const double* dpart,
                      int splits, uint8_t* choice, double* dfin, double reg, cudaStream_t st);
    // per-column full KL terms of eq. 1 for x = the view's X, partials [splits][O]
    static int kl_columns(const View& v, double* dpart, int splits, int64_t s_per,
                          int* status, cudaStream_t st);
    // gradient of eq. 1 w.r.t. X from raw pass-1 sums: G(r, o) at G[r * gr + o * go]
    static int grad_x(const View& v, const double* c, const Tp* Apart, int splits, double scale,
                      Tp* G, int64_t gr, int64_t go, cudaStream_t st);
    // gradient of eq. 1 w.r.t. V: dV(s, o) = scale log(v / z) (0 where v = 0)
    static int grad_v(const View& v, double scale, Tp* dV, int64_t ldd, int* status,
                      cudaStream_t st);
    // adjoint of one H step (see k_adj_elem / k_adj_gemm): Hbar0 = dL/dH_k given
    // Hbar1 = dL/dH_{k+1}; Vbar += dL/dV (Vbar may be null).  Uses A, B (pass 1 of H_k) and
    // the column choices.  With cpart ([ceil(O / 32)][R] float64) also the column-sum part
    // of dL/dW, per block of 32 columns.
    static int adjoint_h(const View& v, const double* c, const Tp* Apart, const Tp* Bpart,
                         int splits1, const uint8_t* choice, const Tp* Hbar1, Tp* Hbar0,
                         Tp* Abar, Tp* Bbar, double* vs, Tp* Hpart, int splits2, int64_t s_per2,
                         Tp* Vbar, int64_t ldvb, double eps, double alpha, int* status,
                         cudaStream_t st, double* cpart = nullptr);
    // after adjoint_h (its Abar, Bbar, cpart): Wbar += dL/dW of the step (k_adj_wgrad),
    // through Wpart [wsplits][R][S], o split in ranges of o_per (a multiple of 64)
    static int adjoint_w(const View& v, const Tp* Abar, const Tp* Bbar, const double* cpart,
                         Tp* Wpart, int wsplits, int64_t o_per, Tp* Wbar, int* status,
                         cudaStream_t st);
    // Fused glue of the single-problem path (glue_kernels.cuh).
    // Candidates as above; with Xmk, Xdk (float only) also their bf16 copies [O_pad][rp]
    // with zero padding.
    static int cand_fused(const View& v, const double* c, const Tp* Apart, const Tp* Bpart,
                          int splits, Tp* Xmu, Tp* Xdna, double eps, double alpha, void* Xmk,
                          void* Xdk, int64_t rp, int64_t O_pad, int64_t plane,
                          cudaStream_t st);
    // A[0] = sum over the splits of A[sp] (and B, if given), each [R][O]: ascending order.
    static int split_sum(Tp* A, Tp* B, int64_t R, int64_t O, int splits, cudaStream_t st);
    // cand_fused keeps a thread's candidates in registers and sums the split partials as
    // they stream in (no split_sum pass needed)
    static bool cand_in_registers(int64_t R);
    // Selection as above, plus fpart[glue_parts(O)][R]: per-block sums of the new X.
    // With dcur: descent selection (dpart = Newton costs [splits][O], dcur = the starting
    // factor's [cur_splits][O]).
    static int select_fused(const View& v, const Tp* Xmu, const Tp* Xdna, const double* dpart,
                            int splits, uint8_t* choice, double* dfin, double* fpart,
                            double reg, cudaStream_t st, const double* dcur = nullptr,
                            int cur_splits = 0);
    // out[r] = in[r] + reg (an exact zero replaced by 1)
    static int add_reg(const double* in, int64_t R, double reg, double* out, cudaStream_t st);
    // MU (eq. 11) in place from the pass-1 split partials, plus fpart as select_fused
    static int mu_fused(const View& v, const double* c, const Tp* Apart, int splits,
                        double* fpart, cudaStream_t st);
    // out[r] = sum over k < nparts of part[k * R + r] + reg (fixed order; an exact zero
    // sum is replaced by 1); with `next`, next[r] = (that sum without reg) / out[r] + reg
    // (guarded the same way)
    static int part_sums(const double* part, int64_t nparts, int64_t R, double reg, double* out,
                         cudaStream_t st, double* next = nullptr);
    // For the half-step `t`: when f is given, X(r, o) *= f_r and Y(s, r) /= f_r (xmul) or
    // X /= f_r and Y *= f_r (written back); when Xk is given (float only), the bf16
    // operands of `t` (Y2tk may be null); when cpart is given, cpart[glue_parts(S)][R] =
    // per-block sums over s of the (scaled) y(s, r).
    static int scale_ops(const View& t, const double* f, bool xmul, void* Xk, void* Yk,
                         void* Ytk, void* Y2tk, int64_t rp, int64_t O_pad, int64_t S_pad,
                         int64_t plane, double* cpart, cudaStream_t st);
    static int64_t glue_parts(int64_t n);   // partial sums per R of the fused glue
    // out[r] = sum over k < nparts of part[k * R + r] (fixed order; no regularisation and
    // no replacement of a zero sum: the column sums c0 of Y that sum_s z needs)
    static int raw_sums(const double* part, int64_t nparts, int64_t R, double* out,
                        cudaStream_t st);
    // Sparse-V form (sparse_kernels.cuh): the view's non-zero k is at s = idx[k] with value
    // val[k], grouped in segments `sg`; Yg is Y as S x R row-major; R <= 128.  Each call is a
    // segment kernel (partials Aseg, Bseg [nseg][R] or dseg) and a per-column reduction.
    static int sp_pass1(const View& v, const SparseSegs& sg, const int32_t* idx, const Tp* val,
                        const Tp* Yg, Tp* Aseg, Tp* Bseg, Tp* A, Tp* B, bool with_b,
                        int* status, cudaStream_t st);
    static int sp_pass2(const View& v, const SparseSegs& sg, const int32_t* idx, const Tp* val,
                        const Tp* Yg, const Tp* Xmu, const Tp* Xdna, const double* c0,
                        double* dseg, double* dpart, int* status, cudaStream_t st);
    static int sp_kl(const View& v, const SparseSegs& sg, const int32_t* idx, const Tp* val,
                     const Tp* Yg, const double* c0, double* dseg, double* part, int* status,
                     cudaStream_t st);
    // out (cols x rows) = in^t (rows x cols), both row-major
    static int transpose(const Tp* in, int64_t rows, int64_t cols, Tp* out, cudaStream_t st);
    // one-time: row and column sums of V (float64) and the transposed copy; with Vc (needs
    // part) also a copy of V into Vc [N][T] in the same pass (V may be pinned host memory)
    static int prepare_v(const Tp* V, int64_t N, int64_t T, int64_t ldv, Tp* Vt, int64_t ldvt,
                         double* colsum, double* rowsum, cudaStream_t st,
                         double* part = nullptr, Tp* Vc = nullptr);
    // how many CTAs of pass 1 / pass 2 fit on one SM
    static int pass1_blocks_per_sm(int64_t R);
    static int pass2_blocks_per_sm(int64_t R);
    static int chunk();   // the s-chunk of passes 1 and 2 (splits are multiples of it)
    static int oblock();  // the o-block of passes 1 and 2
    static int rblock(int64_t R);  // the r-block of pass 1
};

// Tensor-core (tcgen05) operands of one half-step, bf16, zero-padded:
//   Xk [O_pad][RP]  x(r, o) K-major (GEMM1 A)      Yk   [S_pad][RP] y(s, r) (GEMM1 B)
//   Ytk [RP][S_pad] y(s, r) transposed (GEMM2 B)   Y2tk [RP][S_pad] y(s, r)^2 (GEMM3 B)
struct TcOperands {
    int64_t S, O, R, S_pad, O_pad;
    const void* Xk;
    const void* Yk;
    const void* Ytk;
    const void* Y2tk;
    const void* Xmk;    // bf16 candidates [O_pad][RP] (pass 2)
    const void* Xdk;
    const float* V;     // V_so as the passes read it, element (s, o) at V[s * vs + o]
    int64_t vs;
    // FP32 form on the tensor cores: every operand buffer holds a hi plane and, `plane`
    // elements after it, a lo plane (x = hi + lo, both bf16); 0 in the BF16 form
    int64_t plane;
    int ctas;   // CTAs of the persistent kernels (the SM count)
    // pass 1 at RP > 128: bf16 workspace rows Q[o][s], Qbar[o][s] ([O_pad][ldq], ldq a
    // multiple of 128) written by the ratios kernel of pass 1 and read by its contraction;
    // in the FP32 form a lo plane follows each, qplane elements after its hi plane
    void* Qg;
    void* Qbg;
    int64_t ldq;
    int64_t qplane;
    int64_t ldt;   // row stride of Ytk, Y2tk in elements (0: S_pad)
};

// TMA descriptors of one half-step view (built once per bound problem).
struct TcMaps {
    CUtensorMap x, y, yt, y2t, v, xm, xd;
    CUtensorMap q, qb;                                 // Q, Qbar workspace (RP > 128)
    CUtensorMap y128, yt256, y2t256;                   // larger boxes of Y, Yt, Y2t (RP > 128)
    CUtensorMap x_l, y_l, yt_l, y2t_l, xm_l, xd_l;   // lo planes (FP32 form, tensor cores)
    CUtensorMap q_l, qb_l, y128_l, yt256_l, y2t256_l;  // lo planes, FP32 form at RP > 128
};

// One view (0: H step, 1: W step) of one problem of the grouped BF16 form on the tensor
// cores: the device table the grouped kernels read (tensor maps in global memory).
struct alignas(64) TcGView {
    CUtensorMap y, yt, y2t, v, xm, xd;
    int64_t S, O, R, S_pad, O_pad;
    const float* X;                 // the view's factors (float32 masters): x(r, o) at
    int64_t xr, xo;                 // X[r xr + o xo], y(s, r) at Y[s ys + r yr]
    const float* Y;
    int64_t ys, yr;
    void* Xk;                       // bf16 operands: Xk, Xmk, Xdk [O_pad][64],
    void* Yk;                       // Yk [S_pad][64], Ytk, Y2tk [64][S_pad]
    void* Ytk;
    void* Y2tk;
    void* Xmk;
    void* Xdk;
    const float* Xmu;               // candidates [R][O] (float32)
    const float* Xdna;
    float* A;                       // pass-1 partials [splits][R][O]
    float* B;
    double* dpart;                  // pass-2 cost slots [slots][2][O]
    int64_t s_per1;                 // rows of s per pass-1 split (a multiple of 64)
    int64_t nch2, U2;               // pass 2: chunks of 128 per o-block, (o-block, chunk) units
    int slots2;                     // pass-2 cost slots per column
    int64_t ldt;                    // row stride of Ytk, Y2tk (the same for both views)
};

struct TcBf16 {
    // padded rank for the tensor-core kernels (64, 128, 256 or 512), 0 if unsupported
    static int rank_pad(int64_t R);
    // dst[i][j] = bf16(src(i, j)) (or its square), zero-padded to rows_pad x cols_pad
    static int to_bf16(const float* src, int64_t si, int64_t sj, int64_t rows, int64_t cols,
                       void* dst, int64_t ld, int64_t rows_pad, int64_t cols_pad, bool square,
                       cudaStream_t st);
    // Yk, Ytk and (if with_sq) Y2tk of `op` from y(s, r) = Y[s * ys + r * yr] in one pass
    static int y_operands(const float* Y, int64_t ys, int64_t yr, const TcOperands& op,
                          bool with_sq, cudaStream_t st);
    // TMA descriptors for the operand buffers of `op`, V_so (leading dimension vs floats,
    // 16-byte aligned rows) and the bf16 candidates Xmk, Xdk ([O_pad][RP])
    static int make_maps(TcMaps* m, const TcOperands& op, const float* V, int64_t vs,
                         const void* Xmk, const void* Xdk);
    static int pass1(const TcOperands& op, const TcMaps& maps, float* Apart, float* Bpart,
                     int splits, int64_t s_per, bool with_b, int* status, cudaStream_t st);
    // pass 1 at padded rank 256 or 512 (tc_ks.cu): persistent CTAs over (r-block of 128,
    // o-block, split) tiles; s_per must be a multiple of 128
    // pass 1 at RP in {256, 512} as two kernels (tc_mat.cu): Z once per (o-block, chunk) with
    // q, qbar written to the Q, Qbar workspace, then the dual GEMM over 256-wide r-blocks;
    // Apart/Bpart [splits][R][O] with splits = ceil(S / s_per), s_per a multiple of 64
    static int pass1_mat(const TcOperands& op, const TcMaps& maps, float* Apart, float* Bpart,
                         int splits, int64_t s_per, bool with_b, int* status, cudaStream_t st);
    // pass 2 at padded rank 512, and of the split form at 256 and 512 (tc_ks.cu):
    // persistent CTAs over (o-block, split) tiles, s_per a multiple of 128, cost slots
    // dpart[4 splits][2][O]
    static int pass2_large(const TcOperands& op, const TcMaps& maps, double* dpart, int slots,
                           int64_t s_per, int* status, cudaStream_t st);
    // The FP32 form on the tensor cores (tc_split.cu): the same passes with every operand
    // split into hi + lo bf16 planes and three MMAs per product.  Pass 1 runs 2 x splits
    // CTA rows (A and B accumulated by separate CTAs; with_b = false: A only).
    static int pass1_split(const TcOperands& op, const TcMaps& maps, float* Apart,
                           float* Bpart, int splits, int64_t s_per, bool with_b, int* status,
                           cudaStream_t st);
    // pass 1 of the split form at RP in {256, 512} (tc_mats.cu): the ratios kernel writes
    // the hi / lo planes of Q, Qbar, then the contraction accumulates A (and B) per split;
    // s_per a multiple of 64 and at most 1024
    static int pass1_mats(const TcOperands& op, const TcMaps& maps, float* Apart, float* Bpart,
                          int splits, int64_t s_per, bool with_b, int* status, cudaStream_t st);
    // pass 2 of the split form (RP <= 128) and of the BF16 form (RP <= 256)
    static int pass2_split(const TcOperands& op, const TcMaps& maps, double* dpart, int slots,
                           int* status, cudaStream_t st);
    // cost slots per column that pass2_split writes (4 per CTA that an o-block spans)
    static int pass2_split_slots(int64_t O_pad, int64_t S, int ctas);
    // d_KL per column of the view (eq. 1 terms) from the X and Y operands in the split
    // form: dpart[slot][O], `slots` = pass2_split_slots of the view
    static int kl_split(const TcOperands& op, const TcMaps& maps, double* dpart, int slots,
                        int* status, cudaStream_t st);
    static int chunk();
    static int oblock();
    // The grouped BF16 form (R <= 64, padded rank 64), tables in device memory.
    // Operands of view w: tiles (problem, 0 | 1 (X | Y), block of 64, -) of k_g_operands.
    static int group_operands(const TcGView* gv, const void* tiles, int n, int w, int grid,
                              cudaStream_t st);
    // pass 1: `ctas` persistent CTAs over the tiles (problem, o-block, split), CTA i taking
    // tiles i, i + ctas, ...
    static int group_pass1(const TcGView* gv, const void* tiles, int n, int w, bool with_b,
                           int ctas, int* status, cudaStream_t st);
    // pass 2: one CTA per entry (problem, rank, CTAs of that problem)
    static int group_pass2(const TcGView* gv, const void* ctas, int n, int w, int* status,
                           cudaStream_t st);
    // once per group, before any launch (and outside graph capture): kernel attributes
    static int group_prepare();
    static int group_prepare_pass2();
    // one CTA whose bounded wait on a barrier that nothing completes gives up after
    // `limit` SM cycles and sets STATUS_TIMEOUT in *status
    static int check_wait_timeout(long long limit, int* status, cudaStream_t st);
};

// sum of part[0 .. n) into *out in a fixed order (work: REDUCE_PARTS doubles)
constexpr int64_t REDUCE_PARTS = 256;
int reduce_sum(const double* part, int64_t n, double* out, double* work, cudaStream_t st);

}  // namespace dna
