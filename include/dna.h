/*
 * dna.h - C ABI of the GB300 (sm_103a) library for the Diagonalized Newton Algorithm
 * (DNA) for KL-divergence NMF (H. Van hamme, "The Diagonalized Newton Algorithm for
 * Non-negative Matrix Factorization", arXiv 1301.3389).
 *
 * Problem (Section 1, eq. 1): factor a non-negative N x T matrix V as W H with W
 * (N x R) and H (R x T) non-negative, minimising
 *     d_KL(V, WH) = sum v log(v / z) - sum v + sum z,   Z = W H.
 * One DNA iteration (Algorithm 1) updates H with W fixed (steps 4-16), then W with H
 * fixed (steps 17-29).  Each half-step forms the MU candidate (eq. 11) and the
 * diagonal-Newton candidate (eq. 15 / 17 with the step limits of Section 2.3 and the
 * eq. 10 renormalisation), evaluates both costs per column of H (per row of W) and
 * keeps the cheaper one (Section 2.4).
 *
 * Layout: every matrix is dense and row-major.  V is N x T with leading dimension
 * ldv >= T; W is N x R with leading dimension R; H is R x T with leading dimension T.
 * Element type: double for DNA_F64, float for DNA_F32 and DNA_BF16 (the BF16 form
 * keeps float masters and rounds only tensor-core operands to bfloat16).
 *
 * Ownership: the caller owns V, W and H (device memory) and the CUDA stream.  The
 * library owns a context and its device workspace, allocated by dna_create/dna_bind
 * and released by dna_destroy; the step calls allocate nothing and never synchronise
 * the host.  W and H are updated in place.
 *
 * Errors: every int-returning call returns DNA_OK (0) or a negative DNA_ERR_* code.
 * Argument errors are detected on the host before any work is queued.  Errors found by
 * kernels (a non-positive z where v > 0, which makes the cost infinite) are recorded in
 * a device status word and returned by the next synchronising call (dna_kl,
 * dna_get_status, dna_get_choice, dna_get_costs, dna_run_host).
 */
#ifndef DNA_H_
#define DNA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DNA_OK               0
#define DNA_ERR_ARG         (-1)  /* bad argument (size, pointer, option, call order) */
#define DNA_ERR_CUDA        (-2)  /* a CUDA runtime call or kernel launch failed       */
#define DNA_ERR_NONFINITE   (-3)  /* z <= 0 where v > 0, or a non-finite value          */
#define DNA_ERR_TIMEOUT     (-4)  /* a bounded device-side wait gave up                 */
#define DNA_ERR_UNSUPPORTED (-5)  /* valid request this build does not implement       */
#define DNA_ERR_ALLOC       (-6)  /* device allocation failed                           */
#define DNA_ERR_LIMIT       (-7)  /* size beyond a fixed limit of dna_kl_noalloc         */

/* Arithmetic forms. */
#define DNA_F64  0  /* float64 everywhere                                                */
#define DNA_F32  1  /* float32 everywhere, float64 per-column cost sums                  */
#define DNA_BF16 2  /* bfloat16 tensor-core operands, float32 accumulation and masters,
                       float64 per-column cost sums                                      */

/* Engines for the O(NRT) contractions.  AUTO: BF16 on the tensor cores, F32 and F64 on
 * the CUDA cores.  TENSOR with F32 (R <= 512): every float32 operand x is split into
 * bf16 x_hi = bf16(x) and x_lo = bf16(x - x_hi) and every product is formed as
 * x_hi y_hi + x_hi y_lo + x_lo y_hi with float32 accumulation (relative error per product
 * below about 2^-15); dna_step_H_fixed, dna_step_H_adjoint and dna_kl_backward need the
 * SIMT engine. */
#define DNA_ENGINE_AUTO   0
#define DNA_ENGINE_SIMT   1  /* CUDA-core FMA kernels (F64, F32)                          */
#define DNA_ENGINE_TENSOR 2  /* tcgen05 tensor-core kernels with TMEM accumulators         */

typedef struct dna_opts {
    double eps;     /* floor on the Newton gain for a < 0 (Algorithm 1 steps 11, 24);
                       default 0.01 (Section 4)                                          */
    double alpha;   /* the gain of the a >= 0 step is capped at 1 + alpha (Section 2.3,
                       eq. 17); default 4 (Section 4)                                    */
    double rho;     /* regularisation weight on W (eq. 2); default 0 (Section 4)         */
    double lambda;  /* regularisation weight on H (eq. 2); default 0 (Section 4)         */
    int32_t dtype;  /* DNA_F64, DNA_F32 or DNA_BF16; default DNA_F32                     */
    int32_t engine; /* DNA_ENGINE_*; default DNA_ENGINE_AUTO                             */
} dna_opts;

typedef struct dna_ctx dna_ctx;

/* Fill *opts with the defaults above (the parameters of Section 4). */
void dna_default_opts(dna_opts* opts);

/* Create a context for an N x T problem of rank R on the current CUDA device.
 * opts may be NULL (defaults).  Sizes must satisfy N >= 1, T >= 1, 1 <= R <= 512.
 * Allocates the workspace (O(N T) for the transposed copy of V made by dna_bind, plus
 * O((N + T) R)).  On success *out receives the context. */
int dna_create(int64_t N, int64_t T, int64_t R, const dna_opts* opts, dna_ctx** out);

/* Attach the caller's device buffers: V (N x T, leading dimension ldv >= T, read only),
 * W (N x R) and H (R x T), all of the context's element type.  Queues, on the
 * context's stream, the one-time preparation that depends on V (row and column sums of
 * V, and the transposed copy used by the W half-step).  V must not change while bound. */
int dna_bind(dna_ctx* ctx, const void* V, int64_t ldv, void* W, void* H);

/* ---------------------------------------------------------------- sparse-V form
 * The paper's sparse workloads (Section 4.2; the note after Algorithm 1 on zeros in V):
 * V is given in CSR and every O(NRT) step touches only its non-zeros.  z is formed at the
 * non-zeros only; q = v / z and v / z^2 vanish at the zeros, so A and B (eq. 7, 14) and the
 * -v log z part of the candidates' costs (steps 9, 14) are sums over the non-zeros, and
 * sum_n z_nt = sum_r (sum_n w_nr) h_rt needs no zeros either.  Candidates, selection and
 * normalisation are those of the dense form.  F32 and F64 forms on the CUDA cores,
 * R <= 128.  A context made by dna_create_sparse is bound with dna_bind_csr (not
 * dna_bind) and takes dna_normalize, dna_step_H, dna_step_W, dna_iterate, mu_step,
 * mu_iterate, dna_kl, dna_get_choice, dna_get_costs, dna_get_status; the other calls
 * return DNA_ERR_UNSUPPORTED. */

/* Create a sparse-V context for an N x T matrix V with nnz stored entries, rank R
 * (1 <= R <= 128), F32 or F64 (BF16 or the tensor engine: DNA_ERR_UNSUPPORTED).
 * Allocates O(nnz + (N + T) R) of workspace. */
int dna_create_sparse(int64_t N, int64_t T, int64_t R, int64_t nnz, const dna_opts* opts,
                      dna_ctx** out);

/* Attach V in CSR form and the factors, all device memory owned by the caller and kept
 * unchanged while bound: row_ptr (N + 1 int64, row_ptr[0] = 0, non-decreasing,
 * row_ptr[N] = nnz), col_idx (nnz int32 in [0, T), any order within a row), vals (nnz
 * values >= 0 of the context's element type; explicit zeros allowed), W (N x R) and H
 * (R x T).  Copies the structure to the host once, checks it (DNA_ERR_ARG if it is not a
 * valid CSR of an N x T matrix with non-negative values), builds the library's CSC copy
 * (the H half-step's view, rows ascending within a column) and the row and column sums of
 * V.  Synchronises the context's stream. */
int dna_bind_csr(dna_ctx* ctx, const int64_t* row_ptr, const int32_t* col_idx,
                 const void* vals, void* W, void* H);

/* Set the CUDA stream (a cudaStream_t; NULL = legacy default stream) for later calls. */
int dna_set_stream(dna_ctx* ctx, void* stream);

/* Normalisation of Algorithm 1.  which = 1: steps 1 and 29, divide column r of W by
 * sum_n w_nr + lambda and multiply row r of H by the same number.  which = 0: step 16,
 * divide row r of H by sum_t h_rt + rho and multiply column r of W.  W H is unchanged. */
int dna_normalize(dna_ctx* ctx, int which);

/* DNA H half-step, Algorithm 1 steps 4-16 (eq. 7, 10, 11, 14, 15, 17; Section 2.4),
 * with W fixed: H <- per column the lower-cost of the MU and Newton candidates, then
 * the step-16 normalisation (which also rescales the columns of W).  Asynchronous. */
int dna_step_H(dna_ctx* ctx);

/* DNA W half-step, Algorithm 1 steps 17-29: the mirror of dna_step_H by the symmetry
 * d_KL(V, WH) = d_KL(V^t, H^t W^t) (Section 2), selection per row of W, then the
 * step-29 normalisation (which also rescales the rows of H).  Asynchronous. */
int dna_step_W(dna_ctx* ctx);

/* iters DNA iterations: iters times (dna_step_H, dna_step_W).  Asynchronous. */
int dna_iterate(dna_ctx* ctx, int iters);

/* enable != 0: dna_iterate forms the first H half-step's operands and denominators from the
 * current factors, then replays one captured iteration (a CUDA graph, captured on the first
 * such call and kept until the next dna_bind, selection change or change of the profiled
 * phases) iters times; W and H are bit-identical to the direct launches.  Profiled phases
 * of the captured iteration are timed by events recorded inside the graph: dna_phase_times
 * counts each replay with the times of the last one.  Used only with a stream set by
 * dna_set_stream (not the legacy default stream) and dense V; otherwise dna_iterate
 * launches directly.  Default: off. */
int dna_use_graph(dna_ctx* ctx, int enable);

/* Multiplicative update (eq. 11; Algorithm 1 "MU" steps).  which = 0: H <- H (W^t Q) /
 * (W^t 1 + lambda) then step 16; which = 1: W <- W (Q H^t) / (H 1 + rho) then step 29.
 * Asynchronous. */
int mu_step(dna_ctx* ctx, int which);

/* iters MU iterations: iters times (mu_step(ctx, 0), mu_step(ctx, 1)), each half-step
 * leaving the operands of the next one ready (as dna_iterate does).  Asynchronous. */
int mu_iterate(dna_ctx* ctx, int iters);

/* d_KL(V, W H) of eq. 1 in float64, written to *out (host memory): per element
 * z + v log(v / z) - v (z where v = 0), summed in float32 over short runs and in float64
 * beyond.  Z is formed by the context's engine (for F32 with ENGINE_TENSOR: the split
 * bf16 tensor-core product; for BF16: the CUDA-core float32 product).  Synchronises the
 * context's stream; also returns any error recorded by earlier kernels. */
int dna_kl(dna_ctx* ctx, double* out);

/* Gradient of d_KL(V, W H) (eq. 1) with respect to W, H and V, times `scale` (the
 * incoming gradient of a loss), into caller-owned device buffers of the context's element
 * type (any of them may be NULL): dW (N x R) = (1 - Q) H^t, dH (R x T) = W^t (1 - Q) (the
 * KKT gradient of eq. 6 with lambda = 0), dV (N x T, leading dimension T) = log(V / Z)
 * where v > 0 and 0 where v = 0 (the derivative of v log(v / z) - v, taken as 0 at
 * v = 0), with Q = V / Z and Z = W H.  F32 and F64 forms.  Asynchronous; uses the
 * context's workspace (so it must not overlap other calls on the same context). */
int dna_kl_backward(dna_ctx* ctx, double scale, void* dW, void* dH, void* dV);

/* ---------------------------------------------------------------- differentiation
 * An unrolled DNA solve for H at fixed W (the H half-step without the step-16
 * normalisation, repeated), and the adjoint of one such step for reverse-mode
 * differentiation.  F32 and F64 forms; the adjoint needs R <= 128 (F32) or 64 (F64). */

/* One H half-step at fixed W: Algorithm 1 steps 4-15 (eq. 7, 10, 11, 14, 15, 17 and the
 * selection of Section 2.4), without step 16, so W is not modified.  If choice_out (device
 * memory, T bytes) is not NULL it receives the per-column selection (1 = Newton).
 * Asynchronous. */
int dna_step_H_fixed(dna_ctx* ctx, uint8_t* choice_out);

/* Adjoint of dna_step_H_fixed at the state Hk (R x T, device) with the selection `choice`
 * (T bytes, device) that the forward step made (held fixed: the map is piecewise smooth
 * and the selection, the eps floor and the alpha cap are treated as locally constant):
 * given Hbar_next = dL/dH_{k+1} (R x T) writes Hbar_out = dL/dH_k (R x T) and ADDS dL/dV
 * into Vbar (N x T, leading dimension T).  W is treated as a constant.  Uses the context's
 * bound V and W.  Asynchronous. */
int dna_step_H_adjoint(dna_ctx* ctx, const void* Hk, const uint8_t* choice,
                       const void* Hbar_next, void* Hbar_out, void* Vbar);

/* dna_step_H_adjoint with W a variable of the step as well: as above, and ADDS dL/dW of the
 * step into Wbar (N x R, row-major like W): the paths through Z = W H (hence Q = V / Z and
 * Qbar = V / Z^2), through A = W^t Q and B = (W o W)^t Qbar of eq. 7 and 14, and through
 * the column sums c = W^t 1 + lambda that divide them (eq. 7) and weight the eq. 10
 * renormalisation.  Summed over the steps of an unrolled solve (plus the loss's own
 * derivative in W, e.g. dna_kl_backward's dW) this is the gradient of the loss with
 * respect to W.  Vbar and Wbar may each be NULL (the other outputs are still written).
 * The first call with Wbar allocates the context's W-gradient workspace (at most
 * 32 x R x N values of the element type and ceil(T / 32) x R float64); later calls
 * allocate nothing.  Same limits on R as dna_step_H_adjoint. Returns DNA_ERR_ALLOC if the
 * workspace cannot be allocated.
 * Asynchronous. */
int dna_step_H_adjoint_w(dna_ctx* ctx, const void* Hk, const uint8_t* choice,
                         const void* Hbar_next, void* Hbar_out, void* Vbar, void* Wbar);

/* Selection rules (dna_set_selection).  PAPER: Section 2.4 and Algorithm 1 steps 15 / 28,
 * the Newton candidate is kept iff its cost is below the MU candidate's (both costs are
 * evaluated).  DESCENT: the Newton candidate is kept iff its eq. 5 (eq. 4) cost is below
 * that of the column (row) the half-step starts from, else the MU candidate.  MU never
 * increases the eq. 5 cost (Section 2.1), so the cost still never increases, but only the
 * Newton candidate's cost is evaluated: pass 1 accumulates the starting column's cost from
 * the z it forms anyway, and pass 2 forms one candidate's z instead of two (Section 5
 * names step damping that avoids cost evaluations as a way to speed DNA up).  Every column
 * that PAPER gives to Newton, DESCENT does too. */
#define DNA_SELECT_PAPER   0
#define DNA_SELECT_DESCENT 1

/* Choose the selection rule of later DNA half-steps (default PAPER).  DESCENT needs the
 * CUDA-core engine (F32 or F64, dense V; else DNA_ERR_UNSUPPORTED) and allocates its cost
 * buffer on first use.  With DESCENT, dna_get_costs gives (starting cost, Newton cost). */
int dna_set_selection(dna_ctx* ctx, int mode);

/* Copy the selection of the last DNA half-step to host memory: which = 0 gives T bytes
 * (column t of H took the Newton candidate iff out[t] = 1), which = 1 gives N bytes (per
 * row of W).  len must equal T (N).  Synchronises. */
int dna_get_choice(dna_ctx* ctx, int which, uint8_t* out, int64_t len);

/* Copy the per-column (which = 0, T values) or per-row (which = 1, N values) costs of
 * the two candidates of the last DNA half-step to host memory:
 * d = sum_{v>0} (-v log z) + sum z + lambda sum_r h_r over that column (per row:
 * + rho sum_r w_r), i.e. the eq. 5 (eq. 4) sub-problem cost with the
 * candidate-independent constant sum v log v - sum v dropped (Algorithm 1 steps 9, 14,
 * 22, 27).  The selection keeps the Newton candidate iff its d is lower.  Synchronises. */
int dna_get_costs(dna_ctx* ctx, int which, double* d_mu, double* d_dna, int64_t len);

/* Synchronise the stream and return the sticky device status (DNA_OK or an error). */
int dna_get_status(dna_ctx* ctx);

/* End-to-end call on HOST buffers: copy V (N x T, ldv = T), W and H from host memory
 * to library-owned device buffers (allocated on the first call and reused), run
 * iters DNA iterations, copy W and H back and write d_KL(V, WH) to *kl_out (may be
 * NULL).  Pinned host memory gives the fastest copies: a V in pinned (device-mapped)
 * memory is read across the host link by the kernel that forms V's transpose and sums,
 * which writes the device copy in the same pass; other host memory is copied first.
 * Synchronises.  A context used this way must not also be bound with dna_bind. */
int dna_run_host(dna_ctx* ctx, const void* V, void* W, void* H, int iters, double* kl_out);

/* Phases of a half-step, for dna_phase_times. */
#define DNA_PHASE_PASS1      0  /* Z, Q, Qbar and the A, B contractions (steps 2-5, 10)  */
#define DNA_PHASE_CANDIDATES 1  /* MU and Newton candidates, eq. 10 (steps 6, 11)       */
#define DNA_PHASE_PASS2      2  /* candidate costs (steps 7-9, 12-14)                    */
#define DNA_PHASE_SELECT     3  /* per-column selection (step 15)                        */
#define DNA_PHASE_SUMS       4  /* factor sums and rescaling (steps 1, 16, 29)           */
#define DNA_PHASE_KL         5  /* d_KL (eq. 1)                                           */
#define DNA_PHASE_PREPARE    6  /* one-time sums and transpose of V (dna_bind)           */
#define DNA_PHASE_OPERANDS   7  /* bf16 tensor-core operand tiles (BF16 form)            */
#define DNA_NUM_PHASES       8

/* enable = 1: from now on record a CUDA event pair on the context's stream around each
 * phase of every call (no device allocation; up to 16384 pairs are kept, later phases
 * are counted but not timed); enable = 0 stops recording.  Launch counts are always
 * kept. */
int dna_profile(dna_ctx* ctx, int enable);

/* As dna_profile, for the phases whose bit (1u << phase) is set in mask only (mask = 0
 * stops recording).  Timing fewer phases adds fewer events to the stream. */
int dna_profile_phases(dna_ctx* ctx, unsigned mask);

/* Write, for each of the first n phases, the summed device time in milliseconds of the
 * recorded phase instances (ms, may be NULL) and the number of kernel launches of that
 * phase (launches, may be NULL) since the previous call, then reset both.
 * Synchronises the stream. */
int dna_phase_times(dna_ctx* ctx, double* ms, int64_t* launches, int n);

/* ---------------------------------------------------------------- batching form
 * Many independent KL-NMF problems of uneven sizes (count of them; problem q is
 * N[q] x T[q] of rank R[q] <= 64), FP32 or BF16 form.  Each phase of a DNA half-step runs
 * for all problems in one grouped launch (a tile list over (problem, block, split)), and
 * dna_group_iterate can replay one whole iteration as a captured CUDA graph.  FP32: every
 * phase on the CUDA cores.  BF16: the two O(NRT) passes on the tensor cores (the
 * single-problem BF16 kernels at padded rank 64, each problem's operands and tensor maps
 * in a device table), bf16 operands written by grouped conversion kernels, the rest as in
 * FP32.  Every problem follows exactly the single-problem algorithm above (Algorithm 1);
 * only the order of the split sums may differ.  The group owns a private stream that is
 * ordered after and before the caller's stream on every call. */
typedef struct dna_group dna_group;

/* Create a group of `count` problems with sizes N[q], T[q], R[q] (host arrays); opts may
 * be NULL.  DNA_F32 (CUDA-core engine) and DNA_BF16 (tensor-core passes) are supported;
 * R[q] > 64, DNA_F64, F32 on the tensor engine or BF16 on the SIMT engine give
 * DNA_ERR_UNSUPPORTED.  Allocates the whole workspace at once (BF16 adds an aligned copy
 * of each V and the bf16 operands). */
int dna_group_create(int count, const int64_t* N, const int64_t* T, const int64_t* R,
                     const dna_opts* opts, dna_group** out);

/* Attach the caller's device buffers: host arrays of `count` device pointers V[q]
 * (N[q] x T[q], leading dimension ldv[q] >= T[q]; ldv may be NULL for ldv[q] = T[q]),
 * W[q] (N[q] x R[q]) and H[q] (R[q] x T[q]), float32.  Queues the one-time sums and
 * transposes of every V. */
int dna_group_bind(dna_group* g, const void* const* V, const int64_t* ldv, void* const* W,
                   void* const* H);

/* Caller's stream (a cudaStream_t; NULL = legacy default stream). */
int dna_group_set_stream(dna_group* g, void* stream);

/* dna_normalize for every problem (which = 1: steps 1/29, which = 0: step 16). */
int dna_group_normalize(dna_group* g, int which);

/* dna_step_H / dna_step_W for every problem, one grouped launch per phase. */
int dna_group_step_H(dna_group* g);
int dna_group_step_W(dna_group* g);

/* iters DNA iterations of every problem; with dna_group_use_graph(g, 1) the first call
 * captures one iteration as a CUDA graph and every iteration replays it.  BF16 form: each
 * half-step's rescale (steps 16 / 29) also writes the bf16 operands of the half-step after
 * it, and each call first writes those of its first H half-step (one launch). */
int dna_group_iterate(dna_group* g, int iters);
int dna_group_use_graph(dna_group* g, int enable);

/* Autotuner: time `reps` iterations for each candidate tile configuration and keep the
 * fastest; W and H are restored afterwards.  Candidates: the split size (rows of s per
 * tile of the reductions) and, in the BF16 form, the pass-2 tile size ((o-block, chunk)
 * units per CTA, 4 to 128).  The chosen split size is written to *rows_out (may be NULL).
 * Synchronises. */
int dna_group_autotune(dna_group* g, int reps, int64_t* rows_out);

/* The tile configuration in use: rows of s per split and (BF16 form; 0 in FP32) pass-2
 * units per CTA.  Either pointer may be NULL. */
int dna_group_tile_config(dna_group* g, int64_t* split_rows, int64_t* p2_units);

/* d_KL (eq. 1) of every problem into out[0 .. count) (host).  Synchronises. */
int dna_group_kl(dna_group* g, double* out);

/* Synchronise and return the sticky status of the group's kernels. */
int dna_group_get_status(dna_group* g);

/* dna_get_choice for problem q of the group: the selection (Section 2.4, Algorithm 1
 * steps 15 / 28) of its last DNA half-step, 1 = Newton, per column of H (which = 0,
 * len = T[q]) or per row of W (which = 1, len = N[q]), copied to host memory.
 * Synchronises. */
int dna_group_get_choice(dna_group* g, int q, int which, uint8_t* out, int64_t len);

/* Kernel launches of one grouped iteration (both half-steps, as dna_group_iterate runs
 * them; in the BF16 form not counting the one operand launch per dna_group_iterate call). */
int64_t dna_group_launches_per_iteration(dna_group* g);

/* Release the group and its workspace. */
void dna_group_destroy(dna_group* g);

/* Capacity, in float64 partial sums, of the static scratch of dna_kl_noalloc. */
#define DNA_KL_NOALLOC_MAX_PARTIALS (1 << 20)

/* d_KL(V, W H), the value dna_kl returns, for callers that cannot allocate device
 * memory: code whose device memory is all owned by another framework's pool allocator,
 * and latency-critical code that cannot pay for cudaMalloc or the implicit device
 * synchronisation of cudaFree.  The paper has no counterpart of this entry point.
 *
 * Needs no context and allocates nothing: it calls no cudaMalloc, cudaFree or
 * allocating library routine.  Its scratch (a status word and per-column partial sums)
 * is one static device array of 256 + 8 * DNA_KL_NOALLOC_MAX_PARTIALS bytes (about
 * 8 MiB), which every GPU that loads this library holds until the process exits.
 * Inputs, float32 device memory, row-major: V (N x T, leading dimension ldv >= T), W
 * (N x R), H (R x T).  Output: *kl_out, one float64 in device memory owned by the caller,
 * written asynchronously on `stream` (a cudaStream_t; NULL = legacy default stream); it
 * is +infinity if some z <= 0 where v > 0.  Limits: 1 <= R <= 512 and
 * T <= DNA_KL_NOALLOC_MAX_PARTIALS, else DNA_ERR_LIMIT (T too large) or DNA_ERR_ARG,
 * returned before any work is queued.
 *
 * The first call on a device looks up the device address of the static array (with that
 * device current) and keeps it for later calls on that device; make that first call
 * before any stream capture.  The kept address belongs to the CUDA context current at
 * that first call (the device's primary context when the runtime API is used): callers
 * that switch that device to another driver context, or reset it, must not call this
 * entry point afterwards.  All calls share the one array: calls that overlap on the GPU
 * (for example on two unordered streams) race and give wrong results, so order them,
 * e.g. on one stream.  The partial sums (splits x T of them, splits <= 32) are added by a
 * single 1024-thread block at the end, a few microseconds for T in the thousands and up
 * to tens of microseconds near the capacity. */
int dna_kl_noalloc(const float* V, int64_t ldv, const float* W, const float* H, int64_t N,
                   int64_t T, int64_t R, double* kl_out, void* stream);

/* ---------------------------------------------------------------- column shards
 * One DNA iteration of a problem whose columns are split over G ranks (one GPU each): rank
 * g holds V[:, T_g] and H[:, T_g] (a column block) and a full copy of W, in an ordinary
 * dense context of size N x T_g (any form and engine; dna_normalize(ctx, 1) for step 1 as
 * usual, and dna_kl gives this block's share of d_KL, to be summed over the ranks).
 * The H half-step separates over columns (eq. 5); the W half-step and the normalisations
 * need sums over all columns.  The calls below run every step on this rank's block and
 * stop at each such sum: the caller adds the buffer a call wrote over the G ranks (an
 * all-reduce, e.g. NCCL through torch.distributed) and passes the total to the next call.
 * Every buffer is caller-owned device memory; float64 unless stated; every call is
 * asynchronous on the context's stream.  With G = 1 (no reduction) the sequence equals
 * dna_step_H then dna_step_W.
 *
 * Once after dna_bind:
 *   dna_shard_rowsums(out[N]) -> all-reduce -> dna_shard_set_rowsums(total)
 *   (the row sums of V, the eq. 10 targets of the W half-step)
 * H half-step (Algorithm 1 steps 4-16):
 *   dna_shard_H_begin(rsum[R]) -> all-reduce -> dna_shard_H_end(rsum)
 * W half-step (steps 17-29):
 *   dna_shard_W_begin(hsum[R]) -> all-reduce -> dna_shard_W_pass1(hsum, AB[2][R][N], the
 *   context's element type) -> all-reduce AB -> dna_shard_W_pass2(AB, cost[2][N]) ->
 *   all-reduce -> dna_shard_W_end(cost)
 * Sparse and host-buffer contexts: DNA_ERR_UNSUPPORTED. */

/* out[n] = sum over this block's columns of v_nt. */
int dna_shard_rowsums(dna_ctx* ctx, double* out);
/* Set the row sums of V over all columns (the eq. 10 targets of the W half-step). */
int dna_shard_set_rowsums(dna_ctx* ctx, const double* in);
/* Steps 4-15 on this block's columns (each column's selection is local, eq. 5), then
 * rsum[r] = sum over this block of the new h_rt (step 16's sums before rho). */
int dna_shard_H_begin(dna_ctx* ctx, double* rsum);
/* Step 16 with the all-reduced rsum: row r of H divided, column r of W multiplied, by
 * rsum[r] + rho (identical on every rank). */
int dna_shard_H_end(dna_ctx* ctx, const double* rsum);
/* Operands of the W half-step; hsum[r] = sum over this block of h_rt (the eq. 7 / 14
 * denominators of the W half-step before rho). */
int dna_shard_W_begin(dna_ctx* ctx, double* hsum);
/* With the all-reduced hsum: the raw sums over this block's columns of eq. 7 and 14,
 * AB[0][r][n] = sum_t q_nt h_rt and AB[1][r][n] = sum_t qbar_nt h_rt^2 (steps 18, 23). */
int dna_shard_W_pass1(dna_ctx* ctx, const double* hsum, void* AB);
/* With the all-reduced AB: both candidates per row of W (steps 19, 24; identical on every
 * rank) and their costs over this block's columns, cost[0][n] (MU) and cost[1][n]
 * (Newton), each sum_t (-v log z + z) (steps 20-22, 25-27). */
int dna_shard_W_pass2(dna_ctx* ctx, const void* AB, double* cost);
/* With the all-reduced costs: the selection per row (step 28, the rho penalty added as in
 * dna_step_W) and step 29 (W's column sums are local: W is replicated). */
int dna_shard_W_end(dna_ctx* ctx, const double* cost);

/* Failure detection of the device-side waits: every barrier wait of the tensor-core kernels
 * is bounded (about 2 s of SM cycles); when one gives up, the kernel raises an abort flag
 * that its other warps see, waits (bounded) for its own copies and MMAs in flight, frees
 * its tensor memory and returns, and the next synchronising call reports
 * DNA_ERR_TIMEOUT.  This call runs that path on one CTA whose wait, limited to
 * limit_cycles (1 .. 2^32) SM cycles, is on a barrier phase that nothing completes (no
 * copy or MMA is in flight), on the legacy default stream, and returns DNA_ERR_TIMEOUT
 * when the timeout was detected and reported (DNA_OK would mean it was not).
 * Synchronises; allocates and frees one int of device memory. */
int dna_check_wait_timeout(int64_t limit_cycles);

/* Release the context and its workspace (not the caller's buffers). */
void dna_destroy(dna_ctx* ctx);

/* Static English description of a status code. */
const char* dna_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* DNA_H_ */
