// C ABI of the DNA library: context, workspace, and the order of kernel launches for
// each call of include/dna.h.  Host code only; kernels live in simt_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "dna.h"
#include "dna_internal.h"

using dna::View;

struct dna_ctx {
    int64_t N = 0, T = 0, R = 0;
    dna_opts o{};
    int device = 0;
    int num_sms = 1;
    cudaStream_t stream = nullptr;
    size_t esz = 4;
    // caller's buffers
    const void* V = nullptr;
    int64_t ldv = 0;
    void* W = nullptr;
    void* H = nullptr;
    bool bound = false;
    bool host_mode = false;  // buffers owned by the library (dna_run_host)
    void* own_V = nullptr;
    void* own_W = nullptr;
    void* own_H = nullptr;
    // workspace
    void* Vt = nullptr;  // T x ldvt transposed copy of V
    int64_t ldvt = 0;
    double* colsum_v = nullptr;  // T
    double* rowsum_v = nullptr;  // N
    double* c = nullptr;         // R
    double* sig = nullptr;       // R
    double* fwork = nullptr;     // FSUM_SPLITS * R partial factor sums
    double* gpart = nullptr;     // [ceil(max(N, T) / 32)][R] partial sums of the fused glue
    double* vpart = nullptr;     // per-tile column and row sums of V (prepare)
    void* Apart = nullptr;       // [splits][R][O]
    void* Bpart = nullptr;
    void* Xmu = nullptr;         // [R][O]
    void* Xdna = nullptr;
    double* dpart = nullptr;     // [splits][2][O]
    double* dfin_h = nullptr;    // [2][T]
    double* dfin_w = nullptr;    // [2][N]
    uint8_t* choice_h = nullptr; // T
    uint8_t* choice_w = nullptr; // N
    double* kl_dev = nullptr;    // 1
    double* kl_part = nullptr;   // REDUCE_PARTS partial sums of d_KL
    int* status = nullptr;       // 1
    // split plans (pass 1 and pass 2 / KL) for the H view and the W view
    int sp1[2] = {1, 1}, sp2[2] = {1, 1};
    int64_t per1[2] = {0, 0}, per2[2] = {0, 0};
    // tensor-core (BF16) path
    bool tc = false;
    bool split = false;              // FP32 form on the tensor cores (hi + lo bf16 operands)
    int64_t qplane = 0;              // lo plane offset of the Q, Qbar workspace (split, RP > 128)
    int64_t plane = 0;               // elements between the hi and lo planes of each operand
    int rp = 0;                      // padded rank
    int64_t pad_o[2] = {0, 0};       // O_pad of the H view (0) and W view (1)
    int64_t pad_s[2] = {0, 0};       // S_pad
    void* Xk = nullptr;              // bf16 [max O_pad][rp]
    void* Yk = nullptr;              // bf16 [max S_pad][rp]
    void* Ytk = nullptr;             // bf16 [rp][max S_pad]
    void* Y2tk = nullptr;
    void* Xmk = nullptr;             // bf16 [max O_pad][rp]
    void* Xdk = nullptr;
    void* Qg = nullptr;              // BF16 form at RP > 128: Q, Qbar rows [max O_pad][ldq]
    void* Qbg = nullptr;
    int64_t ldq[2] = {0, 0};         // of the H view (0) and W view (1)
    void* Vp = nullptr;              // aligned copy of V when V's rows are not 16-byte aligned
    int64_t ldvp = 0;
    dna::TcMaps maps[2];             // TMA descriptors of the H view (0) and W view (1)
    int tsp1[2] = {1, 1}, tsp2[2] = {1, 1};
    int64_t tper1[2] = {0, 0}, tper2[2] = {0, 0};
    // sparse-V form: the caller's CSR of V (the W half-step's view), the library's CSC (the
    // H half-step's view), a transposed copy of H (gathered by the W half-step) and the
    // column sums c0 of the fixed factor without regularisation (sum_s z = sum_r c0_r x_r)
    bool sparse = false;
    int64_t nnz = 0;
    const int64_t* rptr = nullptr;
    const int32_t* cidx = nullptr;
    const void* rval = nullptr;
    int64_t* cptr = nullptr;
    int32_t* ridx = nullptr;
    void* cval = nullptr;
    void* Yt = nullptr;
    double* c0 = nullptr;
    // segments of at most sparse::SEG non-zeros per view (0: columns of V, 1: rows), built
    // at bind, with their partial sums
    int32_t* seg_col[2] = {nullptr, nullptr};
    int64_t* seg_k0[2] = {nullptr, nullptr};
    int64_t* seg_k1[2] = {nullptr, nullptr};
    int64_t* seg_ptr[2] = {nullptr, nullptr};
    int64_t nseg[2] = {0, 0};
    void* Aseg = nullptr;
    void* Bseg = nullptr;
    double* dseg = nullptr;
    // selection rule: DNA_SELECT_PAPER or DNA_SELECT_DESCENT (with the starting factor's
    // per-column costs from pass 1, [splits][max(N, T)])
    int selection = DNA_SELECT_PAPER;
    double* dcur = nullptr;
    // W-gradient of the H-step adjoint (allocated on first use): partial sums over splits
    // of o [wsp][R][N] and the column-sum terms per block of 32 columns [ceil(T / 32)][R]
    void* wg_part = nullptr;
    double* wg_cpart = nullptr;
    int wsp = 0;
    int64_t wper = 0;
    // dna_iterate replayed as a CUDA graph of one iteration (dna_use_graph): the
    // instantiated graph and the kernel launches it holds, in all and per phase
    bool use_graph = false;
    bool capturing = false;
    cudaGraphExec_t gexec = nullptr;
    int64_t graph_launches = 0;
    int64_t graph_phase_launches[DNA_NUM_PHASES] = {};
    // phase events captured in the graph (their own events: every replay records them
    // again), their (phase, index) pairs, and the replays since the last dna_phase_times
    std::vector<cudaEvent_t> graph_ev;
    size_t graph_ev_used = 0;
    std::vector<std::pair<int, size_t>> graph_recs;
    int64_t graph_replays = 0;
    // profiling: event pairs around phases, launch counts
    unsigned prof_mask = 0;          // phases whose instances get an event pair
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, size_t>> ev_recs;  // (phase, index of the start event)
    size_t ev_used = 0;
    double phase_ms[DNA_NUM_PHASES] = {};
    int64_t phase_launches[DNA_NUM_PHASES] = {};
};

namespace {

int set_device(const dna_ctx* c);
template <class F>
int phase(dna_ctx* c, int ph, int nlaunch, F&& f);

bool valid_opts(const dna_opts& o) {
    if (!(o.eps > 0.0) || !(o.eps <= 1.0)) return false;
    if (!(o.alpha >= 0.0)) return false;
    if (!(o.rho >= 0.0) || !(o.lambda >= 0.0)) return false;
    if (o.dtype != DNA_F64 && o.dtype != DNA_F32 && o.dtype != DNA_BF16) return false;
    if (o.engine < DNA_ENGINE_AUTO || o.engine > DNA_ENGINE_TENSOR) return false;
    return true;
}

template <typename P>
int dmalloc(P** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(reinterpret_cast<void**>(p), bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return DNA_ERR_ALLOC;
    }
    return DNA_OK;
}

View make_view(const dna_ctx* c, bool wstep) {
    View v{};
    v.R = c->R;
    if (!wstep) {  // H half-step: s = n, o = t
        v.S = c->N; v.O = c->T;
        v.V = c->V; v.vs = c->ldv;
        v.X = c->H; v.xr = c->T; v.xo = 1;
        v.Y = c->W; v.ys = c->R; v.yr = 1;
        v.vsum = c->colsum_v;
    } else {       // W half-step: s = t, o = n, on the transposed copy of V
        v.S = c->T; v.O = c->N;
        v.V = c->Vt; v.vs = c->ldvt;
        v.X = c->W; v.xr = 1; v.xo = c->R;
        v.Y = c->H; v.ys = 1; v.yr = c->T;
        v.vsum = c->rowsum_v;
    }
    return v;
}

// Split the reduction over s across CTAs.  Picks the split count that minimises the
// number of full waves per unit of work (ceil(blocks * splits / slots) / splits) plus the
// partial sums each split adds (`part_per_split`, relative to the work of one split-free
// pass) and a small fixed cost per CTA start; each split keeps at least four chunks.
// max_chunks > 0 caps the chunks one split may accumulate (the split FP32 form: the
// tensor pipe's float32 accumulation loses a fraction of an ulp per update, so long
// reductions are cut into partials that are summed with round-to-nearest adds).
void plan_split(int64_t S, int64_t nblocks_os, int slots, int chunk, int* splits, int64_t* per,
                double part_per_split = 0.02, int64_t max_chunks = 0) {
    const int64_t chunks = (S + chunk - 1) / chunk;
    const int64_t min_sp = max_chunks > 0 ? (chunks + max_chunks - 1) / max_chunks : 1;
    const int64_t max_sp = std::max<int64_t>(min_sp, std::min<int64_t>(32, chunks / 4));
    int64_t best = min_sp;
    double best_cost = 1e300;
    for (int64_t sp = min_sp; sp <= max_sp; ++sp) {
        const int64_t waves = (nblocks_os * sp + slots - 1) / slots;
        const double cost = (double)waves / (double)sp + part_per_split * (double)sp +
                            2.0 / (double)chunks * (double)waves;
        if (cost < best_cost - 1e-12) { best_cost = cost; best = sp; }
    }
    const int64_t per_chunks = (chunks + best - 1) / best;
    *per = per_chunks * chunk;
    *splits = (int)((S + *per - 1) / *per);
}

// Chunks of 128 that one pass-1 CTA of the split FP32 form accumulates in tensor memory
// (1024 values of s: the accumulation error stays near 1e-6 relative).
constexpr int64_t SPLIT_CHUNK = 128;
constexpr int64_t SPLIT_MAX_CHUNKS = 8;

// Pass 2 on the tensor cores balances (o-block, chunk) units over the SMs (pass2_split)
// in the split form at RP <= 128 and the BF16 form at RP <= 256; else it streams the X
// operands by K-slices over (o-block, split) tiles (pass2_large).
bool balanced_pass2(const dna_ctx* c) { return c->split ? c->rp <= 128 : c->rp <= 256; }

template <typename Tp>
void plan_all(dna_ctx* c) {
    using S = dna::Simt<Tp>;
    const int ob = S::oblock(), ch = S::chunk();
    const int rb = S::rblock(c->R);
    const int64_t nrb = (c->R + rb - 1) / rb;
    const int b1 = S::pass1_blocks_per_sm(c->R), b2 = S::pass2_blocks_per_sm(c->R);
    for (int w = 0; w < 2; ++w) {
        const int64_t Sdim = w ? c->T : c->N, Odim = w ? c->N : c->T;
        const int64_t nob = (Odim + ob - 1) / ob;
        plan_split(Sdim, nob * nrb, c->num_sms * b1, ch, &c->sp1[w], &c->per1[w]);
        plan_split(Sdim, nob, c->num_sms * b2, ch, &c->sp2[w], &c->per2[w]);
        if (c->tc) {
            const int tob = dna::TcBf16::oblock(), tch = dna::TcBf16::chunk();
            c->pad_o[w] = (Odim + tob - 1) / tob * tob;
            c->pad_s[w] = (Sdim + tch - 1) / tch * tch;
            // partial A, B sums per split relative to V's bytes: 2 R / S
            const double part = 2.0 * (double)c->R / (double)Sdim;
            // CTA rows per o-block of pass 1: the 256-wide r-blocks of the contraction kernel
            // (RP > 128; in the split form each for A and for B), or the A and B halves of
            // the split FP32 kernel
            const int64_t rblocks = (c->split ? 2 : 1) * (c->rp > 128 ? c->rp / 256 : 1);
            // the split form, and pass 1 at ranks above 128, stream s in chunks of 128
            const int sch = c->split ? (int)SPLIT_CHUNK : tch;
            const int sch1 = c->split || c->rp > 128 ? (int)SPLIT_CHUNK : tch;
            // the split form's pass 1 at R <= 128 accumulates a whole split in tensor
            // memory, so its splits are at most SPLIT_MAX_CHUNKS chunks; at R > 128 the
            // contraction kernel cuts each split into such segments itself
            plan_split(Sdim, c->pad_o[w] / tob * rblocks, c->num_sms, sch1, &c->tsp1[w],
                       &c->tper1[w], part, c->split && c->rp <= 128 ? SPLIT_MAX_CHUNKS : 0);
            plan_split(Sdim, c->pad_o[w] / tob, c->num_sms, c->rp > 256 ? (int)SPLIT_CHUNK : sch,
                       &c->tsp2[w], &c->tper2[w], 2.0 / (double)Sdim);
            // pass 2 of the split form at R <= 128 and of the BF16 form at R <= 256 balances
            // (o-block, chunk) units over the SMs instead; otherwise each split has four
            // cost slots (one per column group of the epilogue warps)
            if (balanced_pass2(c))
                c->tsp2[w] = dna::TcBf16::pass2_split_slots(c->pad_o[w], Sdim, c->num_sms);
            else if (!c->split && c->rp == 512) {   // Y-resident pass 2: a slot per s-block
                c->tsp2[w] = (int)((Sdim + SPLIT_CHUNK - 1) / SPLIT_CHUNK);
                c->tper2[w] = SPLIT_CHUNK;
            } else
                c->tsp2[w] *= 4;
        }
    }
}

void free_all(dna_ctx* c) {
    void* ptrs[] = {c->own_V, c->own_W, c->own_H, c->Vt, c->colsum_v, c->rowsum_v, c->c, c->sig,
                    c->fwork, c->gpart, c->vpart, c->Apart, c->Bpart, c->Xmu, c->Xdna, c->dpart, c->dfin_h, c->dfin_w,
                    c->choice_h, c->choice_w, c->kl_dev, c->kl_part, c->status, c->Xk, c->Yk, c->Ytk,
                    c->Y2tk, c->Xmk, c->Xdk, c->Vp, c->Qg, c->Qbg, c->cptr, c->ridx, c->cval, c->Yt, c->c0,
                    c->seg_col[0], c->seg_col[1], c->seg_k0[0], c->seg_k0[1], c->seg_k1[0],
                    c->seg_k1[1], c->seg_ptr[0], c->seg_ptr[1], c->Aseg, c->Bseg, c->dseg,
                    c->dcur, c->wg_part, c->wg_cpart};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t ev : c->ev_pool) cudaEventDestroy(ev);
    c->ev_pool.clear();
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    for (cudaEvent_t ev : c->graph_ev) cudaEventDestroy(ev);
    c->graph_ev.clear();
    c->graph_recs.clear();
}

template <typename Tp>
int alloc_workspace(dna_ctx* c) {
    plan_all<Tp>(c);
    const int64_t N = c->N, T = c->T, R = c->R, M = std::max(N, T);
    int64_t ap = 0, dp = 0;
    for (int w = 0; w < 2; ++w) {
        const int64_t O = w ? N : T;
        ap = std::max<int64_t>(ap, (int64_t)std::max(c->sp1[w], c->tsp1[w]) * R * O);
        dp = std::max<int64_t>(dp, (int64_t)std::max(c->sp2[w], c->tsp2[w]) * 2 * O);
    }
    c->ldvt = (N + 3) / 4 * 4;
    int e = DNA_OK;
    e |= dmalloc(&c->Vt, sizeof(Tp) * (size_t)T * c->ldvt);
    e |= dmalloc(&c->colsum_v, sizeof(double) * T);
    e |= dmalloc(&c->rowsum_v, sizeof(double) * N);
    e |= dmalloc(&c->c, sizeof(double) * R);
    e |= dmalloc(&c->sig, sizeof(double) * R);
    e |= dmalloc(&c->fwork, sizeof(double) * dna::FSUM_SPLITS * R);
    e |= dmalloc(&c->gpart, sizeof(double) * (size_t)(dna::Simt<Tp>::glue_parts(M) * R));
    e |= dmalloc(&c->vpart, sizeof(double) * (size_t)(((N + 31) / 32) * T + ((T + 31) / 32) * N));
    e |= dmalloc(&c->Apart, sizeof(Tp) * (size_t)ap);
    e |= dmalloc(&c->Bpart, sizeof(Tp) * (size_t)ap);
    e |= dmalloc(&c->Xmu, sizeof(Tp) * (size_t)(R * M));
    e |= dmalloc(&c->Xdna, sizeof(Tp) * (size_t)(R * M));
    e |= dmalloc(&c->dpart, sizeof(double) * (size_t)dp);
    e |= dmalloc(&c->dfin_h, sizeof(double) * 2 * T);
    e |= dmalloc(&c->dfin_w, sizeof(double) * 2 * N);
    e |= dmalloc(&c->choice_h, (size_t)T);
    e |= dmalloc(&c->choice_w, (size_t)N);
    e |= dmalloc(&c->kl_dev, sizeof(double));
    e |= dmalloc(&c->kl_part, sizeof(double) * (size_t)dna::REDUCE_PARTS);
    e |= dmalloc(&c->status, sizeof(int));
    if (c->tc) {
        const int64_t mo = std::max(c->pad_o[0], c->pad_o[1]);
        const int64_t ms = std::max(c->pad_s[0], c->pad_s[1]);
        const size_t b = 2;  // bf16
        // one plane size for every operand buffer, so the lo plane is always `plane` after
        // the hi plane (a multiple of 128 elements: TMA bases stay 256-byte aligned)
        c->plane = c->split ? std::max(mo, ms) * c->rp : 0;
        const size_t np = c->split ? 2 : 1;
        const int64_t po = c->split ? c->plane : mo * c->rp, ps = c->split ? c->plane : ms * c->rp;
        e |= dmalloc(&c->Xk, b * np * (size_t)po);
        e |= dmalloc(&c->Yk, b * np * (size_t)ps);
        e |= dmalloc(&c->Ytk, b * np * (size_t)ps);
        e |= dmalloc(&c->Y2tk, b * np * (size_t)ps);
        e |= dmalloc(&c->Xmk, b * np * (size_t)po);
        e |= dmalloc(&c->Xdk, b * np * (size_t)po);
        if (c->rp > 128) {   // pass 1 in two kernels: the Q, Qbar workspace (hi, lo planes)
            size_t q = 0;
            for (int w = 0; w < 2; ++w) {
                c->ldq[w] = ((w ? T : N) + 127) / 128 * 128;
                q = std::max(q, (size_t)(c->pad_o[w] * c->ldq[w]));
            }
            c->qplane = c->split ? (int64_t)q : 0;
            e |= dmalloc(&c->Qg, b * np * q);
            e |= dmalloc(&c->Qbg, b * np * q);
        }
    }
    if (e != DNA_OK) return DNA_ERR_ALLOC;
    // the padding columns of the transposed copy of V are read by 16-byte copies: zero them
    if (cudaMemset(c->Vt, 0, sizeof(Tp) * (size_t)T * c->ldvt) != cudaSuccess) return DNA_ERR_CUDA;
    if (cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) return DNA_ERR_CUDA;
    if (cudaMemset(c->choice_h, 0, (size_t)T) != cudaSuccess) return DNA_ERR_CUDA;
    if (cudaMemset(c->choice_w, 0, (size_t)N) != cudaSuccess) return DNA_ERR_CUDA;
    if (cudaMemset(c->dfin_h, 0, sizeof(double) * 2 * T) != cudaSuccess) return DNA_ERR_CUDA;
    if (cudaMemset(c->dfin_w, 0, sizeof(double) * 2 * N) != cudaSuccess) return DNA_ERR_CUDA;
    return DNA_OK;
}

// Workspace of the sparse-V form: no transposed copy of V (the CSC copy has nnz entries)
// and one split (each view column is reduced by one warp).
template <typename Tp>
int alloc_sparse_workspace(dna_ctx* c) {
    const int64_t N = c->N, T = c->T, R = c->R, M = std::max(N, T);
    int e = DNA_OK;
    e |= dmalloc(&c->colsum_v, sizeof(double) * T);
    e |= dmalloc(&c->rowsum_v, sizeof(double) * N);
    e |= dmalloc(&c->c, sizeof(double) * R);
    e |= dmalloc(&c->c0, sizeof(double) * R);
    e |= dmalloc(&c->sig, sizeof(double) * R);
    e |= dmalloc(&c->fwork, sizeof(double) * dna::FSUM_SPLITS * R);
    e |= dmalloc(&c->gpart, sizeof(double) * (size_t)(dna::Simt<Tp>::glue_parts(M) * R));
    e |= dmalloc(&c->Apart, sizeof(Tp) * (size_t)(R * M));
    e |= dmalloc(&c->Bpart, sizeof(Tp) * (size_t)(R * M));
    e |= dmalloc(&c->Xmu, sizeof(Tp) * (size_t)(R * M));
    e |= dmalloc(&c->Xdna, sizeof(Tp) * (size_t)(R * M));
    e |= dmalloc(&c->dpart, sizeof(double) * (size_t)(2 * M));
    e |= dmalloc(&c->dfin_h, sizeof(double) * 2 * T);
    e |= dmalloc(&c->dfin_w, sizeof(double) * 2 * N);
    e |= dmalloc(&c->choice_h, (size_t)T);
    e |= dmalloc(&c->choice_w, (size_t)N);
    e |= dmalloc(&c->kl_dev, sizeof(double));
    e |= dmalloc(&c->kl_part, sizeof(double) * (size_t)dna::REDUCE_PARTS);
    e |= dmalloc(&c->status, sizeof(int));
    e |= dmalloc(&c->cptr, sizeof(int64_t) * (size_t)(T + 1));
    e |= dmalloc(&c->ridx, sizeof(int32_t) * (size_t)std::max<int64_t>(c->nnz, 1));
    e |= dmalloc(&c->cval, sizeof(Tp) * (size_t)std::max<int64_t>(c->nnz, 1));
    e |= dmalloc(&c->Yt, sizeof(Tp) * (size_t)(T * R));
    if (e != DNA_OK) return DNA_ERR_ALLOC;
    if (cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->choice_h, 0, (size_t)T) != cudaSuccess ||
        cudaMemset(c->choice_w, 0, (size_t)N) != cudaSuccess ||
        cudaMemset(c->dfin_h, 0, sizeof(double) * 2 * T) != cudaSuccess ||
        cudaMemset(c->dfin_w, 0, sizeof(double) * 2 * N) != cudaSuccess)
        return DNA_ERR_CUDA;
    return DNA_OK;
}

// The CSC copy of V and the row and column sums of V (eq. 10 targets), built on the host
// from the caller's CSR (copied in once): the structure is validated first, so no kernel
// can index outside V, W or H.  Within a column the non-zeros keep ascending row order.
template <typename Tp>
int bind_csr(dna_ctx* c, const int64_t* rptr, const int32_t* cidx, const Tp* vals) {
    const int64_t N = c->N, T = c->T, nnz = c->nnz;
    std::vector<int64_t> rp((size_t)N + 1);
    std::vector<int32_t> ci((size_t)nnz);
    std::vector<Tp> vv((size_t)nnz);
    cudaStream_t st = c->stream;
    if (cudaMemcpyAsync(rp.data(), rptr, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        (nnz && cudaMemcpyAsync(ci.data(), cidx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
        (nnz && cudaMemcpyAsync(vv.data(), vals, sizeof(Tp) * nnz, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return DNA_ERR_CUDA;
    if (rp[0] != 0 || rp[N] != nnz) return DNA_ERR_ARG;
    for (int64_t n = 0; n < N; ++n)
        if (rp[n + 1] < rp[n]) return DNA_ERR_ARG;
    for (int64_t k = 0; k < nnz; ++k)
        if (ci[k] < 0 || ci[k] >= T || !(vv[k] >= Tp(0))) return DNA_ERR_ARG;
    std::vector<int64_t> cp((size_t)T + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) ++cp[ci[k] + 1];
    for (int64_t t = 0; t < T; ++t) cp[t + 1] += cp[t];
    std::vector<int64_t> fill(cp.begin(), cp.end() - 1);
    std::vector<int32_t> ri((size_t)nnz);
    std::vector<Tp> cv((size_t)nnz);
    std::vector<double> rs((size_t)N, 0.0), cs((size_t)T, 0.0);
    for (int64_t n = 0; n < N; ++n)
        for (int64_t k = rp[n]; k < rp[n + 1]; ++k) {
            const int64_t at = fill[ci[k]]++;
            ri[at] = (int32_t)n;
            cv[at] = vv[k];
            rs[n] += (double)vv[k];
        }
    for (int64_t t = 0; t < T; ++t)
        for (int64_t k = cp[t]; k < cp[t + 1]; ++k) cs[t] += (double)cv[k];
    // segment tables: view 0 cuts the columns (CSC), view 1 the rows (CSR)
    std::vector<int32_t> scol[2];
    std::vector<int64_t> sk0[2], sk1[2], sptr[2];
    for (int w = 0; w < 2; ++w) {
        const std::vector<int64_t>& p = w ? rp : cp;
        const int64_t O = w ? N : T;
        sptr[w].assign((size_t)O + 1, 0);
        for (int64_t o = 0; o < O; ++o) {
            for (int64_t k = p[o]; k < p[o + 1]; k += dna::SPARSE_SEG) {
                scol[w].push_back((int32_t)o);
                sk0[w].push_back(k);
                sk1[w].push_back(std::min<int64_t>(k + dna::SPARSE_SEG, p[o + 1]));
            }
            sptr[w][o + 1] = (int64_t)scol[w].size();
        }
    }
    const int64_t maxseg = std::max<int64_t>(1, std::max(scol[0].size(), scol[1].size()));
    for (int w = 0; w < 2; ++w) {
        for (void* q : {(void*)c->seg_col[w], (void*)c->seg_k0[w], (void*)c->seg_k1[w],
                        (void*)c->seg_ptr[w]})
            if (q) cudaFree(q);
        const int64_t n = std::max<int64_t>(1, (int64_t)scol[w].size());
        const int64_t O = w ? N : T;
        int e = dmalloc(&c->seg_col[w], sizeof(int32_t) * n);
        e |= dmalloc(&c->seg_k0[w], sizeof(int64_t) * n);
        e |= dmalloc(&c->seg_k1[w], sizeof(int64_t) * n);
        e |= dmalloc(&c->seg_ptr[w], sizeof(int64_t) * (O + 1));
        if (e) return DNA_ERR_ALLOC;
        c->nseg[w] = (int64_t)scol[w].size();
    }
    for (void* q : {c->Aseg, c->Bseg, (void*)c->dseg})
        if (q) cudaFree(q);
    if (dmalloc(&c->Aseg, sizeof(Tp) * (size_t)(maxseg * c->R)) ||
        dmalloc(&c->Bseg, sizeof(Tp) * (size_t)(maxseg * c->R)) ||
        dmalloc(&c->dseg, sizeof(double) * (size_t)(2 * maxseg)))
        return DNA_ERR_ALLOC;
    for (int w = 0; w < 2; ++w) {
        const int64_t O = w ? N : T;
        if ((c->nseg[w] &&
             (cudaMemcpyAsync(c->seg_col[w], scol[w].data(), sizeof(int32_t) * c->nseg[w], cudaMemcpyHostToDevice, st) != cudaSuccess ||
              cudaMemcpyAsync(c->seg_k0[w], sk0[w].data(), sizeof(int64_t) * c->nseg[w], cudaMemcpyHostToDevice, st) != cudaSuccess ||
              cudaMemcpyAsync(c->seg_k1[w], sk1[w].data(), sizeof(int64_t) * c->nseg[w], cudaMemcpyHostToDevice, st) != cudaSuccess)) ||
            cudaMemcpyAsync(c->seg_ptr[w], sptr[w].data(), sizeof(int64_t) * (O + 1), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return DNA_ERR_CUDA;
    }
    if (cudaMemcpyAsync(c->cptr, cp.data(), sizeof(int64_t) * (T + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (nnz && cudaMemcpyAsync(c->ridx, ri.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        (nnz && cudaMemcpyAsync(c->cval, cv.data(), sizeof(Tp) * nnz, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        cudaMemcpyAsync(c->rowsum_v, rs.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(c->colsum_v, cs.data(), sizeof(double) * T, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)   // the host vectors go out of scope
        return DNA_ERR_CUDA;
    return DNA_OK;
}

template <typename Tp>
int prepare(dna_ctx* c, const void* Vsrc = nullptr) {
    // Vsrc: V in pinned host memory, read by the transpose kernel and copied into c->V
    return phase(c, DNA_PHASE_PREPARE, 3, [&] {
        return dna::Simt<Tp>::prepare_v(
            static_cast<const Tp*>(Vsrc ? Vsrc : c->V), c->N, c->T, Vsrc ? c->T : c->ldv,
            static_cast<Tp*>(c->Vt), c->ldvt, c->colsum_v, c->rowsum_v, c->stream, c->vpart,
            Vsrc ? static_cast<Tp*>(const_cast<void*>(c->V)) : nullptr);
    });
}

// Steps 1/29 (which = 1) or 16 (which = 0).
template <typename Tp>
int normalize(dna_ctx* c, int which) {
    using S = dna::Simt<Tp>;
    const View v = make_view(c, which == 1);
    const double reg = which == 1 ? c->o.lambda : c->o.rho;
    return phase(c, DNA_PHASE_SUMS, 2, [&] {
        int e = S::factor_sums_x(v, reg, c->sig, c->fwork, c->stream);
        return e ? e : S::rescale(v, c->sig, c->stream);
    });
}

// V as the tensor-core kernels read it for each view (aligned copy for the H view if needed).
void tc_v(const dna_ctx* c, int wstep, const float** V, int64_t* vs) {
    if (wstep) { *V = static_cast<const float*>(c->Vt); *vs = c->ldvt; }
    else if (c->Vp) { *V = static_cast<const float*>(c->Vp); *vs = c->ldvp; }
    else { *V = static_cast<const float*>(c->V); *vs = c->ldv; }
}

dna::TcOperands tc_operands(const dna_ctx* c, int wstep) {
    const View v = make_view(c, wstep == 1);
    dna::TcOperands op{};
    op.S = v.S; op.O = v.O; op.R = v.R;
    op.S_pad = c->pad_s[wstep]; op.O_pad = c->pad_o[wstep];
    op.Xk = c->Xk; op.Yk = c->Yk; op.Ytk = c->Ytk; op.Y2tk = c->Y2tk;
    op.Xmk = c->Xmk; op.Xdk = c->Xdk;
    op.plane = c->plane;
    op.ctas = c->num_sms;
    op.Qg = c->Qg; op.Qbg = c->Qbg; op.ldq = c->ldq[wstep]; op.qplane = c->qplane;
    tc_v(c, wstep, &op.V, &op.vs);
    return op;
}

int build_tc_maps(dna_ctx* c) {
    for (int w = 0; w < 2; ++w) {
        const float* V;
        int64_t vs;
        tc_v(c, w, &V, &vs);
        if (int e = dna::TcBf16::make_maps(&c->maps[w], tc_operands(c, w), V, vs, c->Xmk, c->Xdk))
            return e;
    }
    return DNA_OK;
}

// One H half-step at fixed W (Algorithm 1 steps 4-15, no step-16 normalisation); the
// per-column choice is also copied to `choice_out` (device, T bytes) when given.
template <typename Tp>
int step_h_fixed(dna_ctx* c, uint8_t* choice_out) {
    using S = dna::Simt<Tp>;
    const View v = make_view(c, false);
    cudaStream_t st = c->stream;
    Tp* A = static_cast<Tp*>(c->Apart);
    Tp* B = static_cast<Tp*>(c->Bpart);
    Tp* Xmu = static_cast<Tp*>(c->Xmu);
    Tp* Xdna = static_cast<Tp*>(c->Xdna);
    int e = phase(c, DNA_PHASE_SUMS, 1, [&] { return S::factor_sums_y(v, c->o.lambda, c->c, c->fwork, st); });
    if (!e) e = phase(c, DNA_PHASE_PASS1, 1, [&] {
        return S::pass1(v, A, B, c->sp1[0], c->per1[0], true, c->status, st);
    });
    if (!e) e = phase(c, DNA_PHASE_CANDIDATES, 1, [&] {
        return S::candidates(v, c->c, A, B, c->sp1[0], Xmu, Xdna, c->o.eps, c->o.alpha, st);
    });
    if (!e) e = phase(c, DNA_PHASE_PASS2, 1, [&] {
        return S::pass2(v, Xmu, Xdna, c->dpart, c->sp2[0], c->per2[0], c->status, st);
    });
    if (!e) e = phase(c, DNA_PHASE_SELECT, 1, [&] {
        return S::select(v, Xmu, Xdna, c->dpart, c->sp2[0], c->choice_h, c->dfin_h, c->o.lambda,
                         st);
    });
    if (!e && choice_out &&
        cudaMemcpyAsync(choice_out, c->choice_h, (size_t)c->T, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
        e = DNA_ERR_CUDA;
    return e;
}

// Adjoint of step_h_fixed at state Hk with the recorded choices: Hbar_out = dL/dH_k from
// Hbar_next = dL/dH_{k+1}; Vbar += dL/dV and Wbar += dL/dW (either may be null).
template <typename Tp>
int step_h_adjoint(dna_ctx* c, const Tp* Hk, const uint8_t* choice, const Tp* Hbar_next,
                   Tp* Hbar_out, Tp* Vbar, Tp* Wbar) {
    using S = dna::Simt<Tp>;
    View v = make_view(c, false);
    v.X = const_cast<Tp*>(Hk);
    cudaStream_t st = c->stream;
    if (Wbar && !c->wg_part) {
        // o split so that the s-blocks x splits fill the SMs (one CTA per SM)
        plan_split(c->T, (c->N + 63) / 64, c->num_sms, 64, &c->wsp, &c->wper);
        if (dmalloc(&c->wg_part, sizeof(Tp) * (size_t)c->wsp * (size_t)c->R * (size_t)c->N) ||
            dmalloc(&c->wg_cpart, sizeof(double) * (size_t)((c->T + 31) / 32) * (size_t)c->R))
            return DNA_ERR_ALLOC;
    }
    Tp* A = static_cast<Tp*>(c->Apart);
    Tp* B = static_cast<Tp*>(c->Bpart);
    Tp* Abar = static_cast<Tp*>(c->Xmu);
    Tp* Bbar = static_cast<Tp*>(c->Xdna);
    int e = S::factor_sums_y(v, c->o.lambda, c->c, c->fwork, st);
    if (!e) e = S::pass1(v, A, B, c->sp1[0], c->per1[0], true, c->status, st);
    if (!e)
        e = S::adjoint_h(v, c->c, A, B, c->sp1[0], choice, Hbar_next, Hbar_out, Abar, Bbar,
                         c->dpart, A, c->sp1[0], c->per1[0], Vbar, c->T, c->o.eps, c->o.alpha,
                         c->status, st, Wbar ? c->wg_cpart : nullptr);
    if (!e && Wbar)
        e = S::adjoint_w(v, Abar, Bbar, c->wg_cpart, static_cast<Tp*>(c->wg_part), c->wsp,
                         c->wper, Wbar, c->status, st);
    return e;
}

// The BF16 precision form: the two O(NRT) passes on tcgen05 tensor cores (bf16 operands,
// float32 accumulation in TMEM), everything else as in the FP32 form.
// The operand buffers of half-step w for scale_ops (tensor-core form), else nulls.
struct OpsOut {
    void *Xk = nullptr, *Yk = nullptr, *Ytk = nullptr, *Y2tk = nullptr;
    int64_t rp = 0, O_pad = 0, S_pad = 0, plane = 0;
};
OpsOut ops_out(const dna_ctx* c, int w, bool with_sq) {
    OpsOut o;
    if (!c->tc) return o;
    o.Xk = c->Xk; o.Yk = c->Yk; o.Ytk = c->Ytk; o.Y2tk = with_sq ? c->Y2tk : nullptr;
    o.rp = c->rp; o.O_pad = c->pad_o[w]; o.S_pad = c->pad_s[w]; o.plane = c->plane;
    return o;
}

// Operands (tensor-core form) and eq. 7 / 14 denominators c of half-step w from the
// current W and H.
template <typename Tp>
int prep_step(dna_ctx* c, int w, bool with_sq) {
    using S = dna::Simt<Tp>;
    const View v = make_view(c, w == 1);
    const OpsOut o = ops_out(c, w, with_sq);
    int e = phase(c, c->tc ? DNA_PHASE_OPERANDS : DNA_PHASE_SUMS, 1, [&] {
        return S::scale_ops(v, nullptr, false, o.Xk, o.Yk, o.Ytk, o.Y2tk, o.rp, o.O_pad, o.S_pad,
                            o.plane, c->gpart, c->stream);
    });
    if (e) return e;
    return phase(c, DNA_PHASE_SUMS, 1, [&] {
        return S::part_sums(c->gpart, S::glue_parts(v.S), c->R, w ? c->o.rho : c->o.lambda, c->c,
                            c->stream);
    });
}

template <typename Tp>
int finish_step(dna_ctx* c, int w, bool next);
enum { STOP_NONE = 0, STOP_PASS1 = 1, STOP_PASS2 = 2, STOP_SELECT = 3 };
template <typename Tp>
int sparse_half_step(dna_ctx* c, int w, bool mu_only, bool prepared, bool next);

// One half-step (w = 0: Algorithm 1 steps 4-16, w = 1: steps 17-29).  mu_only: the
// multiplicative update of eq. 11 instead of DNA.  prepared: the operands and c of this
// half-step were left by the previous one (inside one dna_iterate call); next: leave them
// for half-step 1 - w (the step 16 / 29 normalisation writes them in the same pass).
template <typename Tp>
int step_core(dna_ctx* c, int w, bool mu_only, bool prepared, int stop);

template <typename Tp>
int half_step(dna_ctx* c, int w, bool mu_only, bool prepared, bool next) {
    if (c->sparse) return sparse_half_step<Tp>(c, w, mu_only, prepared, next);
    if (int e = step_core<Tp>(c, w, mu_only, prepared, STOP_NONE)) return e;
    return finish_step<Tp>(c, w, next);
}

// Steps of half_step up to and including the selection (the MU update with mu_only), which
// leaves the new factor and its per-block sums (gpart).  stop: STOP_PASS1 returns after
// pass 1 (the split partials of A, B in Apart, Bpart); STOP_PASS2 starts from A, B already
// summed into split 0 and returns after pass 2 (the cost slots in dpart); STOP_SELECT
// starts from the costs summed into slot 0 and runs the selection only.
template <typename Tp>
int step_core(dna_ctx* c, int w, bool mu_only, bool prepared, int stop) {
    using S = dna::Simt<Tp>;
    const View v = make_view(c, w == 1);
    Tp* A = static_cast<Tp*>(c->Apart);
    Tp* B = static_cast<Tp*>(c->Bpart);
    Tp* Xmu = static_cast<Tp*>(c->Xmu);
    Tp* Xdna = static_cast<Tp*>(c->Xdna);
    cudaStream_t st = c->stream;
    const bool tc = c->tc;
    const int sp1 = tc ? c->tsp1[w] : c->sp1[w], sp2 = tc ? c->tsp2[w] : c->sp2[w];
    int e = DNA_OK;
    // descent selection (CUDA-core engine): pass 1 also gives the starting factor's costs,
    // pass 2 evaluates the Newton candidate only
    const bool descent = c->selection == DNA_SELECT_DESCENT && !mu_only && !tc;
    if (stop <= STOP_PASS1) {
        if (!prepared)
            if ((e = prep_step<Tp>(c, w, !mu_only))) return e;
        e = phase(c, DNA_PHASE_PASS1, 1, [&] {
            if constexpr (sizeof(Tp) == 4)
                if (tc)
                    return c->split
                               ? dna::TcBf16::pass1_split(tc_operands(c, w), c->maps[w], A, B, sp1,
                                                          c->tper1[w], !mu_only, c->status, st)
                               : dna::TcBf16::pass1(tc_operands(c, w), c->maps[w], A, B, sp1,
                                                    c->tper1[w], !mu_only, c->status, st);
            return S::pass1(v, A, B, sp1, c->per1[w], !mu_only, c->status, st,
                            descent ? c->dcur : nullptr);
        });
        if (e || stop == STOP_PASS1) return e;
        if (mu_only)   // eq. 11 in place, with the first level of the step 16 / 29 sums
            return phase(c, DNA_PHASE_CANDIDATES, 1,
                         [&] { return S::mu_fused(v, c->c, A, sp1, c->gpart, st); });
    }
    int slots = sp2;
    if (stop <= STOP_PASS2) {
        // split partials over many columns: one streaming pass sums them into split 0 first
        // (in the candidates kernel each further split is another round of dependent loads;
        // the sums are the same, ascending split order either way)
        const int parts = stop == STOP_PASS2 ? 1 : sp1;
        const bool presum = (int64_t)parts * v.O >= 32768 && parts > 1;
        e = phase(c, DNA_PHASE_CANDIDATES, presum ? 2 : 1, [&] {
            if (presum)
                if (int r = S::split_sum(A, B, c->R, v.O, parts, st)) return r;
            return S::cand_fused(v, c->c, A, B, presum ? 1 : parts, Xmu, Xdna, c->o.eps,
                                 c->o.alpha, tc ? c->Xmk : nullptr, tc ? c->Xdk : nullptr, c->rp,
                                 c->pad_o[w], c->plane, st);
        });
        if (e) return e;
        e = phase(c, DNA_PHASE_PASS2, 1, [&] {
            if constexpr (sizeof(Tp) == 4)
                if (tc)
                    return balanced_pass2(c)
                               ? dna::TcBf16::pass2_split(tc_operands(c, w), c->maps[w], c->dpart,
                                                          sp2, c->status, st)
                               : dna::TcBf16::pass2_large(tc_operands(c, w), c->maps[w],
                                                          c->dpart, sp2, c->tper2[w], c->status,
                                                          st);
            if (descent) return S::pass2_one(v, Xdna, c->dpart, sp2, c->per2[w], c->status, st);
            return S::pass2(v, Xmu, Xdna, c->dpart, sp2, c->per2[w], c->status, st);
        });
        if (e || stop == STOP_PASS2) return e;
    } else {
        slots = 1;
    }
    return phase(c, DNA_PHASE_SELECT, 1, [&] {
        return S::select_fused(v, Xmu, Xdna, c->dpart, slots, w ? c->choice_w : c->choice_h,
                               w ? c->dfin_w : c->dfin_h, c->gpart, w ? c->o.rho : c->o.lambda,
                               st, descent ? c->dcur : nullptr, sp1);
    });
}

// Steps 16 / 29 after the new factor and its per-block sums (gpart) are written: f_r = sum
// over o of the new x(r, o) + (rho | lambda), then the rescale, fused (next) with the
// preparation of half-step 1 - w.  That half-step's eq. 7 / 14 denominators are the sums
// of its Y (this step's X after the rescale) plus the same rho | lambda: sum_o x(r, o) / f_r
// + reg, formed from f_r's own sum (equal to summing the rescaled factor up to rounding).
// The sparse form sums the rescaled factor instead (its pass 2 reads the raw sums from
// gpart).
template <typename Tp>
int finish_step(dna_ctx* c, int w, bool next) {
    using S = dna::Simt<Tp>;
    const View v = make_view(c, w == 1);
    cudaStream_t st = c->stream;
    int e = DNA_OK;
    const bool derive = next && !c->sparse;   // the next denominators from f_r's sums
    // steps 16 / 29: f_r = sum over o of the new x(r, o) + (rho | lambda)
    e = phase(c, DNA_PHASE_SUMS, 1, [&] {
        return S::part_sums(c->gpart, S::glue_parts(v.O), c->R, w ? c->o.lambda : c->o.rho,
                            c->sig, st, derive ? c->c : nullptr);
    });
    if (e) return e;
    if (!next)
        return phase(c, DNA_PHASE_SUMS, 1, [&] {
            return S::scale_ops(v, c->sig, false, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, 0,
                                nullptr, st);
        });
    // half-step 1 - w sees this step's X as its Y and this step's Y as its X
    const int wn = 1 - w;
    const View t = make_view(c, wn == 1);
    const OpsOut o = ops_out(c, wn, true);
    e = phase(c, DNA_PHASE_SUMS, 1, [&] {
        return S::scale_ops(t, c->sig, true, o.Xk, o.Yk, o.Ytk, o.Y2tk, o.rp, o.O_pad, o.S_pad,
                            o.plane, derive ? nullptr : c->gpart, st);
    });
    if (e || derive) return e;
    return phase(c, DNA_PHASE_SUMS, 1, [&] {
        return S::part_sums(c->gpart, S::glue_parts(t.S), c->R, wn ? c->o.rho : c->o.lambda, c->c,
                            st);
    });
}

dna::SparseSegs segs(const dna_ctx* c, int w) {
    return dna::SparseSegs{c->seg_col[w], c->seg_k0[w], c->seg_k1[w], c->seg_ptr[w], c->nseg[w]};
}

// One half-step of the sparse-V form: the same steps as half_step with the two O(NRT)
// passes replaced by passes over the non-zeros (sparse_kernels.cuh); candidates, selection
// and normalisation are the dense glue kernels (they touch only W, H and O-vectors).
template <typename Tp>
int sparse_half_step(dna_ctx* c, int w, bool mu_only, bool prepared, bool next) {
    using S = dna::Simt<Tp>;
    const View v = make_view(c, w == 1);
    Tp* A = static_cast<Tp*>(c->Apart);
    Tp* B = static_cast<Tp*>(c->Bpart);
    Tp* Xmu = static_cast<Tp*>(c->Xmu);
    Tp* Xdna = static_cast<Tp*>(c->Xdna);
    cudaStream_t st = c->stream;
    int e = DNA_OK;
    if (!prepared)
        if ((e = prep_step<Tp>(c, w, false))) return e;
    // c0 from the per-block column sums of Y that the preparation left in gpart
    e = phase(c, DNA_PHASE_SUMS, 1, [&] {
        return S::raw_sums(c->gpart, S::glue_parts(v.S), c->R, c->c0, st);
    });
    if (e) return e;
    const Tp* Yg = static_cast<const Tp*>(c->W);   // H-step: W is already S x R
    if (w == 1) {                                   // W-step: gather rows of H^t
        e = phase(c, DNA_PHASE_OPERANDS, 1, [&] {
            return S::transpose(static_cast<const Tp*>(c->H), c->R, c->T, static_cast<Tp*>(c->Yt), st);
        });
        if (e) return e;
        Yg = static_cast<const Tp*>(c->Yt);
    }
    const dna::SparseSegs sg = segs(c, w);
    const int32_t* idx = w ? c->cidx : c->ridx;
    const Tp* val = static_cast<const Tp*>(w ? c->rval : c->cval);
    Tp* Aseg = static_cast<Tp*>(c->Aseg);
    Tp* Bseg = static_cast<Tp*>(c->Bseg);
    e = phase(c, DNA_PHASE_PASS1, 2, [&] {
        return S::sp_pass1(v, sg, idx, val, Yg, Aseg, Bseg, A, B, !mu_only, c->status, st);
    });
    if (e) return e;
    if (mu_only) {
        e = phase(c, DNA_PHASE_CANDIDATES, 1, [&] { return S::mu_fused(v, c->c, A, 1, c->gpart, st); });
        return e ? e : finish_step<Tp>(c, w, next);
    }
    e = phase(c, DNA_PHASE_CANDIDATES, 1, [&] {
        return S::cand_fused(v, c->c, A, B, 1, Xmu, Xdna, c->o.eps, c->o.alpha, nullptr, nullptr,
                             0, 0, 0, st);
    });
    if (e) return e;
    e = phase(c, DNA_PHASE_PASS2, 2, [&] {
        return S::sp_pass2(v, sg, idx, val, Yg, Xmu, Xdna, c->c0, c->dseg, c->dpart, c->status, st);
    });
    if (e) return e;
    e = phase(c, DNA_PHASE_SELECT, 1, [&] {
        return S::select_fused(v, Xmu, Xdna, c->dpart, 1, w ? c->choice_w : c->choice_h,
                               w ? c->dfin_w : c->dfin_h, c->gpart, w ? c->o.rho : c->o.lambda,
                               st);
    });
    if (e) return e;
    return finish_step<Tp>(c, w, next);
}

// d_KL of the sparse-V form: per column of V the non-zeros' v log(v / z) - v plus
// sum_r c0_r h(r, t) (c0 = column sums of W), then the fixed-order total.
template <typename Tp>
int sparse_kl(dna_ctx* c) {
    using S = dna::Simt<Tp>;
    const View v = make_view(c, false);
    cudaStream_t st = c->stream;
    return phase(c, DNA_PHASE_KL, 5, [&] {
        int e = S::scale_ops(v, nullptr, false, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, 0,
                             c->gpart, st);
        if (!e) e = S::raw_sums(c->gpart, S::glue_parts(v.S), c->R, c->c0, st);
        if (!e) e = S::sp_kl(v, segs(c, 0), c->ridx, static_cast<const Tp*>(c->cval),
                             static_cast<const Tp*>(c->W), c->c0, c->dseg, c->dpart, c->status,
                             st);
        return e ? e : dna::reduce_sum(c->dpart, c->T, c->kl_dev, c->kl_part, st);
    });
}

// Gradient of eq. 1 (no regularisation) with respect to W, H and V, scaled by `scale`:
// dH = W^t (1 - Q) = (W^t 1) - W^t Q, dW = (1 - Q) H^t = (H 1)^t - Q H^t, dV = log(V / Z).
// The raw W^t Q and Q H^t are pass 1 of the H and W views without the Qbar half.
template <typename Tp>
int kl_backward(dna_ctx* c, double scale, Tp* dW, Tp* dH, Tp* dV) {
    using S = dna::Simt<Tp>;
    cudaStream_t st = c->stream;
    Tp* A = static_cast<Tp*>(c->Apart);
    for (int w = 0; w < 2; ++w) {
        Tp* G = w ? dW : dH;
        if (!G) continue;
        const View v = make_view(c, w == 1);
        int e = S::factor_sums_y(v, 0.0, c->c, c->fwork, st);
        if (!e) e = S::pass1(v, A, A, c->sp1[w], c->per1[w], false, c->status, st);
        if (!e) e = w ? S::grad_x(v, c->c, A, c->sp1[w], scale, G, 1, c->R, st)
                      : S::grad_x(v, c->c, A, c->sp1[w], scale, G, c->T, 1, st);
        if (e) return e;
    }
    if (dV) return S::grad_v(make_view(c, false), scale, dV, c->T, c->status, st);
    return DNA_OK;
}

template <typename Tp>
int kl_async(dna_ctx* c) {
    if (c->sparse) return sparse_kl<Tp>(c);
    const View v = make_view(c, false);
    if constexpr (sizeof(Tp) == 4)
        if (c->split && c->rp <= 128) {   // the split tensor-core pass 2 on the H view's operands
            if (int e = prep_step<Tp>(c, 0, false)) return e;
            return phase(c, DNA_PHASE_KL, 2, [&] {
                int e = dna::TcBf16::kl_split(tc_operands(c, 0), c->maps[0], c->dpart,
                                              c->tsp2[0], c->status, c->stream);
                return e ? e
                         : dna::reduce_sum(c->dpart, (int64_t)c->tsp2[0] * c->T, c->kl_dev,
                                           c->kl_part, c->stream);
            });
        }
    return phase(c, DNA_PHASE_KL, 2, [&] {
        int e = dna::Simt<Tp>::kl_columns(v, c->dpart, c->sp2[0], c->per2[0], c->status, c->stream);
        return e ? e
                 : dna::reduce_sum(c->dpart, (int64_t)c->sp2[0] * c->T, c->kl_dev, c->kl_part,
                                   c->stream);
    });
}

int read_status(dna_ctx* c) {
    int st = 0;
    if (cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DNA_ERR_CUDA;
    if (st & dna::STATUS_NONFINITE) return DNA_ERR_NONFINITE;
    if (st & dna::STATUS_TIMEOUT) return DNA_ERR_TIMEOUT;
    return DNA_OK;
}

bool is_f64(const dna_ctx* c) { return c->o.dtype == DNA_F64; }

int check_ready(const dna_ctx* c) {
    if (!c) return DNA_ERR_ARG;
    if (!c->bound) return DNA_ERR_ARG;
    return DNA_OK;
}

int set_device(const dna_ctx* c) {
    return cudaSetDevice(c->device) == cudaSuccess ? DNA_OK : DNA_ERR_CUDA;
}

// Run f as one instance of phase ph, bracketed by an event pair when profiling is on;
// the kernels it launches are counted (nlaunch is the expected count, for reading only).
template <class F>
int phase(dna_ctx* c, int ph, int nlaunch, F&& f) {
    // events of a profiled phase: from the pool, or while a graph is being captured two
    // events of the graph's own, recorded as graph nodes (cudaEventRecordExternal)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((c->prof_mask >> ph) & 1u) {
        if (c->capturing) {
            if (c->graph_ev_used + 2 <= c->graph_ev.size()) {
                e0 = c->graph_ev[c->graph_ev_used];
                e1 = c->graph_ev[c->graph_ev_used + 1];
                c->graph_recs.emplace_back(ph, c->graph_ev_used);
                c->graph_ev_used += 2;
            }
        } else if (c->ev_used + 2 <= c->ev_pool.size()) {
            e0 = c->ev_pool[c->ev_used];
            e1 = c->ev_pool[c->ev_used + 1];
            c->ev_recs.emplace_back(ph, c->ev_used);
            c->ev_used += 2;
        }
    }
    auto record = [&](cudaEvent_t ev) {
        return c->capturing ? cudaEventRecordWithFlags(ev, c->stream, cudaEventRecordExternal)
                            : cudaEventRecord(ev, c->stream);
    };
    if (e0 && record(e0) != cudaSuccess) return DNA_ERR_CUDA;
    const int64_t before = dna::launch_count();
    const int e = f();
    if (e1 && record(e1) != cudaSuccess) return DNA_ERR_CUDA;
    c->phase_launches[ph] += dna::launch_count() - before;
    return e;
}

// ---------------------------------------------------------------- column shards
int shard_ready(dna_ctx* c) {
    if (int e = check_ready(c)) return e;
    if (c->sparse || c->host_mode || c->selection != DNA_SELECT_PAPER) return DNA_ERR_UNSUPPORTED;
    return set_device(c) ? DNA_ERR_CUDA : DNA_OK;
}

int d2d(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess
               ? DNA_OK
               : DNA_ERR_CUDA;
}

template <typename Tp>
int shard_H_begin(dna_ctx* c, double* rsum) {
    using S = dna::Simt<Tp>;
    if (int e = step_core<Tp>(c, 0, false, false, STOP_NONE)) return e;
    if (int e = S::raw_sums(c->gpart, S::glue_parts(c->T), c->R, c->sig, c->stream)) return e;
    return d2d(rsum, c->sig, sizeof(double) * c->R, c->stream);
}

template <typename Tp>
int shard_H_end(dna_ctx* c, const double* rsum) {
    using S = dna::Simt<Tp>;
    if (int e = S::add_reg(rsum, c->R, c->o.rho, c->sig, c->stream)) return e;
    return S::scale_ops(make_view(c, false), c->sig, false, nullptr, nullptr, nullptr, nullptr, 0,
                        0, 0, 0, nullptr, c->stream);
}

template <typename Tp>
int shard_W_begin(dna_ctx* c, double* hsum) {
    using S = dna::Simt<Tp>;
    if (int e = prep_step<Tp>(c, 1, true)) return e;
    if (int e = S::raw_sums(c->gpart, S::glue_parts(c->T), c->R, c->sig, c->stream)) return e;
    return d2d(hsum, c->sig, sizeof(double) * c->R, c->stream);
}

template <typename Tp>
int shard_W_pass1(dna_ctx* c, const double* hsum, void* AB) {
    using S = dna::Simt<Tp>;
    if (int e = S::add_reg(hsum, c->R, c->o.rho, c->c, c->stream)) return e;
    if (int e = step_core<Tp>(c, 1, false, true, STOP_PASS1)) return e;
    const int sp1 = c->tc ? c->tsp1[1] : c->sp1[1];
    Tp* A = static_cast<Tp*>(c->Apart);
    Tp* B = static_cast<Tp*>(c->Bpart);
    if (int e = S::split_sum(A, B, c->R, c->N, sp1, c->stream)) return e;
    const size_t n = sizeof(Tp) * (size_t)(c->R * c->N);
    if (int e = d2d(AB, A, n, c->stream)) return e;
    return d2d(static_cast<char*>(AB) + n, B, n, c->stream);
}

template <typename Tp>
int shard_W_pass2(dna_ctx* c, const void* AB, double* cost) {
    const size_t n = sizeof(Tp) * (size_t)(c->R * c->N);
    if (int e = d2d(c->Apart, AB, n, c->stream)) return e;
    if (int e = d2d(c->Bpart, static_cast<const char*>(AB) + n, n, c->stream)) return e;
    if (int e = step_core<Tp>(c, 1, false, true, STOP_PASS2)) return e;
    const int sp2 = c->tc ? c->tsp2[1] : c->sp2[1];
    // the cost slots [sp2][2][N] summed into slot 0 (float64, ascending slot order)
    if (int e = dna::Simt<double>::split_sum(c->dpart, nullptr, 1, 2 * c->N, sp2, c->stream))
        return e;
    return d2d(cost, c->dpart, sizeof(double) * 2 * c->N, c->stream);
}

template <typename Tp>
int shard_W_end(dna_ctx* c, const double* cost) {
    if (int e = d2d(c->dpart, cost, sizeof(double) * 2 * c->N, c->stream)) return e;
    if (int e = step_core<Tp>(c, 1, false, true, STOP_SELECT)) return e;
    return finish_step<Tp>(c, 1, false);
}

// dna_iterate as graph replays: the H half-step's operands and denominators are formed
// from the current factors (as the first half-step of an eager call does), then each
// iteration replays one captured iteration whose half-steps both leave the next one's
// operands (the last one's are not used).  The factors match the eager path bit for bit.
template <typename Tp>
int iterate_graph(dna_ctx* c, int iters) {
    if (int e = prep_step<Tp>(c, 0, true)) return e;
    if (!c->gexec) {   // one iteration, captured once; pointers are fixed until the next bind
        // events for the profiled phases of the captured iteration (created before capture)
        c->graph_recs.clear();
        c->graph_ev_used = 0;
        if (c->prof_mask && c->graph_ev.empty()) {
            c->graph_ev.resize(64, nullptr);
            for (auto& ev : c->graph_ev)
                if (cudaEventCreate(&ev) != cudaSuccess) return DNA_ERR_CUDA;
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return DNA_ERR_CUDA;
        int64_t ph0[DNA_NUM_PHASES];
        std::copy(c->phase_launches, c->phase_launches + DNA_NUM_PHASES, ph0);
        const int64_t before = dna::launch_count();
        c->capturing = true;
        int e = half_step<Tp>(c, 0, false, true, true);
        if (!e) e = half_step<Tp>(c, 1, false, true, true);
        c->capturing = false;
        const cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
        // the capture ran nothing: move its launch counts from the counters to the graph
        c->graph_launches = dna::launch_count() - before;
        dna::launch_count() = before;
        for (int p = 0; p < DNA_NUM_PHASES; ++p) {
            c->graph_phase_launches[p] = c->phase_launches[p] - ph0[p];
            c->phase_launches[p] = ph0[p];
        }
        if (e || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            c->graph_recs.clear();
            return e ? e : DNA_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            c->gexec = nullptr;
            c->graph_recs.clear();
            cudaGetLastError();
            return DNA_ERR_CUDA;
        }
        c->graph_replays = 0;
    }
    for (int i = 0; i < iters; ++i) {
        if (cudaGraphLaunch(c->gexec, c->stream) != cudaSuccess) return DNA_ERR_CUDA;
        dna::launch_count() += c->graph_launches;
        for (int p = 0; p < DNA_NUM_PHASES; ++p) c->phase_launches[p] += c->graph_phase_launches[p];
    }
    c->graph_replays += iters;
    return DNA_OK;
}

void drop_graph(dna_ctx* c) {
    if (c->gexec) {
        cudaStreamSynchronize(c->stream);
        cudaGraphExecDestroy(c->gexec);
    }
    c->gexec = nullptr;
    for (cudaEvent_t ev : c->graph_ev) cudaEventDestroy(ev);
    c->graph_ev.clear();
    c->graph_recs.clear();
    c->graph_replays = 0;
}

}  // namespace

namespace dna {

// out[b] = sum of part[b * per .. min(n, (b + 1) * per)), one CTA of 256 threads per b:
// strided per-thread sums, then a fixed tree.
__global__ void k_reduce_sum(const double* __restrict__ part, int64_t n, int64_t per,
                             double* __restrict__ out) {
    __shared__ double red[256];
    const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(n, i0 + per);
    double s0 = 0.0, s1 = 0.0;
    int64_t i = i0 + threadIdx.x;
    for (; i + 256 < i1; i += 512) { s0 += part[i]; s1 += part[i + 256]; }
    if (i < i1) s0 += part[i];
    red[threadIdx.x] = s0 + s1;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// Two levels: up to REDUCE_PARTS CTA sums into `work`, then one CTA over those.
int reduce_sum(const double* part, int64_t n, double* out, double* work, cudaStream_t st) {
    const int64_t per = std::max<int64_t>(4096, (n + REDUCE_PARTS - 1) / REDUCE_PARTS);
    const int64_t blocks = (n + per - 1) / per;
    if (blocks <= 1) {
        k_reduce_sum<<<1, 256, 0, st>>>(part, n, std::max<int64_t>(n, 1), out);
        return after_launch();
    }
    k_reduce_sum<<<(unsigned)blocks, 256, 0, st>>>(part, n, per, work);
    if (int e = after_launch()) return e;
    k_reduce_sum<<<1, 256, 0, st>>>(work, blocks, blocks, out);
    return after_launch();
}

}  // namespace dna

extern "C" {

void dna_default_opts(dna_opts* o) {
    if (!o) return;
    o->eps = 0.01;
    o->alpha = 4.0;
    o->rho = 0.0;
    o->lambda = 0.0;
    o->dtype = DNA_F32;
    o->engine = DNA_ENGINE_AUTO;
}

const char* dna_strerror(int code) {
    switch (code) {
        case DNA_OK: return "ok";
        case DNA_ERR_ARG: return "invalid argument";
        case DNA_ERR_CUDA: return "CUDA runtime error";
        case DNA_ERR_NONFINITE: return "non-positive z where v > 0 (infinite cost)";
        case DNA_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case DNA_ERR_UNSUPPORTED: return "not supported by this build";
        case DNA_ERR_ALLOC: return "device allocation failed";
        case DNA_ERR_LIMIT: return "size beyond the static scratch limit of dna_kl_noalloc";
        default: return "unknown status code";
    }
}

int dna_create(int64_t N, int64_t T, int64_t R, const dna_opts* opts, dna_ctx** out) {
    if (!out) return DNA_ERR_ARG;
    *out = nullptr;
    if (N < 1 || T < 1 || R < 1 || R > 512) return DNA_ERR_ARG;
    if (N > (int64_t)1 << 31 || T > (int64_t)1 << 31) return DNA_ERR_ARG;
    dna_opts o;
    dna_default_opts(&o);
    if (opts) o = *opts;
    if (!valid_opts(o)) return DNA_ERR_ARG;
    // Engines: BF16 runs on the tensor cores (R <= 512).  F32 runs on the CUDA cores by
    // default and on the tensor cores (split hi + lo bf16 operands, R <= 512) when the
    // tensor engine is asked for.  F64 runs on the CUDA cores.
    const bool split = o.dtype == DNA_F32 && o.engine == DNA_ENGINE_TENSOR;
    const bool tc = o.dtype == DNA_BF16 || split;
    if (o.dtype == DNA_BF16 && (o.engine == DNA_ENGINE_SIMT || dna::TcBf16::rank_pad(R) == 0))
        return DNA_ERR_UNSUPPORTED;
    if (split && dna::TcBf16::rank_pad(R) == 0) return DNA_ERR_UNSUPPORTED;
    if (o.dtype == DNA_F64 && o.engine == DNA_ENGINE_TENSOR) return DNA_ERR_UNSUPPORTED;
    dna_ctx* c = new (std::nothrow) dna_ctx();
    if (!c) return DNA_ERR_ALLOC;
    c->N = N; c->T = T; c->R = R; c->o = o;
    c->tc = tc;
    c->split = split;
    c->rp = tc ? dna::TcBf16::rank_pad(R) : 0;
    c->esz = o.dtype == DNA_F64 ? 8 : 4;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete c;
        return DNA_ERR_CUDA;
    }
    const int e = is_f64(c) ? alloc_workspace<double>(c) : alloc_workspace<float>(c);
    if (e != DNA_OK) {
        free_all(c);
        delete c;
        return e;
    }
    *out = c;
    return DNA_OK;
}

int dna_create_sparse(int64_t N, int64_t T, int64_t R, int64_t nnz, const dna_opts* opts,
                      dna_ctx** out) {
    if (!out) return DNA_ERR_ARG;
    *out = nullptr;
    if (N < 1 || T < 1 || R < 1 || nnz < 0) return DNA_ERR_ARG;
    if (N > ((int64_t)1 << 31) - 1 || T > ((int64_t)1 << 31) - 1 || nnz > ((int64_t)1 << 40))
        return DNA_ERR_ARG;
    dna_opts o;
    dna_default_opts(&o);
    if (opts) o = *opts;
    if (!valid_opts(o)) return DNA_ERR_ARG;
    if (R > 128 || o.dtype == DNA_BF16 || o.engine == DNA_ENGINE_TENSOR) return DNA_ERR_UNSUPPORTED;
    dna_ctx* c = new (std::nothrow) dna_ctx();
    if (!c) return DNA_ERR_ALLOC;
    c->N = N; c->T = T; c->R = R; c->o = o;
    c->sparse = true;
    c->nnz = nnz;
    c->esz = o.dtype == DNA_F64 ? 8 : 4;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete c;
        return DNA_ERR_CUDA;
    }
    const int e = is_f64(c) ? alloc_sparse_workspace<double>(c) : alloc_sparse_workspace<float>(c);
    if (e != DNA_OK) {
        free_all(c);
        delete c;
        return e;
    }
    *out = c;
    return DNA_OK;
}

int dna_bind_csr(dna_ctx* c, const int64_t* row_ptr, const int32_t* col_idx, const void* vals,
                 void* W, void* H) {
    if (!c || !c->sparse || !row_ptr || (c->nnz && (!col_idx || !vals)) || !W || !H)
        return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    const int e = is_f64(c) ? bind_csr<double>(c, row_ptr, col_idx, static_cast<const double*>(vals))
                            : bind_csr<float>(c, row_ptr, col_idx, static_cast<const float*>(vals));
    if (e) return e;
    c->rptr = row_ptr; c->cidx = col_idx; c->rval = vals;
    c->W = W; c->H = H;
    c->bound = true;
    return DNA_OK;
}

int dna_bind(dna_ctx* c, const void* V, int64_t ldv, void* W, void* H) {
    if (!c || !V || !W || !H || ldv < c->T) return DNA_ERR_ARG;
    if (c->host_mode || c->sparse) return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    c->V = V; c->ldv = ldv; c->W = W; c->H = H;
    c->bound = true;
    drop_graph(c);
    if (c->tc && (ldv % 4 != 0 || reinterpret_cast<uintptr_t>(V) % 16 != 0)) {
        // the tensor-core kernels copy V in 16-byte pieces: keep an aligned, padded copy
        c->ldvp = (c->T + 3) / 4 * 4;
        if (!c->Vp) {
            if (dmalloc(&c->Vp, sizeof(float) * (size_t)(c->N * c->ldvp))) return DNA_ERR_ALLOC;
            if (cudaMemset(c->Vp, 0, sizeof(float) * (size_t)(c->N * c->ldvp)) != cudaSuccess)
                return DNA_ERR_CUDA;
        }
        if (cudaMemcpy2DAsync(c->Vp, sizeof(float) * c->ldvp, V, sizeof(float) * ldv,
                              sizeof(float) * c->T, c->N, cudaMemcpyDeviceToDevice,
                              c->stream) != cudaSuccess)
            return DNA_ERR_CUDA;
    }
    if (c->tc)
        if (int e = build_tc_maps(c)) return e;
    return is_f64(c) ? prepare<double>(c) : prepare<float>(c);
}

int dna_set_stream(dna_ctx* c, void* stream) {
    if (!c) return DNA_ERR_ARG;
    c->stream = static_cast<cudaStream_t>(stream);
    return DNA_OK;
}

int dna_normalize(dna_ctx* c, int which) {
    if (int e = check_ready(c)) return e;
    if (which != 0 && which != 1) return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    return is_f64(c) ? normalize<double>(c, which) : normalize<float>(c, which);
}

int dna_step_H(dna_ctx* c) {
    if (int e = check_ready(c)) return e;
    if (set_device(c)) return DNA_ERR_CUDA;
    return is_f64(c) ? half_step<double>(c, 0, false, false, false)
                     : half_step<float>(c, 0, false, false, false);
}

int dna_step_W(dna_ctx* c) {
    if (int e = check_ready(c)) return e;
    if (set_device(c)) return DNA_ERR_CUDA;
    return is_f64(c) ? half_step<double>(c, 1, false, false, false)
                     : half_step<float>(c, 1, false, false, false);
}

int dna_iterate(dna_ctx* c, int iters) {
    if (int e = check_ready(c)) return e;
    if (iters < 0) return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    if (iters > 0 && c->use_graph && c->stream && !c->sparse)
        return is_f64(c) ? iterate_graph<double>(c, iters) : iterate_graph<float>(c, iters);
    // each half-step leaves the operands and denominators of the next one
    for (int i = 0; i < iters; ++i) {
        const bool more = i + 1 < iters;
        int e = is_f64(c) ? half_step<double>(c, 0, false, i > 0, true)
                          : half_step<float>(c, 0, false, i > 0, true);
        if (!e) e = is_f64(c) ? half_step<double>(c, 1, false, true, more)
                              : half_step<float>(c, 1, false, true, more);
        if (e) return e;
    }
    return DNA_OK;
}

int mu_step(dna_ctx* c, int which) {
    if (int e = check_ready(c)) return e;
    if (which != 0 && which != 1) return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    return is_f64(c) ? half_step<double>(c, which, true, false, false)
                     : half_step<float>(c, which, true, false, false);
}

int mu_iterate(dna_ctx* c, int iters) {
    if (int e = check_ready(c)) return e;
    if (iters < 0) return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    for (int i = 0; i < iters; ++i) {
        const bool more = i + 1 < iters;
        int e = is_f64(c) ? half_step<double>(c, 0, true, i > 0, true)
                          : half_step<float>(c, 0, true, i > 0, true);
        if (!e) e = is_f64(c) ? half_step<double>(c, 1, true, true, more)
                              : half_step<float>(c, 1, true, true, more);
        if (e) return e;
    }
    return DNA_OK;
}

int dna_set_selection(dna_ctx* c, int mode) {
    if (!c || (mode != DNA_SELECT_PAPER && mode != DNA_SELECT_DESCENT)) return DNA_ERR_ARG;
    if (mode == DNA_SELECT_DESCENT && (c->tc || c->sparse)) return DNA_ERR_UNSUPPORTED;
    if (set_device(c)) return DNA_ERR_CUDA;
    if (mode == DNA_SELECT_DESCENT && !c->dcur) {
        const int sp = std::max(c->sp1[0], c->sp1[1]);
        if (dmalloc(&c->dcur, sizeof(double) * (size_t)sp * std::max(c->N, c->T)))
            return DNA_ERR_ALLOC;
    }
    if (mode != c->selection) drop_graph(c);
    c->selection = mode;
    return DNA_OK;
}

int dna_use_graph(dna_ctx* c, int enable) {
    if (!c) return DNA_ERR_ARG;
    c->use_graph = enable != 0;
    return DNA_OK;
}

int dna_check_wait_timeout(int64_t limit_cycles) {
    if (limit_cycles < 1 || limit_cycles > ((int64_t)1 << 32)) return DNA_ERR_ARG;
    int* status = nullptr;
    if (dmalloc(&status, sizeof(int))) return DNA_ERR_ALLOC;
    int st = 0;
    int e = cudaMemset(status, 0, sizeof(int)) == cudaSuccess ? DNA_OK : DNA_ERR_CUDA;
    if (!e) e = dna::TcBf16::check_wait_timeout(limit_cycles, status, nullptr);
    if (!e && (cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess))
        e = DNA_ERR_CUDA;
    cudaFree(status);
    if (e) return e;
    return (st & dna::STATUS_TIMEOUT) ? DNA_ERR_TIMEOUT : DNA_OK;
}

int dna_shard_rowsums(dna_ctx* c, double* out) {
    if (!out) return DNA_ERR_ARG;
    if (int e = shard_ready(c)) return e;
    return d2d(out, c->rowsum_v, sizeof(double) * c->N, c->stream);
}

int dna_shard_set_rowsums(dna_ctx* c, const double* in) {
    if (!in) return DNA_ERR_ARG;
    if (int e = shard_ready(c)) return e;
    return d2d(c->rowsum_v, in, sizeof(double) * c->N, c->stream);
}

int dna_shard_H_begin(dna_ctx* c, double* rsum) {
    if (!rsum) return DNA_ERR_ARG;
    if (int e = shard_ready(c)) return e;
    return is_f64(c) ? shard_H_begin<double>(c, rsum) : shard_H_begin<float>(c, rsum);
}

int dna_shard_H_end(dna_ctx* c, const double* rsum) {
    if (!rsum) return DNA_ERR_ARG;
    if (int e = shard_ready(c)) return e;
    return is_f64(c) ? shard_H_end<double>(c, rsum) : shard_H_end<float>(c, rsum);
}

int dna_shard_W_begin(dna_ctx* c, double* hsum) {
    if (!hsum) return DNA_ERR_ARG;
    if (int e = shard_ready(c)) return e;
    return is_f64(c) ? shard_W_begin<double>(c, hsum) : shard_W_begin<float>(c, hsum);
}

int dna_shard_W_pass1(dna_ctx* c, const double* hsum, void* AB) {
    if (!hsum || !AB) return DNA_ERR_ARG;
    if (int e = shard_ready(c)) return e;
    return is_f64(c) ? shard_W_pass1<double>(c, hsum, AB) : shard_W_pass1<float>(c, hsum, AB);
}

int dna_shard_W_pass2(dna_ctx* c, const void* AB, double* cost) {
    if (!AB || !cost) return DNA_ERR_ARG;
    if (int e = shard_ready(c)) return e;
    return is_f64(c) ? shard_W_pass2<double>(c, AB, cost) : shard_W_pass2<float>(c, AB, cost);
}

int dna_shard_W_end(dna_ctx* c, const double* cost) {
    if (!cost) return DNA_ERR_ARG;
    if (int e = shard_ready(c)) return e;
    return is_f64(c) ? shard_W_end<double>(c, cost) : shard_W_end<float>(c, cost);
}

int dna_kl(dna_ctx* c, double* out) {
    if (int e = check_ready(c)) return e;
    if (!out) return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    int e = is_f64(c) ? kl_async<double>(c) : kl_async<float>(c);
    if (e) return e;
    if (cudaMemcpyAsync(out, c->kl_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
        return DNA_ERR_CUDA;
    return read_status(c);
}

int dna_step_H_fixed(dna_ctx* c, uint8_t* choice_out) {
    if (int e = check_ready(c)) return e;
    if (c->tc || c->sparse) return DNA_ERR_UNSUPPORTED;
    if (set_device(c)) return DNA_ERR_CUDA;
    return is_f64(c) ? step_h_fixed<double>(c, choice_out) : step_h_fixed<float>(c, choice_out);
}

int dna_step_H_adjoint_w(dna_ctx* c, const void* Hk, const uint8_t* choice,
                         const void* Hbar_next, void* Hbar_out, void* Vbar, void* Wbar) {
    if (int e = check_ready(c)) return e;
    if (!Hk || !choice || !Hbar_next || !Hbar_out) return DNA_ERR_ARG;
    if (c->tc || c->sparse || (is_f64(c) ? c->R > 64 : c->R > 128)) return DNA_ERR_UNSUPPORTED;
    if (set_device(c)) return DNA_ERR_CUDA;
    if (is_f64(c))
        return step_h_adjoint<double>(c, static_cast<const double*>(Hk), choice,
                                      static_cast<const double*>(Hbar_next),
                                      static_cast<double*>(Hbar_out), static_cast<double*>(Vbar),
                                      static_cast<double*>(Wbar));
    return step_h_adjoint<float>(c, static_cast<const float*>(Hk), choice,
                                 static_cast<const float*>(Hbar_next), static_cast<float*>(Hbar_out),
                                 static_cast<float*>(Vbar), static_cast<float*>(Wbar));
}

int dna_step_H_adjoint(dna_ctx* c, const void* Hk, const uint8_t* choice, const void* Hbar_next,
                       void* Hbar_out, void* Vbar) {
    if (!Vbar) return DNA_ERR_ARG;
    return dna_step_H_adjoint_w(c, Hk, choice, Hbar_next, Hbar_out, Vbar, nullptr);
}

int dna_kl_backward(dna_ctx* c, double scale, void* dW, void* dH, void* dV) {
    if (int e = check_ready(c)) return e;
    if (c->tc || c->sparse) return DNA_ERR_UNSUPPORTED;
    if (set_device(c)) return DNA_ERR_CUDA;
    if (is_f64(c))
        return kl_backward<double>(c, scale, static_cast<double*>(dW), static_cast<double*>(dH),
                                   static_cast<double*>(dV));
    return kl_backward<float>(c, scale, static_cast<float*>(dW), static_cast<float*>(dH),
                              static_cast<float*>(dV));
}

int dna_get_choice(dna_ctx* c, int which, uint8_t* out, int64_t len) {
    if (int e = check_ready(c)) return e;
    if (!out || (which != 0 && which != 1) || len != (which ? c->N : c->T)) return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    if (cudaMemcpyAsync(out, which ? c->choice_w : c->choice_h, (size_t)len, cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess)
        return DNA_ERR_CUDA;
    return read_status(c);
}

int dna_get_costs(dna_ctx* c, int which, double* d_mu, double* d_dna, int64_t len) {
    if (int e = check_ready(c)) return e;
    if (!d_mu || !d_dna || (which != 0 && which != 1) || len != (which ? c->N : c->T))
        return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    const double* src = which ? c->dfin_w : c->dfin_h;
    if (cudaMemcpyAsync(d_mu, src, sizeof(double) * len, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_dna, src + len, sizeof(double) * len, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess)
        return DNA_ERR_CUDA;
    return read_status(c);
}

int dna_get_status(dna_ctx* c) {
    if (!c) return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    return read_status(c);
}

int dna_run_host(dna_ctx* c, const void* V, void* W, void* H, int iters, double* kl_out) {
    if (!c || !V || !W || !H || iters < 0) return DNA_ERR_ARG;
    if (c->sparse) return DNA_ERR_UNSUPPORTED;
    if (c->bound && !c->host_mode) return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    const size_t es = c->esz;
    const size_t bv = es * (size_t)(c->N * c->T), bw = es * (size_t)(c->N * c->R),
                 bh = es * (size_t)(c->R * c->T);
    if (!c->host_mode) {
        int e = DNA_OK;
        e |= dmalloc(&c->own_V, bv);
        e |= dmalloc(&c->own_W, bw);
        e |= dmalloc(&c->own_H, bh);
        if (e) return DNA_ERR_ALLOC;
        c->host_mode = true;
        c->V = c->own_V; c->ldv = c->T; c->W = c->own_W; c->H = c->own_H;
        c->bound = true;
        if (c->tc && (c->T % 4 != 0)) return DNA_ERR_UNSUPPORTED;  // rows must be 16-byte aligned
        if (c->tc)
            if (int e2 = build_tc_maps(c)) return e2;
    }
    cudaStream_t st = c->stream;
    // V in pinned (page-locked, device-mapped) host memory: the transpose-and-sums kernel
    // reads it across the host link and writes the device copy in the same pass; other
    // host memory: a copy first
    const void* vsrc = nullptr;
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, V) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer)
        vsrc = pa.devicePointer;
    cudaGetLastError();
    if ((!vsrc && cudaMemcpyAsync(c->own_V, V, bv, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        cudaMemcpyAsync(c->own_W, W, bw, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(c->own_H, H, bh, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return DNA_ERR_CUDA;
    int e = is_f64(c) ? prepare<double>(c, vsrc) : prepare<float>(c, vsrc);
    if (e) return e;
    if ((e = dna_iterate(c, iters))) return e;
    double kl = 0.0;
    if ((e = is_f64(c) ? kl_async<double>(c) : kl_async<float>(c))) return e;
    if (cudaMemcpyAsync(W, c->own_W, bw, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(H, c->own_H, bh, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&kl, c->kl_dev, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return DNA_ERR_CUDA;
    e = read_status(c);
    if (kl_out) *kl_out = kl;
    return e;
}

int dna_profile_phases(dna_ctx* c, unsigned mask) {
    if (!c) return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    if (mask && c->ev_pool.empty()) {
        c->ev_pool.resize(2 * 16384, nullptr);
        for (auto& ev : c->ev_pool)
            if (cudaEventCreate(&ev) != cudaSuccess) return DNA_ERR_CUDA;
    }
    mask &= (1u << DNA_NUM_PHASES) - 1u;
    if (mask != c->prof_mask) drop_graph(c);   // a captured graph holds the old mask's events
    c->prof_mask = mask;
    return DNA_OK;
}

int dna_profile(dna_ctx* c, int enable) {
    return dna_profile_phases(c, enable ? (1u << DNA_NUM_PHASES) - 1u : 0u);
}

int dna_phase_times(dna_ctx* c, double* ms, int64_t* launches, int n) {
    if (!c || n < 0 || n > DNA_NUM_PHASES) return DNA_ERR_ARG;
    if (set_device(c)) return DNA_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DNA_ERR_CUDA;
    for (const auto& rec : c->ev_recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, c->ev_pool[rec.second], c->ev_pool[rec.second + 1]) !=
            cudaSuccess)
            return DNA_ERR_CUDA;
        c->phase_ms[rec.first] += t;
    }
    c->ev_recs.clear();
    c->ev_used = 0;
    // graph replays: the captured phases' times of the last replay, once per replay
    if (c->graph_replays > 0)
        for (const auto& rec : c->graph_recs) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, c->graph_ev[rec.second], c->graph_ev[rec.second + 1]) !=
                cudaSuccess)
                return DNA_ERR_CUDA;
            c->phase_ms[rec.first] += (double)t * (double)c->graph_replays;
        }
    c->graph_replays = 0;
    for (int i = 0; i < n; ++i) {
        if (ms) ms[i] = c->phase_ms[i];
        if (launches) launches[i] = c->phase_launches[i];
    }
    for (int i = 0; i < DNA_NUM_PHASES; ++i) {
        c->phase_ms[i] = 0.0;
        c->phase_launches[i] = 0;
    }
    return DNA_OK;
}

void dna_destroy(dna_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
