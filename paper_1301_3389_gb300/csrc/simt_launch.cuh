// Host launchers for the SIMT kernels (instantiated for float and double).
#pragma once

#include <algorithm>

#include "glue_kernels.cuh"
#include "simt_kernels.cuh"
#include "sparse_kernels.cuh"

namespace dna {

namespace simt {

template <typename Tp> constexpr int rblock_for(int64_t R) {
    return sizeof(Tp) == 4 ? (R <= 32 ? 32 : (R <= 64 ? 64 : 128)) : (R <= 32 ? 32 : 64);
}

inline int launch_status() { return after_launch(); }

template <typename Kern>
inline int prep_smem(Kern k, size_t bytes) {
    static_assert(sizeof(Kern) > 0, "");
    if (bytes > 48 * 1024) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
            cudaSuccess)
            return DNA_ERR_CUDA;
    }
    return DNA_OK;
}

template <typename Tp, int RB>
int pass1_rb(const View& v, Tp* A, Tp* B, int splits, int64_t s_per, bool with_b, int* status,
             cudaStream_t st, double* dcur) {
    const size_t smem = Pass1Cfg<Tp, RB>::smem;
    dim3 grid((unsigned)((v.O + OB - 1) / OB), (unsigned)((v.R + RB - 1) / RB), (unsigned)splits);
    if (with_b) {
        auto k = k_pass1<Tp, RB, true>;
        if (prep_smem(k, smem)) return DNA_ERR_CUDA;
        k<<<grid, NT, smem, st>>>(v, A, B, s_per, status, dcur);
    } else {
        auto k = k_pass1<Tp, RB, false>;
        if (prep_smem(k, smem)) return DNA_ERR_CUDA;
        k<<<grid, NT, smem, st>>>(v, A, B, s_per, status, dcur);
    }
    return launch_status();
}

template <typename Tp, int RB, int NC, bool FULL>
int pass2_rb(const View& v, const Tp* X0, const Tp* X1, int64_t xr, int64_t xo, double* dpart,
             int splits, int64_t s_per, int* status, cudaStream_t st) {
    const size_t smem = Pass2Cfg<Tp, RB, NC>::smem;
    auto k = k_pass2<Tp, RB, NC, FULL>;
    if (prep_smem(k, smem)) return DNA_ERR_CUDA;
    dim3 grid((unsigned)((v.O + OB - 1) / OB), (unsigned)splits);
    k<<<grid, NT, smem, st>>>(v, X0, X1, xr, xo, dpart, s_per, status);
    return launch_status();
}

template <typename Tp, int NC, bool FULL>
int pass2_any(const View& v, const Tp* X0, const Tp* X1, int64_t xr, int64_t xo, double* dpart,
              int splits, int64_t s_per, int* status, cudaStream_t st) {
    switch (rblock_for<Tp>(v.R)) {
        case 32: return pass2_rb<Tp, 32, NC, FULL>(v, X0, X1, xr, xo, dpart, splits, s_per, status, st);
        case 64: return pass2_rb<Tp, 64, NC, FULL>(v, X0, X1, xr, xo, dpart, splits, s_per, status, st);
        default:
            if constexpr (sizeof(Tp) == 4)
                return pass2_rb<Tp, 128, NC, FULL>(v, X0, X1, xr, xo, dpart, splits, s_per, status, st);
            return DNA_ERR_UNSUPPORTED;
    }
}

template <typename Tp, int RB>
int occupancy_pass1() {
    int nb = 0;
    auto k = k_pass1<Tp, RB, true>;
    if (prep_smem(k, Pass1Cfg<Tp, RB>::smem)) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, Pass1Cfg<Tp, RB>::smem) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

template <typename Tp, int RB>
int occupancy_pass2() {
    int nb = 0;
    auto k = k_pass2<Tp, RB, 2, false>;
    if (prep_smem(k, Pass2Cfg<Tp, RB, 2>::smem)) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, Pass2Cfg<Tp, RB, 2>::smem) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace simt

namespace simt {
// sum over i < n of M(i, r) + reg -> out[r], M(i, r) at M[i * si + r * sr]: one CTA per r
// when rows are contiguous, else a two-level column sum through `work`
// (at least FSUM_SPLITS * R float64).
template <typename Tp>
int factor_sums(const Tp* M, int64_t n, int64_t R, int64_t si, int64_t sr, double reg,
                double* out, double* work, cudaStream_t st) {
    if (sr != 1 && si == 1) {
        k_row_sums<Tp><<<(unsigned)R, 256, 0, st>>>(M, n, sr, reg, out, true);
        return launch_status();
    }
    const int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>(FSUM_SPLITS, (n + 63) / 64));
    const int64_t rows_per = (n + nsplit - 1) / nsplit;
    dim3 blk(32, 8);
    dim3 grid((unsigned)((R + 31) / 32), (unsigned)nsplit);
    k_colsum_part<Tp><<<grid, blk, 0, st>>>(M, n, R, si, sr, rows_per, work);
    if (launch_status()) return DNA_ERR_CUDA;
    k_colsum_final<<<(unsigned)((R + 31) / 32), dim3(32, 32), 0, st>>>(work, (int)nsplit, R, reg, out,
                                                                      true);
    return launch_status();
}
}  // namespace simt

template <typename Tp>
int Simt<Tp>::factor_sums_y(const View& v, double reg, double* out, double* work,
                            cudaStream_t st) {
    return simt::factor_sums<Tp>(static_cast<const Tp*>(v.Y), v.S, v.R, v.ys, v.yr, reg, out,
                                 work, st);
}

template <typename Tp>
int Simt<Tp>::factor_sums_x(const View& v, double reg, double* out, double* work,
                            cudaStream_t st) {
    return simt::factor_sums<Tp>(static_cast<const Tp*>(v.X), v.O, v.R, v.xo, v.xr, reg, out,
                                 work, st);
}

template <typename Tp>
int Simt<Tp>::rescale(const View& v, const double* f, cudaStream_t st) {
    const int64_t rgroups = (v.R + 7) / 8;
    const int64_t longest = std::max(v.O, v.S);
    const int64_t bx = std::max<int64_t>(1, std::min<int64_t>(64, (longest + 511) / 512));
    dim3 grid((unsigned)bx, (unsigned)(2 * rgroups));
    simt::k_rescale<Tp><<<grid, dim3(32, 8), 0, st>>>(v, f, rgroups);
    return simt::launch_status();
}

template <typename Tp>
int Simt<Tp>::pass1(const View& v, Tp* A, Tp* B, int splits, int64_t s_per, bool with_b,
                    int* status, cudaStream_t st, double* dcur) {
    switch (simt::rblock_for<Tp>(v.R)) {
        case 32: return simt::pass1_rb<Tp, 32>(v, A, B, splits, s_per, with_b, status, st, dcur);
        case 64: return simt::pass1_rb<Tp, 64>(v, A, B, splits, s_per, with_b, status, st, dcur);
        default:
            if constexpr (sizeof(Tp) == 4)
                return simt::pass1_rb<Tp, 128>(v, A, B, splits, s_per, with_b, status, st, dcur);
            return DNA_ERR_UNSUPPORTED;
    }
}

template <typename Tp>
int Simt<Tp>::candidates(const View& v, const double* c, const Tp* A, const Tp* B, int splits,
                         Tp* Xmu, Tp* Xdna, double eps, double alpha, cudaStream_t st) {
    simt::k_candidates<Tp><<<(unsigned)((v.O + 31) / 32), dim3(32, 8), 0, st>>>(
        v, c, A, B, splits, Xmu, Xdna, (Tp)eps, (Tp)alpha);
    return simt::launch_status();
}

template <typename Tp>
int Simt<Tp>::mu_apply(const View& v, const double* c, const Tp* A, int splits, cudaStream_t st) {
    simt::k_mu_apply<Tp><<<(unsigned)((v.O + 127) / 128), 128, 0, st>>>(v, c, A, splits);
    return simt::launch_status();
}

template <typename Tp>
int Simt<Tp>::pass2(const View& v, const Tp* Xmu, const Tp* Xdna, double* dpart, int splits,
                    int64_t s_per, int* status, cudaStream_t st) {
    return simt::pass2_any<Tp, 2, false>(v, Xmu, Xdna, v.O, 1, dpart, splits, s_per, status, st);
}

template <typename Tp>
int Simt<Tp>::pass2_one(const View& v, const Tp* X, double* dpart, int splits, int64_t s_per,
                        int* status, cudaStream_t st) {
    return simt::pass2_any<Tp, 1, false>(v, X, X, v.O, 1, dpart, splits, s_per, status, st);
}

template <typename Tp>
int Simt<Tp>::select(const View& v, const Tp* Xmu, const Tp* Xdna, const double* dpart,
                     int splits, uint8_t* choice, double* dfin, double reg, cudaStream_t st) {
    simt::k_select<Tp><<<(unsigned)((v.O + 31) / 32), dim3(32, 8), 0, st>>>(
        v, Xmu, Xdna, dpart, splits, choice, dfin, reg);
    return simt::launch_status();
}

template <typename Tp>
int Simt<Tp>::kl_columns(const View& v, double* dpart, int splits, int64_t s_per, int* status,
                         cudaStream_t st) {
    const Tp* X = static_cast<const Tp*>(v.X);
    return simt::pass2_any<Tp, 1, true>(v, X, X, v.xr, v.xo, dpart, splits, s_per, status, st);
}

template <typename Tp>
int Simt<Tp>::grad_x(const View& v, const double* c, const Tp* A, int splits, double scale,
                     Tp* G, int64_t gr, int64_t go, cudaStream_t st) {
    simt::k_grad_x<Tp><<<(unsigned)((v.O + 31) / 32), dim3(32, 8), 0, st>>>(v, c, A, splits, scale,
                                                                           G, gr, go);
    return simt::launch_status();
}

namespace simt {
template <typename Tp, int RB>
int grad_v_rb(const View& v, double scale, Tp* dV, int64_t ldd, int* status, cudaStream_t st) {
    const size_t smem = (size_t)(2 * RB * LD) * sizeof(Tp);
    auto k = k_grad_v<Tp, RB>;
    if (prep_smem(k, smem)) return DNA_ERR_CUDA;
    dim3 grid((unsigned)((v.O + OB - 1) / OB), (unsigned)((v.S + SB - 1) / SB));
    k<<<grid, NT, smem, st>>>(v, scale, dV, ldd, status);
    return launch_status();
}
}  // namespace simt

template <typename Tp>
int Simt<Tp>::grad_v(const View& v, double scale, Tp* dV, int64_t ldd, int* status,
                     cudaStream_t st) {
    switch (simt::rblock_for<Tp>(v.R)) {
        case 32: return simt::grad_v_rb<Tp, 32>(v, scale, dV, ldd, status, st);
        case 64: return simt::grad_v_rb<Tp, 64>(v, scale, dV, ldd, status, st);
        default:
            if constexpr (sizeof(Tp) == 4) return simt::grad_v_rb<Tp, 128>(v, scale, dV, ldd, status, st);
            return DNA_ERR_UNSUPPORTED;
    }
}

namespace simt {
template <typename Tp, int RB>
int adj_gemm_rb(const View& v, const Tp* Abar, const Tp* Bbar, const double* vs, Tp* Hpart,
                int splits, int64_t s_per, Tp* Vbar, int64_t ldvb, int* status, cudaStream_t st) {
    const size_t smem = AdjCfg<Tp, RB>::smem;
    auto k = k_adj_gemm<Tp, RB>;
    if (prep_smem(k, smem)) return DNA_ERR_CUDA;
    dim3 grid((unsigned)((v.O + OB - 1) / OB), (unsigned)splits);
    k<<<grid, NT, smem, st>>>(v, Abar, Bbar, vs, Hpart, Vbar, ldvb, s_per, status);
    return launch_status();
}
}  // namespace simt

template <typename Tp>
int Simt<Tp>::adjoint_h(const View& v, const double* c, const Tp* Apart, const Tp* Bpart,
                        int splits1, const uint8_t* choice, const Tp* Hbar1, Tp* Hbar0, Tp* Abar,
                        Tp* Bbar, double* vs, Tp* Hpart, int splits2, int64_t s_per2, Tp* Vbar,
                        int64_t ldvb, double eps, double alpha, int* status, cudaStream_t st,
                        double* cpart) {
    simt::k_adj_elem<Tp><<<(unsigned)((v.O + 31) / 32), dim3(32, 8), 0, st>>>(
        v, c, Apart, Bpart, splits1, choice, Hbar1, Hbar0, Abar, Bbar, vs, (Tp)eps, (Tp)alpha,
        cpart);
    if (simt::launch_status()) return DNA_ERR_CUDA;
    int e;
    switch (simt::rblock_for<Tp>(v.R)) {
        case 32: e = simt::adj_gemm_rb<Tp, 32>(v, Abar, Bbar, vs, Hpart, splits2, s_per2, Vbar, ldvb, status, st); break;
        case 64: e = simt::adj_gemm_rb<Tp, 64>(v, Abar, Bbar, vs, Hpart, splits2, s_per2, Vbar, ldvb, status, st); break;
        default:
            if constexpr (sizeof(Tp) == 4) {
                if (v.R <= 128) {
                    e = simt::adj_gemm_rb<Tp, 128>(v, Abar, Bbar, vs, Hpart, splits2, s_per2, Vbar, ldvb, status, st);
                    break;
                }
            }
            return DNA_ERR_UNSUPPORTED;
    }
    if (e) return e;
    simt::k_adj_combine<Tp><<<(unsigned)((v.O + 31) / 32), dim3(32, 8), 0, st>>>(v, Hpart, splits2,
                                                                                 Hbar0);
    return simt::launch_status();
}

namespace simt {
template <typename Tp, int RB>
int adj_wgrad_rb(const View& v, const Tp* Abar, const Tp* Bbar, Tp* Wpart, int wsplits,
                 int64_t o_per, int* status, cudaStream_t st) {
    const size_t smem = WgradCfg<Tp, RB>::smem;
    auto k = k_adj_wgrad<Tp, RB>;
    if (prep_smem(k, smem)) return DNA_ERR_CUDA;
    dim3 grid((unsigned)((v.S + SB - 1) / SB), (unsigned)wsplits);
    k<<<grid, NT, smem, st>>>(v, Abar, Bbar, Wpart, o_per, status);
    return launch_status();
}
}  // namespace simt

template <typename Tp>
int Simt<Tp>::adjoint_w(const View& v, const Tp* Abar, const Tp* Bbar, const double* cpart,
                        Tp* Wpart, int wsplits, int64_t o_per, Tp* Wbar, int* status,
                        cudaStream_t st) {
    if (v.R > 128 || o_per % simt::OB) return DNA_ERR_UNSUPPORTED;
    int e;
    switch (simt::rblock_for<Tp>(v.R)) {
        case 32: e = simt::adj_wgrad_rb<Tp, 32>(v, Abar, Bbar, Wpart, wsplits, o_per, status, st); break;
        case 64: e = simt::adj_wgrad_rb<Tp, 64>(v, Abar, Bbar, Wpart, wsplits, o_per, status, st); break;
        default:
            if constexpr (sizeof(Tp) == 4) {
                e = simt::adj_wgrad_rb<Tp, 128>(v, Abar, Bbar, Wpart, wsplits, o_per, status, st);
                break;
            }
            return DNA_ERR_UNSUPPORTED;
    }
    if (e) return e;
    simt::k_adj_wcombine<Tp><<<(unsigned)((v.S + 31) / 32), dim3(32, 8), 0, st>>>(
        v, Wpart, wsplits, cpart, (v.O + 31) / 32, Wbar);
    return simt::launch_status();
}

template <typename Tp>
int64_t Simt<Tp>::glue_parts(int64_t n) { return (n + glue::TO - 1) / glue::TO; }

template <typename Tp>
int Simt<Tp>::cand_fused(const View& v, const double* c, const Tp* A, const Tp* B, int splits,
                         Tp* Xmu, Tp* Xdna, double eps, double alpha, void* Xmk, void* Xdk,
                         int64_t rp, int64_t O_pad, int64_t plane, cudaStream_t st) {
    const bool bf = Xmk != nullptr;
    if (bf && (sizeof(Tp) != 4 || !Xdk || rp < v.R || rp % 2 != 0 || O_pad < v.O))
        return DNA_ERR_ARG;
    const unsigned grid = (unsigned)((bf ? O_pad : v.O) + glue::TO - 1) / glue::TO;
    if (cand_in_registers(v.R) && (!bf || rp <= 16 * (v.R <= 128 ? 8 : 16))) {
        // candidates of a thread in registers, at most 16 groups of r
        const int rs = v.R <= 128 ? 8 : 16;
        const int64_t rows = std::max<int64_t>((v.R + rs - 1) / rs, bf ? (rp + rs - 1) / rs : 0);
        const dim3 blk(32, (unsigned)rows);
        if (bf && rp % 8 != 0) return DNA_ERR_ARG;
        if (bf) {
            if constexpr (sizeof(Tp) == 4) {
                auto* bm = static_cast<glue::bf16*>(Xmk);
                auto* bd = static_cast<glue::bf16*>(Xdk);
                if (rs == 8)
                    glue::k_cand_reg<Tp, true, 8><<<grid, blk, 0, st>>>(
                        v, c, A, B, splits, Xmu, Xdna, (Tp)eps, (Tp)alpha, bm, bd, rp, plane);
                else
                    glue::k_cand_reg<Tp, true, 16><<<grid, blk, 0, st>>>(
                        v, c, A, B, splits, Xmu, Xdna, (Tp)eps, (Tp)alpha, bm, bd, rp, plane);
            }
        } else if (rs == 8) {
            glue::k_cand_reg<Tp, false, 8><<<grid, blk, 0, st>>>(
                v, c, A, B, splits, Xmu, Xdna, (Tp)eps, (Tp)alpha, nullptr, nullptr, 0, 0);
        } else {
            glue::k_cand_reg<Tp, false, 16><<<grid, blk, 0, st>>>(
                v, c, A, B, splits, Xmu, Xdna, (Tp)eps, (Tp)alpha, nullptr, nullptr, 0, 0);
        }
        return simt::launch_status();
    }
    const size_t smem = glue::cand_smem<Tp>(v.R, bf);
    if (bf) {
        if constexpr (sizeof(Tp) == 4) {
            auto k = glue::k_cand_fused<Tp, true>;
            if (simt::prep_smem(k, smem)) return DNA_ERR_CUDA;
            k<<<grid, dim3(32, glue::TY), smem, st>>>(v, c, A, B, splits, Xmu, Xdna, (Tp)eps, (Tp)alpha,
                                               static_cast<glue::bf16*>(Xmk),
                                               static_cast<glue::bf16*>(Xdk), rp, plane);
        }
    } else {
        auto k = glue::k_cand_fused<Tp, false>;
        if (simt::prep_smem(k, smem)) return DNA_ERR_CUDA;
        k<<<grid, dim3(32, glue::TY), smem, st>>>(v, c, A, B, splits, Xmu, Xdna, (Tp)eps, (Tp)alpha,
                                           nullptr, nullptr, 0, 0);
    }
    return simt::launch_status();
}

template <typename Tp>
bool Simt<Tp>::cand_in_registers(int64_t R) { return R <= (sizeof(Tp) == 8 ? 128 : 256); }

template <typename Tp>
int Simt<Tp>::split_sum(Tp* A, Tp* B, int64_t R, int64_t O, int splits, cudaStream_t st) {
    if (splits <= 1) return DNA_OK;
    const int64_t n = R * O;
    const int64_t work = (sizeof(Tp) == 4 && n % 4 == 0) ? n / 4 : n;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 8));
    glue::k_split_sum<Tp><<<(unsigned)blocks, 256, 0, st>>>(A, B, n, splits);
    return simt::launch_status();
}

template <typename Tp>
int Simt<Tp>::select_fused(const View& v, const Tp* Xmu, const Tp* Xdna, const double* dpart,
                           int splits, uint8_t* choice, double* dfin, double* fpart,
                           double reg, cudaStream_t st, const double* dcur, int cur_splits) {
    const size_t smem = glue::select_smem<Tp>(v.R);
    auto k = glue::k_select_fused<Tp>;
    if (simt::prep_smem(k, smem)) return DNA_ERR_CUDA;
    k<<<(unsigned)glue_parts(v.O), dim3(32, 8), smem, st>>>(v, Xmu, Xdna, dpart, splits, choice,
                                                           dfin, fpart, reg, dcur, cur_splits);
    return simt::launch_status();
}

template <typename Tp>
int Simt<Tp>::mu_fused(const View& v, const double* c, const Tp* A, int splits, double* fpart,
                       cudaStream_t st) {
    const size_t smem = glue::select_smem<Tp>(v.R);
    auto k = glue::k_mu_fused<Tp>;
    if (simt::prep_smem(k, smem)) return DNA_ERR_CUDA;
    k<<<(unsigned)glue_parts(v.O), dim3(32, 8), smem, st>>>(v, c, A, splits, fpart);
    return simt::launch_status();
}

template <typename Tp>
int Simt<Tp>::part_sums(const double* part, int64_t nparts, int64_t R, double reg, double* out,
                        cudaStream_t st, double* next) {
    if (R <= 1024)   // a CTA per r: latency of one load round and a tree, not of nparts / 32
        simt::k_colsum_small<0><<<(unsigned)R, 256, 0, st>>>(part, (int)nparts, R, reg, out, true,
                                                             next);
    else
        simt::k_colsum_final<<<(unsigned)((R + 31) / 32), dim3(32, 32), 0, st>>>(
            part, (int)nparts, R, reg, out, true, next);
    return simt::launch_status();
}

template <typename Tp>
int Simt<Tp>::scale_ops(const View& t, const double* f, bool xmul, void* Xk, void* Yk, void* Ytk,
                        void* Y2tk, int64_t rp, int64_t O_pad, int64_t S_pad, int64_t plane,
                        double* cpart, cudaStream_t st) {
    const bool bf = Xk != nullptr;
    if (bf && (sizeof(Tp) != 4 || !Yk || !Ytk || rp < t.R || O_pad < t.O || S_pad < t.S))
        return DNA_ERR_ARG;
    glue::OpsArgs a{};
    a.X = t.X; a.xr = t.xr; a.xo = t.xo; a.O = t.O;
    a.Y = const_cast<void*>(t.Y); a.ys = t.ys; a.yr = t.yr; a.S = t.S;
    a.R = t.R; a.f = f; a.xmul = xmul;
    a.Xk = static_cast<glue::bf16*>(Xk); a.Yk = static_cast<glue::bf16*>(Yk);
    a.Ytk = static_cast<glue::bf16*>(Ytk); a.Y2tk = static_cast<glue::bf16*>(Y2tk);
    a.rp = rp; a.O_pad = O_pad; a.S_pad = S_pad; a.plane = bf ? plane : 0; a.cpart = cpart;
    const int64_t rcov = bf ? rp : t.R, ocov = bf ? O_pad : t.O, scov = bf ? S_pad : t.S;
    const int rt = rcov <= 32 ? 32 : rcov <= 64 ? 64 : 128;   // values of r per tile
    a.tiles_r = (rcov + rt - 1) / rt;
    // without scaling and operands the X tiles have nothing to do
    a.xtiles_o = (f || bf) ? glue_parts(ocov) : 0;
    a.xtiles = a.xtiles_o * a.tiles_r;
    const int64_t ytiles = (f || bf || cpart) ? glue_parts(scov) * a.tiles_r : 0;
    const int64_t blocks = a.xtiles + ytiles;
    if (blocks == 0) return DNA_OK;
    if (rt == 32)
        glue::k_scale_ops<Tp, 32><<<(unsigned)blocks, dim3(32, 8), 0, st>>>(a);
    else if (rt == 64)
        glue::k_scale_ops<Tp, 64><<<(unsigned)blocks, dim3(32, 8), 0, st>>>(a);
    else
        glue::k_scale_ops<Tp, 128><<<(unsigned)blocks, dim3(32, 8), 0, st>>>(a);
    return simt::launch_status();
}

template <typename Tp>
int Simt<Tp>::prepare_v(const Tp* V, int64_t N, int64_t T, int64_t ldv, Tp* Vt, int64_t ldvt,
                        double* colsum, double* rowsum, cudaStream_t st, double* part, Tp* Vc) {
    dim3 blk(32, 8);
    dim3 grid((unsigned)((T + 31) / 32), (unsigned)((N + 31) / 32));
    if (Vc && !part) return DNA_ERR_ARG;
    if (part) {   // one pass over V: transpose and per-tile sums, then the float64 totals
        double* colpart = part;                                // [ceil(N / 32)][T]
        double* rowpart = part + (size_t)((N + 31) / 32) * T;  // [ceil(T / 32)][N]
        simt::k_transpose_sums<Tp><<<grid, blk, 0, st>>>(V, N, T, ldv, Vt, ldvt, colpart, rowpart,
                                                         Vc);
        if (simt::launch_status()) return DNA_ERR_CUDA;
        simt::k_colsum_final<<<(unsigned)((T + 31) / 32), dim3(32, 32), 0, st>>>(
            colpart, (int)((N + 31) / 32), T, 0.0, colsum, false);
        if (simt::launch_status()) return DNA_ERR_CUDA;
        simt::k_colsum_final<<<(unsigned)((N + 31) / 32), dim3(32, 32), 0, st>>>(
            rowpart, (int)((T + 31) / 32), N, 0.0, rowsum, false);
        return simt::launch_status();
    }
    simt::k_transpose<Tp><<<grid, blk, 0, st>>>(V, N, T, ldv, Vt, ldvt);
    if (simt::launch_status()) return DNA_ERR_CUDA;
    // column sums of V: sum over n of V[n][t]  (coalesced across t)
    simt::k_factor_sums<Tp><<<(unsigned)((T + 31) / 32), blk, 0, st>>>(V, N, T, ldv, 1, 0.0, colsum,
                                                                             false);
    if (simt::launch_status()) return DNA_ERR_CUDA;
    // row sums of V: rows are contiguous
    simt::k_row_sums<Tp><<<(unsigned)N, 256, 0, st>>>(V, T, ldv, 0.0, rowsum, false);
    return simt::launch_status();
}

template <typename Tp>
int Simt<Tp>::pass1_blocks_per_sm(int64_t R) {
    switch (simt::rblock_for<Tp>(R)) {
        case 32: return simt::occupancy_pass1<Tp, 32>();
        case 64: return simt::occupancy_pass1<Tp, 64>();
        default:
            if constexpr (sizeof(Tp) == 4) return simt::occupancy_pass1<Tp, 128>();
            return 1;
    }
}

template <typename Tp>
int Simt<Tp>::pass2_blocks_per_sm(int64_t R) {
    switch (simt::rblock_for<Tp>(R)) {
        case 32: return simt::occupancy_pass2<Tp, 32>();
        case 64: return simt::occupancy_pass2<Tp, 64>();
        default:
            if constexpr (sizeof(Tp) == 4) return simt::occupancy_pass2<Tp, 128>();
            return 1;
    }
}

template <typename Tp> int Simt<Tp>::chunk() { return simt::SB; }
template <typename Tp> int Simt<Tp>::oblock() { return simt::OB; }
template <typename Tp> int Simt<Tp>::rblock(int64_t R) { return simt::rblock_for<Tp>(R); }

template <typename Tp>
int Simt<Tp>::add_reg(const double* in, int64_t R, double reg, double* out, cudaStream_t st) {
    glue::k_add_reg<0><<<(unsigned)((R + 255) / 256), 256, 0, st>>>(in, R, reg, out);
    return simt::launch_status();
}

template <typename Tp>
int Simt<Tp>::raw_sums(const double* part, int64_t nparts, int64_t R, double* out,
                       cudaStream_t st) {
    if (R <= 1024)
        simt::k_colsum_small<0><<<(unsigned)R, 256, 0, st>>>(part, (int)nparts, R, 0.0, out, false);
    else
        simt::k_colsum_final<<<(unsigned)((R + 31) / 32), dim3(32, 32), 0, st>>>(
            part, (int)nparts, R, 0.0, out, false);
    return simt::launch_status();
}

namespace simt {
inline unsigned sp_grid(int64_t n) { return (unsigned)((n + sparse::WARPS - 1) / sparse::WARPS); }

template <typename Tp, int RPL>
int sp_pass1_r(const View& v, const SparseSegs& sg, const int32_t* idx, const Tp* val,
               const Tp* Yg, Tp* Aseg, Tp* Bseg, Tp* A, Tp* B, bool with_b, int* status,
               cudaStream_t st) {
    if (sg.n > 0) {
        sparse::k_sp_pass1<Tp, RPL><<<sp_grid(sg.n), sparse::WARPS * 32, 0, st>>>(
            v, sg, idx, val, Yg, Aseg, Bseg, with_b, status);
        if (launch_status()) return DNA_ERR_CUDA;
    }
    sparse::k_sp_reduce_ab<Tp, RPL><<<sp_grid(v.O), sparse::WARPS * 32, 0, st>>>(
        v.O, v.R, sg.sptr, Aseg, Bseg, A, B, with_b);
    return launch_status();
}
template <typename Tp, int RPL>
int sp_pass2_r(const View& v, const SparseSegs& sg, const int32_t* idx, const Tp* val,
               const Tp* Yg, const Tp* Xmu, const Tp* Xdna, const double* c0, double* dseg,
               double* dpart, int* status, cudaStream_t st) {
    if (sg.n > 0) {
        sparse::k_sp_pass2<Tp, RPL><<<sp_grid(sg.n), sparse::WARPS * 32, 0, st>>>(
            v, sg, idx, val, Yg, Xmu, Xdna, dseg);
        if (launch_status()) return DNA_ERR_CUDA;
    }
    sparse::k_sp_reduce_cost<Tp, RPL><<<sp_grid(v.O), sparse::WARPS * 32, 0, st>>>(
        v.O, v.R, sg.sptr, dseg, Xmu, Xdna, c0, dpart, status);
    return launch_status();
}
template <typename Tp, int RPL>
int sp_kl_r(const View& v, const SparseSegs& sg, const int32_t* idx, const Tp* val,
            const Tp* Yg, const double* c0, double* dseg, double* part, int* status,
            cudaStream_t st) {
    if (sg.n > 0) {
        sparse::k_sp_kl<Tp, RPL><<<sp_grid(sg.n), sparse::WARPS * 32, 0, st>>>(v, sg, idx, val,
                                                                               Yg, dseg);
        if (launch_status()) return DNA_ERR_CUDA;
    }
    sparse::k_sp_reduce_kl<Tp, RPL><<<sp_grid(v.O), sparse::WARPS * 32, 0, st>>>(
        v, sg.sptr, dseg, c0, part, status);
    return launch_status();
}
}  // namespace simt

template <typename Tp>
int Simt<Tp>::sp_pass1(const View& v, const SparseSegs& sg, const int32_t* idx, const Tp* val,
                       const Tp* Yg, Tp* Aseg, Tp* Bseg, Tp* A, Tp* B, bool with_b, int* status,
                       cudaStream_t st) {
    if (v.R <= 32) return simt::sp_pass1_r<Tp, 1>(v, sg, idx, val, Yg, Aseg, Bseg, A, B, with_b, status, st);
    if (v.R <= 64) return simt::sp_pass1_r<Tp, 2>(v, sg, idx, val, Yg, Aseg, Bseg, A, B, with_b, status, st);
    if (v.R <= 128) return simt::sp_pass1_r<Tp, 4>(v, sg, idx, val, Yg, Aseg, Bseg, A, B, with_b, status, st);
    return DNA_ERR_UNSUPPORTED;
}

template <typename Tp>
int Simt<Tp>::sp_pass2(const View& v, const SparseSegs& sg, const int32_t* idx, const Tp* val,
                       const Tp* Yg, const Tp* Xmu, const Tp* Xdna, const double* c0,
                       double* dseg, double* dpart, int* status, cudaStream_t st) {
    if (v.R <= 32) return simt::sp_pass2_r<Tp, 1>(v, sg, idx, val, Yg, Xmu, Xdna, c0, dseg, dpart, status, st);
    if (v.R <= 64) return simt::sp_pass2_r<Tp, 2>(v, sg, idx, val, Yg, Xmu, Xdna, c0, dseg, dpart, status, st);
    if (v.R <= 128) return simt::sp_pass2_r<Tp, 4>(v, sg, idx, val, Yg, Xmu, Xdna, c0, dseg, dpart, status, st);
    return DNA_ERR_UNSUPPORTED;
}

template <typename Tp>
int Simt<Tp>::sp_kl(const View& v, const SparseSegs& sg, const int32_t* idx, const Tp* val,
                    const Tp* Yg, const double* c0, double* dseg, double* part, int* status,
                    cudaStream_t st) {
    if (v.R <= 32) return simt::sp_kl_r<Tp, 1>(v, sg, idx, val, Yg, c0, dseg, part, status, st);
    if (v.R <= 64) return simt::sp_kl_r<Tp, 2>(v, sg, idx, val, Yg, c0, dseg, part, status, st);
    if (v.R <= 128) return simt::sp_kl_r<Tp, 4>(v, sg, idx, val, Yg, c0, dseg, part, status, st);
    return DNA_ERR_UNSUPPORTED;
}

template <typename Tp>
int Simt<Tp>::transpose(const Tp* in, int64_t rows, int64_t cols, Tp* out, cudaStream_t st) {
    const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    sparse::k_transpose<Tp><<<grid, dim3(32, 8), 0, st>>>(in, rows, cols, out);
    return simt::launch_status();
}

}  // namespace dna
