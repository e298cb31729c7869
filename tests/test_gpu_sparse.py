"""The sparse-V form (dna_create_sparse / dna_bind_csr) against the FP64 oracle.

The oracle is the dense one applied to V with its zeros written out: the sparse kernels
must give the same half-steps, because zeros contribute nothing to A, B (eq. 7, 14) or to
the -v log z part of the costs, and sum_n z = sum_r (sum_n w_nr) h_r (the note after
Algorithm 1).  Tolerances are those of the dense FP32 / FP64 forms (test_gpu_parity.py):
W and H within 1e-4 (FP32) / 1e-10 (FP64) relative per iteration with selections replayed
at near ties, the one-step element-wise bound of gpu_helpers.step_elementwise on every
half-step, d_KL within 1e-4 (FP32) / 1e-10 (FP64).
"""
import numpy as np
import pytest

import workloads
from gpu_helpers import SparseGpuProblem, rel_fro, replay_choice, step_elementwise, step_pair
from oracle import dna as o

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f64": 1e-10}

# (N, T, R, density): several warps' worth of columns, ragged ranks per lane class
# (R <= 32, <= 64, <= 128), a dense-ish and a very sparse case
CASES = [(300, 500, 16, 0.05), (97, 131, 33, 0.2), (200, 150, 128, 0.1), (500, 400, 64, 0.01),
         (64, 64, 1, 0.3)]


def _sparse_case(N, T, R, density, seed):
    sp = workloads.sparse_custom(N, T, R, density, seed=seed)
    return sp, sp.dense()


@pytest.mark.parametrize("kind", ["f32", "f64"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[:3])) + f"@{c[3]}")
def test_sparse_trajectory_matches_oracle(case, kind):
    N, T, R, density = case
    sp, V = _sparse_case(N, T, R, density, seed=N + T + R)
    with SparseGpuProblem(sp, kind, V_dense=V) as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(sp.W, sp.H)
        for it in range(3):
            for which in (0, 1):
                W, H, _ = step_pair(gp, W, H, which)   # includes the element-wise bound
                Wg, Hg = gp.WH()
                assert rel_fro(Wg, W) < TOL[kind] and rel_fro(Hg, H) < TOL[kind], (it, which)
        kl = gp.dna.dna_kl(gp.ctx)
        ref = o.kl_divergence(V, W @ H)
        assert abs(kl - ref) <= TOL[kind] * abs(ref), (kl, ref)


@pytest.mark.parametrize("kind", ["f32", "f64"])
def test_sparse_mu_and_regularised(kind):
    """MU iterations (eq. 11) and DNA with lambda, rho > 0 on a sparse V."""
    sp, V = _sparse_case(150, 220, 12, 0.08, seed=5)
    with SparseGpuProblem(sp, kind, V_dense=V) as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(sp.W, sp.H)
        for _ in range(3):
            W, H = o.mu_iteration(V, W, H)
        gp.dna.mu_iterate(gp.ctx, 3)
        Wg, Hg = gp.WH()
        assert rel_fro(Wg, W) < TOL[kind] and rel_fro(Hg, H) < TOL[kind]
    opts = {"rho": 0.3, "lam": 0.5}
    with SparseGpuProblem(sp, kind, V_dense=V, rho=0.3, lam=0.5) as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(sp.W, sp.H, 0.5)
        for _ in range(2):
            for which in (0, 1):
                W, H, _ = step_pair(gp, W, H, which, opts=opts)
                Wg, Hg = gp.WH()
                assert rel_fro(Wg, W) < TOL[kind] and rel_fro(Hg, H) < TOL[kind]


def test_sparse_equals_dense_path_f64():
    """The sparse kernels and the dense FP64 kernels agree on the same data (to rounding)."""
    from gpu_helpers import GpuProblem
    sp, V = _sparse_case(180, 260, 20, 0.06, seed=9)
    with SparseGpuProblem(sp, "f64", V_dense=V) as gs:
        gs.dna.dna_normalize(gs.ctx, 1)
        gs.dna.dna_iterate(gs.ctx, 3)
        Ws, Hs = gs.WH()
        kls = gs.dna.dna_kl(gs.ctx)
    with GpuProblem(V.astype(np.float32), sp.W, sp.H, "f64") as gd:
        gd.dna.dna_normalize(gd.ctx, 1)
        gd.dna.dna_iterate(gd.ctx, 3)
        Wd, Hd = gd.WH()
        kld = gd.dna.dna_kl(gd.ctx)
    assert rel_fro(Ws, Wd) < 1e-11 and rel_fro(Hs, Hd) < 1e-11
    assert abs(kls - kld) <= 1e-11 * abs(kld)


def test_sparse_explicit_zeros_and_empty_lines():
    """Stored zeros, an empty row and an empty column of V: q = 0 there, the empty column of
    H goes to 0, and the results equal those of the same matrix without the stored zeros."""
    sp, V = _sparse_case(90, 120, 8, 0.1, seed=13)
    V[5, :] = 0
    V[:, 7] = 0
    rows, cols = np.nonzero(V)
    # store every non-zero plus ten explicit zeros
    extra_r, extra_c = np.array([1, 2, 3, 4, 6, 8, 9, 10, 11, 12]), np.arange(10) + 20
    keep = V[extra_r, extra_c] == 0
    r_all = np.concatenate([rows, extra_r[keep]])
    c_all = np.concatenate([cols, extra_c[keep]])
    order = np.lexsort((c_all, r_all))
    r_all, c_all = r_all[order], c_all[order]
    vals = V[r_all, c_all].astype(np.float32)
    row_ptr = np.zeros(91, dtype=np.int64)
    np.add.at(row_ptr, r_all + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    sz = workloads.SparseProblem("z", 90, 120, row_ptr, c_all.astype(np.int32), vals, sp.W, sp.H, 0)
    with SparseGpuProblem(sz, "f64", V_dense=V) as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(sp.W, sp.H)
        for which in (0, 1, 0, 1):
            W, H, _ = step_pair(gp, W, H, which)
        Wg, Hg = gp.WH()
        assert rel_fro(Wg, W) < 1e-10 and rel_fro(Hg, H) < 1e-10
        assert np.all(Hg[:, 7] == 0)


def test_sparse_rejects_bad_input_and_reports_nonfinite():
    import torch

    import paper_1301_3389_gb300 as dna
    sp, V = _sparse_case(40, 50, 4, 0.2, seed=3)
    with pytest.raises(dna.DNAError) as e:
        dna.dna_create_sparse(40, 50, 200, sp.nnz)
    assert e.value.code == dna.DNA_ERR_UNSUPPORTED
    ctx = dna.dna_create_sparse(40, 50, 4, sp.nnz)
    try:
        W = torch.from_numpy(sp.W).cuda()
        H = torch.from_numpy(sp.H).cuda()
        bad = sp.col_idx.copy()
        bad[3] = 50                                          # column out of range
        with pytest.raises(dna.DNAError) as e:
            dna.dna_bind_csr(ctx, torch.from_numpy(sp.row_ptr).cuda(),
                             torch.from_numpy(bad).cuda(), torch.from_numpy(sp.vals).cuda(), W, H)
        assert e.value.code == dna.DNA_ERR_ARG
        neg = sp.vals.copy()
        neg[0] = -1.0                                        # V must be non-negative
        with pytest.raises(dna.DNAError) as e:
            dna.dna_bind_csr(ctx, torch.from_numpy(sp.row_ptr).cuda(),
                             torch.from_numpy(sp.col_idx).cuda(), torch.from_numpy(neg).cuda(), W, H)
        assert e.value.code == dna.DNA_ERR_ARG
    finally:
        dna.dna_destroy(ctx)
    sp2 = workloads.SparseProblem("z", 40, 50, sp.row_ptr, sp.col_idx, sp.vals,
                                  np.zeros_like(sp.W), sp.H, 0)
    with SparseGpuProblem(sp2, "f32") as gp:               # z = 0 where v > 0
        gp.dna.dna_step_H(gp.ctx)
        assert gp.dna.dna_get_status(gp.ctx) == dna.DNA_ERR_NONFINITE


def test_sparse_tdt2_size_sampled():
    """The TDT2-shaped workload (36771 x 10212, 0.35 % non-zeros, R = 64): one H and one W
    half-step against the oracle on sampled columns and rows (each separates exactly,
    eq. 5), the step 16 / 29 factor read from the GPU."""
    import dataclasses
    sp = workloads.sparse_tdt2(0)
    g = np.random.default_rng(3)
    cols = np.sort(g.choice(sp.T, 40, replace=False))
    rows = np.sort(g.choice(sp.N, 40, replace=False))
    rr = np.repeat(np.arange(sp.N), np.diff(sp.row_ptr))
    Vc = np.zeros((sp.N, cols.size))
    pos = {int(t): i for i, t in enumerate(cols)}
    m = np.isin(sp.col_idx, cols)
    Vc[rr[m], [pos[int(t)] for t in sp.col_idx[m]]] = sp.vals[m]
    Vr = np.zeros((rows.size, sp.T))
    for i, n in enumerate(rows):
        a, b = sp.row_ptr[n], sp.row_ptr[n + 1]
        Vr[i, sp.col_idx[a:b]] = sp.vals[a:b]
    with SparseGpuProblem(sp, "f32") as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W0, H0 = gp.WH()
        gp.dna.dna_step_H(gp.ctx)
        W1, H1 = gp.WH()
        half = o.h_half_step(Vc, W0, H0[:, cols])
        mask, _ = replay_choice(half, gp.choice(0)[cols], "f32")
        X = np.where(mask[None, :], half.X_dna, half.X_mu)
        sigma = W1.sum(axis=0) / W0.sum(axis=0)
        assert rel_fro(H1[:, cols], X / sigma[:, None]) < 1e-4
        assert step_elementwise(dataclasses.replace(half, choice=mask), 0, W0, H0[:, cols], W1,
                                H1[:, cols], "f32", sig=sigma, check_y=False) <= 1.0
        gp.dna.dna_step_W(gp.ctx)
        W2, H2 = gp.WH()
        half = o.w_half_step(Vr, W1[rows, :], H1)
        mask, _ = replay_choice(half, gp.choice(1)[rows], "f32")
        X = np.where(mask[:, None], half.X_dna, half.X_mu)
        sigma = H2.sum(axis=1) / H1.sum(axis=1)
        assert rel_fro(W2[rows, :], X / sigma[None, :]) < 1e-4
        assert step_elementwise(dataclasses.replace(half, choice=mask), 1, W1[rows, :], H1,
                                W2[rows, :], H2, "f32", sig=sigma, check_y=False) <= 1.0
