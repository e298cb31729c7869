"""The FP32 form on the tensor cores (DNA_ENGINE_TENSOR with DNA_F32): every float32
operand is split into bf16 hi + lo planes and every product is x_hi y_hi + x_hi y_lo +
x_lo y_hi with float32 accumulation.  Held to the FP32 form's tolerances against the FP64
oracle (W, H within 1e-4 relative per half-step).  The trajectory, final-d_KL, ragged-size
and regularised checks are in test_gpu_parity.py and the bench-size sampled check in
test_gpu_fullsize.py, parametrised over the CUDA-core and tensor-core FP32 forms.
"""
import numpy as np
import pytest

import workloads
from gpu_helpers import ELEM_TOL, SPLIT_LARGE_R_TOL, GpuProblem, rel_elem, rel_fro, step_pair
from oracle import dna as o

pytestmark = pytest.mark.gpu

SHAPES = [(64, 128, 8), (300, 500, 100), (257, 300, 128), (640, 130, 64), (129, 257, 33)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_split_half_steps(shape):
    """Two DNA iterations from the oracle's state: each half-step within 1e-4 relative."""
    N, T, R = shape
    p = workloads.custom(N, T, R, seed=N + 5 * T + 11 * R)
    with GpuProblem(p.V, p.W, p.H, "f32t") as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(p.W, p.H)
        worst = 0.0
        for _ in range(2):
            for which in (0, 1):
                W, H, _ = step_pair(gp, W, H, which)
                Wg, Hg = gp.WH()
                worst = max(worst, rel_fro(Wg, W), rel_fro(Hg, H))
                assert rel_elem(Wg, W, "f32t W") < ELEM_TOL["f32t"]
                assert rel_elem(Hg, H, "f32t H") < ELEM_TOL["f32t"]
        print(f"\n{shape}: worst W/H error over 2 iterations {worst:.2e}")
        assert worst < 1e-4


def test_split_persistent_tiles_and_segments():
    """Sizes where the persistent kernels' schedules matter: pass 1 has more tiles than
    SMs (188 in the H step, 192 in the W step, so CTAs run two tiles back to back) and
    pass 2 splits o-blocks between CTAs (752 (o-block, chunk) units over the SMs, cost
    slots per segment).  One DNA iteration from the oracle's state, W and H within 1e-4."""
    N, T, R = 1000, 12000, 64
    p = workloads.custom(N, T, R, seed=4242)
    with GpuProblem(p.V, p.W, p.H, "f32t") as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(p.W, p.H)
        worst = 0.0
        for which in (0, 1):
            W, H, _ = step_pair(gp, W, H, which)
            Wg, Hg = gp.WH()
            worst = max(worst, rel_fro(Wg, W), rel_fro(Hg, H))
            assert rel_elem(Wg, W, "f32t W") < ELEM_TOL["f32t"]
            assert rel_elem(Hg, H, "f32t H") < ELEM_TOL["f32t"]
        kl_gpu = gp.dna.dna_kl(gp.ctx)
        kl_ref = o.kl_divergence(p.V.astype(np.float64), W @ H)
        print(f"\n{(N, T, R)}: worst W/H error {worst:.2e}, d_KL {kl_gpu:.6e} vs {kl_ref:.6e}")
        assert worst < 1e-4
        assert abs(kl_gpu - kl_ref) <= 1e-5 * abs(kl_ref)


LARGE = [(300, 700, 129), (257, 500, 300), (520, 640, 512)]


@pytest.mark.parametrize("shape", LARGE, ids=lambda s: "x".join(map(str, s)))
def test_split_large_rank_half_steps(shape):
    """Padded ranks 256 and 512 (the ratios + contraction pass 1 and the K-sliced pass 2 of
    the split form): two DNA iterations from the oracle's state, each half-step within the
    element-wise bound and, over both iterations, within 1e-4 relative (Frobenius; for
    R > 300, SPLIT_LARGE_R_TOL, derived in gpu_helpers); final d_KL to the same bound."""
    N, T, R = shape
    p = workloads.custom(N, T, R, seed=N + 3 * T + 7 * R)
    with GpuProblem(p.V, p.W, p.H, "f32t") as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(p.W, p.H)
        worst = 0.0
        for _ in range(2):
            for which in (0, 1):
                W, H, _ = step_pair(gp, W, H, which)
                Wg, Hg = gp.WH()
                worst = max(worst, rel_fro(Wg, W), rel_fro(Hg, H))
                assert rel_elem(Wg, W, "f32t-large W") < ELEM_TOL["f32t"]
                assert rel_elem(Hg, H, "f32t-large H") < ELEM_TOL["f32t"]
        kl_gpu = gp.dna.dna_kl(gp.ctx)
        kl_ref = o.kl_divergence(p.V.astype(np.float64), W @ H)
        print(f"\n{shape}: worst W/H error over 2 iterations {worst:.2e}")
        tol = SPLIT_LARGE_R_TOL if R > 300 else 1e-4
        assert worst < tol
        assert abs(kl_gpu - kl_ref) <= tol * abs(kl_ref)


def test_split_large_rank_many_tiles():
    """R = 300 (padded 512) at a size where each kernel's CTAs run several tiles: the
    contraction has two (H step) and three (W step) splits of s, the ratios kernel several
    chunks per tile, pass 2 several (o-block, split) tiles per CTA.  One iteration from the
    oracle's state, then four MU iterations (the ratios kernel without Qbar)."""
    N, T, R = 2100, 2600, 300
    p = workloads.custom(N, T, R, seed=77)
    with GpuProblem(p.V, p.W, p.H, "f32t") as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(p.W, p.H)
        for which in (0, 1):
            W, H, _ = step_pair(gp, W, H, which)
            Wg, Hg = gp.WH()
            assert rel_fro(Wg, W) < 1e-4 and rel_fro(Hg, H) < 1e-4
            assert rel_elem(Wg, W, "f32t-tiles W") < ELEM_TOL["f32t"]
            assert rel_elem(Hg, H, "f32t-tiles H") < ELEM_TOL["f32t"]
        gp.dna.mu_iterate(gp.ctx, 4)
        V = p.V.astype(np.float64)
        for _ in range(4):
            W, H = o.mu_iteration(V, W, H)
        Wg, Hg = gp.WH()
        assert rel_fro(Wg, W) < 1e-4 and rel_fro(Hg, H) < 1e-4
        assert rel_elem(Wg, W, "f32t-tiles mu W") < ELEM_TOL["f32t"]
        assert rel_elem(Hg, H, "f32t-tiles mu H") < ELEM_TOL["f32t"]


def test_split_rank_limits():
    """The split form takes every rank the library does (1 <= R <= 512), and the sparse-V
    form stays on the CUDA cores."""
    import paper_1301_3389_gb300 as dna
    opts = dna.make_opts(dtype=dna.DNA_F32, engine=dna.DNA_ENGINE_TENSOR)
    for R in (1, 200, 512):
        dna.dna_destroy(dna.dna_create(64, 64, R, opts))
    with pytest.raises(dna.DNAError) as e:
        dna.dna_create(64, 64, 513, opts)
    assert e.value.code == dna.DNA_ERR_ARG
    with pytest.raises(dna.DNAError) as e:
        dna.dna_create_sparse(64, 64, 8, 10, opts)
    assert e.value.code == dna.DNA_ERR_UNSUPPORTED


def test_split_unaligned_leading_dimension():
    """V with a leading dimension that is not a multiple of 4 floats (aligned copy)."""
    import torch
    p = workloads.custom(90, 150, 12, seed=17)
    V = np.zeros((90, 153), dtype=np.float32)
    V[:, :150] = p.V
    with GpuProblem(p.V, p.W, p.H, "f32t") as ref:
        ref.dna.dna_iterate(ref.ctx, 2)
        Wr, Hr = ref.WH()
    import paper_1301_3389_gb300 as dna
    Vd = torch.from_numpy(V).cuda()
    Wd = torch.from_numpy(p.W).cuda()
    Hd = torch.from_numpy(p.H).cuda()
    ctx = dna.dna_create(90, 150, 12, dna.make_opts(dtype=dna.DNA_F32, engine=dna.DNA_ENGINE_TENSOR))
    try:
        dna.dna_set_stream(ctx)
        dna.dna_bind(ctx, Vd, Wd, Hd, ldv=153)
        dna.dna_iterate(ctx, 2)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(Wd.cpu().numpy(), Wr.astype(np.float32))
        np.testing.assert_array_equal(Hd.cpu().numpy(), Hr.astype(np.float32))
    finally:
        dna.dna_destroy(ctx)
