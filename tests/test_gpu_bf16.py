"""The BF16 precision form (tcgen05 tensor cores, bf16 operands, float32 accumulation)
against the FP64 oracle.

Tolerance, derived from the arithmetic: bf16 keeps 8 significant bits, unit roundoff
u = 2^-9 ~ 2e-3.  z is a sum of positive products of two rounded operands (relative error
<= 2u); q = v/z is rounded again (u); A = sum w q rounds w (u): the eq. 7 ratio (1 + a) is
off by ~4u ~ 8e-3 element-wise in the worst case; the Newton step a / b of eq. 17 can
magnify that where a is small.  Measured one-step errors (relative Frobenius, first
iteration): H half-step 1e-4 - 3e-3, W half-step 2e-3 - 9e-3 (largest when R exceeds N or
T).  So: W and H within 2e-2 (about 10 u) after each half-step; candidate costs within
1e-2 of their summed terms; selections may differ where the oracle's relative cost margin
is below 1e-2.  The float64 cost log (dna_kl) uses float32 products and must match the
oracle to 1e-4.
"""
import numpy as np
import pytest

import workloads
import dataclasses

from gpu_helpers import GpuProblem, one_step_check, rel_elem, rel_fro, step_elementwise
from oracle import dna as o

pytestmark = pytest.mark.gpu

TOL_BF16 = 2e-2
TOL_COST = 1e-2
MARGIN_BF16 = 1e-2


def _replay(half, gpu_choice):
    diff = np.asarray(gpu_choice, bool) != half.choice
    if diff.any():
        assert half.margin[diff].max() < MARGIN_BF16, half.margin[diff].max()
    return np.asarray(gpu_choice, bool), int(diff.sum())


def _bf16_steps(p, iters, check_costs=True, restart=True):
    """GPU half-steps against the oracle.  restart=True: the oracle starts every half-step
    from the GPU's own current W and H, so each comparison measures one step's bf16 error
    (the bound in the module docstring); restart=False: both run free (with replayed
    selections) and errors accumulate over the trajectory."""
    V = p.V.astype(np.float64)
    errs = []
    with GpuProblem(p.V, p.W, p.H, "bf16") as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(p.W, p.H)
        for _ in range(iters):
            for which in (0, 1):
                Wg0, Hg0 = gp.WH()
                if restart:
                    W, H = Wg0, Hg0
                half = (o.h_half_step if which == 0 else o.w_half_step)(V, W, H)
                (gp.dna.dna_step_H if which == 0 else gp.dna.dna_step_W)(gp.ctx)
                if check_costs:
                    # the cost d' of a column is a sum of terms of size ~v (|log z| + 1); its
                    # bf16 error scales with that sum, not with d' (which can cross zero)
                    dm, dd = gp.costs(which)
                    scale = V.sum(axis=0 if which == 0 else 1) + 1.0
                    assert np.all(np.abs(dm - half.d_mu) <= TOL_COST * (np.abs(half.d_mu) + scale))
                    assert np.all(np.abs(dd - half.d_dna) <= TOL_COST * (np.abs(half.d_dna) + scale))
                mask, _ = _replay(half, gp.choice(which))
                step = o.dna_step_h if which == 0 else o.dna_step_w
                W, H, _ = step(V, W, H, choice=mask)
                Wg, Hg = gp.WH()
                errs.append((rel_fro(Wg, W), rel_fro(Hg, H)))
                assert errs[-1][0] < TOL_BF16 and errs[-1][1] < TOL_BF16, errs[-1]
                # element-wise, one step from the GPU's own state (bound in gpu_helpers)
                ratio = one_step_check(gp, which, Wg0, Hg0, label="bf16")
                assert ratio <= 1.0, ratio
        kl = gp.dna.dna_kl(gp.ctx)
        Wg, Hg = gp.WH()
        assert abs(kl - o.kl_divergence(V, Wg @ Hg)) <= 1e-4 * kl
    return errs


SHAPES = [(200, 300, 16), (130, 257, 64), (256, 512, 100), (70, 1000, 128), (1000, 70, 128),
          (129, 131, 65), (1, 1, 1),
          # ranks above 128: the large-rank kernels (RP = 256, 512), including the
          # smallest rank of each padding class and ragged o-blocks and chunks
          (300, 500, 200), (257, 300, 512), (640, 130, 300), (150, 700, 129), (700, 150, 257),
          (333, 1025, 256)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_bf16_half_steps(shape):
    N, T, R = shape
    p = workloads.custom(N, T, R, seed=N + 3 * T + 7 * R)
    _bf16_steps(p, 2)


@pytest.mark.parametrize("shape", [(1500, 3000, 300), (2100, 1700, 256)],
                         ids=lambda s: "x".join(map(str, s)))
def test_bf16_large_rank_persistent_tiles(shape):
    """Ranks above 128 at sizes where the persistent pass 1 gives a CTA several
    (r-block, o-block, split) tiles and splits s into several 128-wide-chunk ranges."""
    N, T, R = shape
    _bf16_steps(workloads.custom(N, T, R, seed=N + T + R), 1)


def test_bf16_plain_small_trajectory():
    """N=256 T=512 R=16: a free-running 5-iteration trajectory stays within the tolerance."""
    errs = _bf16_steps(workloads.plain_small(0), 5, restart=False)
    assert max(max(e) for e in errs) < TOL_BF16


def test_bf16_reaches_fp32_kl():
    """50 iterations: the BF16 form's d_KL is within 1e-2 of the FP32 form's (the target of
    the precision form)."""
    p = workloads.plain_small(0)
    kls = {}
    for kind in ("f32", "bf16"):
        with GpuProblem(p.V, p.W, p.H, kind) as gp:
            gp.dna.dna_normalize(gp.ctx, 1)
            gp.dna.dna_iterate(gp.ctx, 50)
            kls[kind] = gp.dna.dna_kl(gp.ctx)
    assert abs(kls["bf16"] - kls["f32"]) <= 1e-2 * kls["f32"], kls


def test_bf16_mu_steps():
    p = workloads.custom(150, 260, 24, seed=8)
    V = p.V.astype(np.float64)
    with GpuProblem(p.V, p.W, p.H, "bf16") as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(p.W, p.H)
        for which in (0, 1, 0, 1):
            gp.dna.mu_step(gp.ctx, which)
            W, H = (o.mu_step_h if which == 0 else o.mu_step_w)(V, W, H)
            Wg, Hg = gp.WH()
            assert rel_fro(Wg, W) < TOL_BF16 and rel_fro(Hg, H) < TOL_BF16
            # MU: x (1 + a) carries the relative error of (1 + a), 2^-7 (4u)
            assert rel_elem(Wg, W, "bf16 mu W") < 4 * 2.0 ** -7
            assert rel_elem(Hg, H, "bf16 mu H") < 4 * 2.0 ** -7


def test_bf16_unaligned_leading_dimension():
    """A V whose rows are not 16-byte aligned (ldv = T = 131) takes the aligned copy."""
    p = workloads.custom(90, 131, 20, seed=21)
    _bf16_steps(p, 1)


def test_bf16_plain_large_sampled():
    """Full bench size (N=4096 T=16384 R=128): sampled columns and rows vs the oracle."""
    big = workloads.plain_large(0)
    g = np.random.default_rng(1)
    N, T = big.V.shape
    cols = np.sort(g.choice(T, 32, replace=False))
    rows = np.sort(g.choice(N, 32, replace=False))
    with GpuProblem(big.V, big.W, big.H, "bf16") as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W0, H0 = gp.WH()
        gp.dna.dna_step_H(gp.ctx)
        W1, H1 = gp.WH()
        half = o.h_half_step(big.V[:, cols].astype(np.float64), W0, H0[:, cols])
        mask, _ = _replay(half, gp.choice(0)[cols])
        X = np.where(mask[None, :], half.X_dna, half.X_mu)
        sigma = W1.sum(axis=0) / W0.sum(axis=0)
        assert rel_fro(H1[:, cols], X / sigma[:, None]) < TOL_BF16
        half = dataclasses.replace(half, choice=mask)
        assert step_elementwise(half, 0, W0, H0[:, cols], W1, H1[:, cols], "bf16",
                                sig=sigma, check_y=False, label="H sampled") <= 1.0
        gp.dna.dna_step_W(gp.ctx)
        W2, H2 = gp.WH()
        half = o.w_half_step(big.V[rows, :].astype(np.float64), W1[rows, :], H1)
        mask, _ = _replay(half, gp.choice(1)[rows])
        X = np.where(mask[:, None], half.X_dna, half.X_mu)
        sigma = H2.sum(axis=1) / H1.sum(axis=1)
        assert rel_fro(W2[rows, :], X / sigma[None, :]) < TOL_BF16
        half = dataclasses.replace(half, choice=mask)
        assert step_elementwise(half, 1, W1[rows, :], H1, W2[rows, :], H2, "bf16",
                                sig=sigma, check_y=False, label="W sampled") <= 1.0


def test_bf16_precision_large_sampled():
    """N=8192 T=32768 R=512 (the precision-form workload): sampled columns and rows."""
    big = workloads.precision_large(0)
    g = np.random.default_rng(2)
    N, T = big.V.shape
    cols = np.sort(g.choice(T, 16, replace=False))
    rows = np.sort(g.choice(N, 16, replace=False))
    with GpuProblem(big.V, big.W, big.H, "bf16") as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W0, H0 = gp.WH()
        gp.dna.dna_step_H(gp.ctx)
        W1, H1 = gp.WH()
        half = o.h_half_step(big.V[:, cols].astype(np.float64), W0, H0[:, cols])
        mask, _ = _replay(half, gp.choice(0)[cols])
        X = np.where(mask[None, :], half.X_dna, half.X_mu)
        sigma = W1.sum(axis=0) / W0.sum(axis=0)
        assert rel_fro(H1[:, cols], X / sigma[:, None]) < TOL_BF16
        half = dataclasses.replace(half, choice=mask)
        assert step_elementwise(half, 0, W0, H0[:, cols], W1, H1[:, cols], "bf16",
                                sig=sigma, check_y=False, label="H sampled") <= 1.0
        gp.dna.dna_step_W(gp.ctx)
        W2, H2 = gp.WH()
        half = o.w_half_step(big.V[rows, :].astype(np.float64), W1[rows, :], H1)
        mask, _ = _replay(half, gp.choice(1)[rows])
        X = np.where(mask[:, None], half.X_dna, half.X_mu)
        sigma = H2.sum(axis=1) / H1.sum(axis=1)
        assert rel_fro(W2[rows, :], X / sigma[None, :]) < TOL_BF16
        half = dataclasses.replace(half, choice=mask)
        assert step_elementwise(half, 1, W1[rows, :], H1, W2[rows, :], H2, "bf16",
                                sig=sigma, check_y=False, label="W sampled") <= 1.0
