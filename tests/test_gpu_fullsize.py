"""Parity at the benchmark's full size (N=4096 T=16384 R=128, FP32 form), on sampled
outputs the oracle computes one by one.

The H half-step separates over columns (eq. 5) and the W half-step over rows, so the
oracle runs either on a sample of columns (rows) exactly.  The step-16 (29)
normalisation couples all of them only through one factor per r, which is read from
the GPU's own rescaling of the other factor.  Tolerance: 1e-4 relative (FP32 form, on the
CUDA cores and on the tensor cores with split operands); the per-column costs to 1e-5
(CUDA cores) and 1e-4 (split tensor-core products, relative error per product below
about 2^-15).
"""
import numpy as np
import pytest

import workloads
import dataclasses

from gpu_helpers import GpuProblem, rel_fro, replay_choice, step_elementwise
from oracle import dna as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    return workloads.plain_large(0)


@pytest.mark.parametrize("kind", ["f32", "f32t"])
def test_plain_large_sampled(big, kind):
    _sampled(big, kind, 1e-5 if kind == "f32" else 1e-4, 1e-4)


def test_precision_large_split_sampled():
    """N=8192 T=32768 R=512 in the FP32 form on the tensor cores (the form the bench's
    time-to-target runs at this size): sampled columns and rows against the oracle, with
    the tolerance derived for the split operands at R > 300 (tests/gpu_helpers.py)."""
    from gpu_helpers import SPLIT_LARGE_R_TOL
    _sampled(workloads.precision_large(0), "f32t", SPLIT_LARGE_R_TOL, SPLIT_LARGE_R_TOL)


def _sampled(big, kind, ctol, tol):
    g = np.random.default_rng(0)
    N, T = big.V.shape
    cols = np.sort(g.choice(T, 48, replace=False))
    rows = np.sort(g.choice(N, 48, replace=False))
    with GpuProblem(big.V, big.W, big.H, kind) as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        kl0 = gp.dna.dna_kl(gp.ctx)
        W0, H0 = gp.WH()
        # H half-step on sampled columns
        gp.dna.dna_step_H(gp.ctx)
        W1, H1 = gp.WH()
        dm, dd = gp.costs(0)
        ch = gp.choice(0)
        Vc = big.V[:, cols].astype(np.float64)
        half = o.h_half_step(Vc, W0, H0[:, cols])
        np.testing.assert_allclose(dm[cols], half.d_mu, rtol=ctol)
        np.testing.assert_allclose(dd[cols], half.d_dna, rtol=ctol)
        mask, _ = replay_choice(half, ch[cols], kind)
        X = np.where(mask[None, :], half.X_dna, half.X_mu)
        sigma = W1.sum(axis=0) / W0.sum(axis=0)          # step 16 factor per r
        eh = rel_fro(H1[:, cols], X / sigma[:, None])
        print(f"\n{kind}: H half-step error on sampled columns {eh:.2e}")
        assert eh < tol
        half = dataclasses.replace(half, choice=mask)
        assert step_elementwise(half, 0, W0, H0[:, cols], W1, H1[:, cols], kind, sig=sigma,
                                check_y=False, label="H sampled") <= 1.0
        # W half-step on sampled rows
        gp.dna.dna_step_W(gp.ctx)
        W2, H2 = gp.WH()
        ch = gp.choice(1)
        Vr = big.V[rows, :].astype(np.float64)
        half = o.w_half_step(Vr, W1[rows, :], H1)
        mask, _ = replay_choice(half, ch[rows], kind)
        X = np.where(mask[:, None], half.X_dna, half.X_mu)
        sigma = H2.sum(axis=1) / H1.sum(axis=1)          # step 29 factor per r
        ew = rel_fro(W2[rows, :], X / sigma[None, :])
        print(f"{kind}: W half-step error on sampled rows {ew:.2e}")
        assert ew < tol
        half = dataclasses.replace(half, choice=mask)
        assert step_elementwise(half, 1, W1[rows, :], H1, W2[rows, :], H2, kind, sig=sigma,
                                check_y=False, label="W sampled") <= 1.0
        # properties at full size: cost does not increase; eq. 9 per row after the W step
        kl1 = gp.dna.dna_kl(gp.ctx)
        assert kl1 <= kl0
        import torch
        Z = gp.W @ gp.H
        rs = Z.double().sum(dim=1).cpu().numpy()
        np.testing.assert_allclose(rs, big.V.astype(np.float64).sum(axis=1), rtol=tol)
