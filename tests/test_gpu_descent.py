"""Descent selection (dna_set_selection(DNA_SELECT_DESCENT)): the Newton candidate is kept
iff its eq. 5 (eq. 4) cost is below the starting column's (row's).  Against the FP64
oracle's descent rule, with the tolerances of test_gpu_parity.py: W and H within 1e-4
(FP32) / 1e-10 (FP64) per half-step with selections replayed at near ties, the one-step
element-wise bound, the compared costs (starting, Newton) per column and row, and d_KL
never increasing."""
import numpy as np
import pytest

import workloads
from gpu_helpers import NEAR_TIE, GpuProblem, rel_fro, step_pair
from oracle import dna as o

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f64": 1e-10}
COST_RTOL = {"f32": 1e-5, "f64": 1e-11}


@pytest.mark.parametrize("kind", ["f32", "f64"])
@pytest.mark.parametrize("reg", [0.0, 1.5])
def test_descent_matches_oracle(kind, reg):
    p = workloads.custom(130, 270, 12, seed=61)
    V = p.V.astype(np.float64)
    opts = {"selection": "descent", "rho": reg, "lam": reg}
    with GpuProblem(p.V, p.W, p.H, kind, selection="descent", rho=reg, lam=reg) as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(p.W, p.H, reg)
        prev = gp.dna.dna_kl(gp.ctx)
        for it in range(4):
            for which in (0, 1):
                Wg0, Hg0 = gp.WH()
                W, H, _ = step_pair(gp, W, H, which, opts=opts)   # includes the element-wise bound
                Wg, Hg = gp.WH()
                assert rel_fro(Wg, W) < TOL[kind] and rel_fro(Hg, H) < TOL[kind], (it, which)
                # the two costs the GPU compared, from its own starting state
                half = (o.h_half_step(V, Wg0, Hg0, lam=reg, selection="descent") if which == 0
                        else o.w_half_step(V, Wg0, Hg0, rho=reg, selection="descent"))
                # d' sums terms of size ~ v (|log z| + 1) and can cross zero: its error scales
                # with |d'| + sum v of the column (row), not with d'
                dc, dd = gp.costs(which)
                scale = V.sum(axis=0 if which == 0 else 1) + 1.0
                for got, ref in ((dc, half.d_cur), (dd, half.d_dna)):
                    assert np.all(np.abs(got - ref) <= COST_RTOL[kind] * (np.abs(ref) + scale))
            if reg == 0.0:
                kl = gp.dna.dna_kl(gp.ctx)
                assert kl <= prev * (1 + 1e-7), (kl, prev)          # never increases
                prev = kl


def test_descent_keeps_the_papers_newton_columns():
    """From the same state, every column the paper's rule gives to Newton, descent does too."""
    p = workloads.custom(200, 400, 16, seed=62)
    with GpuProblem(p.V, p.W, p.H, "f64") as a, GpuProblem(p.V, p.W, p.H, "f64",
                                                         selection="descent") as b:
        for gp in (a, b):
            gp.dna.dna_normalize(gp.ctx, 1)
            gp.dna.dna_step_H(gp.ctx)
        ca, cb = a.choice(0), b.choice(0)
        assert np.all(cb[ca]) and cb.sum() >= ca.sum()


def test_descent_rejected_on_tensor_engines_and_sparse():
    import paper_1301_3389_gb300 as dna
    p = workloads.custom(64, 64, 8, seed=63)
    for kind in ("f32t", "bf16"):
        with GpuProblem(p.V, p.W, p.H, kind) as gp:
            with pytest.raises(dna.DNAError) as e:
                dna.dna_set_selection(gp.ctx, dna.DNA_SELECT_DESCENT)
            assert e.value.code == dna.DNA_ERR_UNSUPPORTED
