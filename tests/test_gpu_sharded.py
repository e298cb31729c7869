"""The column-sharded iteration (dna_shard_* through paper_1301_3389_gb300.sharded) with
the shards emulated on one GPU: G contexts over column blocks of one problem, each with its
own copy of W, the exchanges summed over the blocks.  Checked against the FP64 oracle on
the whole problem (selections replayed at near ties, the FP32 / FP64 tolerances of
test_gpu_parity.py) and against the unsharded GPU path; the W replicas must stay
bit-identical across the blocks."""
import numpy as np
import pytest

import workloads
from gpu_helpers import NEAR_TIE, GpuProblem, rel_fro
from oracle import dna as o

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f32t": 1e-4, "f64": 1e-10}


def _blocks(T, G):
    cuts = np.linspace(0, T, G + 1).astype(int)
    cuts[1:-1] += 3          # uneven blocks
    return [(int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:])]


def _sharded(p, kind, G, **opts):
    from paper_1301_3389_gb300.sharded import ShardedDNA
    shards = []
    for a, b in _blocks(p.V.shape[1], G):
        gp = GpuProblem(np.ascontiguousarray(p.V[:, a:b]), p.W.copy(),
                        np.ascontiguousarray(p.H[:, a:b]), kind, **opts)
        gp.dna.dna_normalize(gp.ctx, 1)
        shards.append(gp)
    import torch
    sh = ShardedDNA([s.ctx for s in shards], p.V.shape[0], p.W.shape[1], shards[0].tdt)
    return sh, shards


def _gather(shards):
    Ws = [s.WH()[0] for s in shards]
    H = np.concatenate([s.WH()[1] for s in shards], axis=1)
    return Ws, H


@pytest.mark.parametrize("kind", ["f32", "f32t", "f64"])
@pytest.mark.parametrize("G", [2, 3])
def test_sharded_matches_oracle(kind, G):
    p = workloads.custom(160, 300, 12, seed=40 + G)
    V = p.V.astype(np.float64)
    sh, shards = _sharded(p, kind, G)
    try:
        W, H = o.normalize_w_columns(p.W, p.H)
        for it in range(3):
            sh.step_H()
            ch = np.concatenate([s.choice(0) for s in shards])
            half = o.h_half_step(V, W, H)
            diff = ch != half.choice
            if diff.any():
                assert half.margin[diff].max() < NEAR_TIE[kind]
            W, H, _ = o.dna_step_h(V, W, H, choice=ch)
            Ws, Hg = _gather(shards)
            for Wg in Ws[1:]:
                np.testing.assert_array_equal(Wg, Ws[0])      # replicas stay identical
            assert rel_fro(Ws[0], W) < TOL[kind] and rel_fro(Hg, H) < TOL[kind], (it, "H")
            sh.step_W()
            chs = [s.choice(1) for s in shards]
            for c in chs[1:]:
                np.testing.assert_array_equal(c, chs[0])      # one selection per row
            half = o.w_half_step(V, W, H)
            diff = chs[0] != half.choice
            if diff.any():
                assert half.margin[diff].max() < NEAR_TIE[kind]
            W, H, _ = o.dna_step_w(V, W, H, choice=chs[0])
            Ws, Hg = _gather(shards)
            for Wg in Ws[1:]:
                np.testing.assert_array_equal(Wg, Ws[0])
            assert rel_fro(Ws[0], W) < TOL[kind] and rel_fro(Hg, H) < TOL[kind], (it, "W")
        kl = sh.kl()
        ref = o.kl_divergence(V, W @ H)
        assert abs(kl - ref) <= TOL[kind] * abs(ref)
    finally:
        for s in shards:
            s.close()


def test_sharded_equals_unsharded_f64():
    """G = 3 blocks and the unsharded context give the same iterates to rounding (FP64)."""
    p = workloads.custom(120, 250, 9, seed=77)
    sh, shards = _sharded(p, "f64", 3, rho=0.1, lam=0.2)
    try:
        sh.iterate(3)
        Ws, Hs = _gather(shards)
    finally:
        for s in shards:
            s.close()
    with GpuProblem(p.V, p.W, p.H, "f64", rho=0.1, lam=0.2) as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        gp.dna.dna_iterate(gp.ctx, 3)
        Wd, Hd = gp.WH()
    assert rel_fro(Ws[0], Wd) < 1e-11 and rel_fro(Hs, Hd) < 1e-11


def test_single_shard_equals_plain_steps():
    """G = 1: the phases reproduce dna_step_H then dna_step_W bit for bit (FP32)."""
    p = workloads.custom(100, 180, 10, seed=78)
    sh, shards = _sharded(p, "f32", 1)
    try:
        sh.iterate(2)
        Ws, Hs = _gather(shards)
    finally:
        shards[0].close()
    with GpuProblem(p.V, p.W, p.H, "f32") as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        for _ in range(2):
            gp.dna.dna_step_H(gp.ctx)
            gp.dna.dna_step_W(gp.ctx)
        Wd, Hd = gp.WH()
    np.testing.assert_array_equal(Ws[0], Wd)
    np.testing.assert_array_equal(Hs, Hd)
