"""The batching form: many uneven problems, one grouped launch per phase, CUDA graph.

FP32 form (CUDA cores): each problem of a group must follow the single-problem FP32 path
and its d_KL must match the FP64 oracle's to 1e-4 after the same iterations.  BF16 form
(tensor-core passes): every problem against the FP64 oracle half-step by half-step with the
BF16 form's bounds (test_gpu_bf16.py).  The two paths share the pass tiles
but not the reductions between them (split sums, the eq. 10 denominator and the step
16 / 29 sums are taken in different fixed orders), so their float32 trajectories agree
to rounding amplified by two DNA iterations: 5e-5 relative.  Graph replay must equal
direct launches bit for bit.
"""
import numpy as np
import pytest

import workloads
import dataclasses

from gpu_helpers import (ELEM_TOL, GpuProblem, rel_elem, rel_fro, replay_choice,
                         step_elementwise)
from oracle import dna as o

pytestmark = pytest.mark.gpu

SHAPES = [(64, 128, 8), (700, 300, 16), (150, 900, 32), (333, 129, 64), (90, 517, 1),
          (257, 257, 33), (1, 200, 4), (400, 1, 12), (128, 640, 64), (77, 77, 7)]


def _group(problems, bf16=False, **opts):
    import torch

    import paper_1301_3389_gb300 as dna
    dev = torch.device("cuda")
    V = [torch.from_numpy(p.V).to(dev) for p in problems]
    W = [torch.from_numpy(p.W).to(dev) for p in problems]
    H = [torch.from_numpy(p.H).to(dev) for p in problems]
    if bf16:
        opts["dtype"] = dna.DNA_BF16
    opts = dna.make_opts(**opts) if opts else None
    g = dna.dna_group_create([p.V.shape[0] for p in problems], [p.V.shape[1] for p in problems],
                             [p.W.shape[1] for p in problems], opts)
    dna.dna_group_set_stream(g)
    dna.dna_group_bind(g, V, W, H)
    return dna, g, V, W, H


def _problems(seed=0):
    return [workloads.custom(n, t, r, seed=seed * 1000 + i) for i, (n, t, r) in enumerate(SHAPES)]


def test_group_matches_single_path():
    import torch
    probs = _problems()
    dna, g, V, W, H = _group(probs)
    try:
        dna.dna_group_normalize(g, 1)
        dna.dna_group_iterate(g, 2)
        kl = dna.dna_group_kl(g, len(probs))
        torch.cuda.synchronize()
        for q, p in enumerate(probs):
            with GpuProblem(p.V, p.W, p.H, "f32") as gp:
                gp.dna.dna_normalize(gp.ctx, 1)
                gp.dna.dna_iterate(gp.ctx, 2)
                Ws, Hs = gp.WH()
                kls = gp.dna.dna_kl(gp.ctx)
            _, _, costs = o.run(p.V, p.W, p.H, 2, "dna")
            assert abs(kl[q] - costs[-1]) <= 1e-4 * max(costs[-1], 1.0), (q, kl[q], costs[-1])
            if min(p.V.shape) < 8:
                # one data point per row (or column): the per-row optimum is a continuum,
                # MU and Newton costs tie, and rounding-level differences in the factor sums
                # flip selections; both trajectories are valid, so only d_KL is compared
                continue
            assert rel_fro(W[q].double().cpu().numpy(), Ws) < 5e-5, q
            assert rel_fro(H[q].double().cpu().numpy(), Hs) < 5e-5, q
            assert abs(kl[q] - kls) <= 1e-5 * max(abs(kls), 1.0), (q, kl[q], kls)
    finally:
        dna.dna_group_destroy(g)


def test_group_matches_oracle_per_half_step():
    """Every problem of the group against the FP64 oracle, half-step by half-step, with the
    oracle replaying the group's selections where they differ at near ties: W and H within
    the FP32 form's 1e-4 relative (Frobenius) and element-wise tolerance after each of two
    iterations, and d_KL within 1e-4."""
    import torch
    probs = _problems(3)
    dna, g, V, W, H = _group(probs)
    try:
        dna.dna_group_normalize(g, 1)
        ref = [o.normalize_w_columns(p.W, p.H) for p in probs]
        V64 = [p.V.astype(np.float64) for p in probs]
        for it in range(2):
            for which in (0, 1):
                torch.cuda.synchronize()
                before = [(w.double().cpu().numpy(), h.double().cpu().numpy()) for w, h in zip(W, H)]
                (dna.dna_group_step_H if which == 0 else dna.dna_group_step_W)(g)
                torch.cuda.synchronize()
                for q, p in enumerate(probs):
                    Wr, Hr = ref[q]
                    n = p.V.shape[1] if which == 0 else p.V.shape[0]
                    ch = dna.dna_group_get_choice(g, q, which, n)
                    # element-wise, one step from the group's own state (gpu_helpers bound)
                    W0, H0 = before[q]
                    one = (o.h_half_step if which == 0 else o.w_half_step)(V64[q], W0, H0)
                    m1, _ = replay_choice(one, ch, "f32")
                    assert step_elementwise(dataclasses.replace(one, choice=m1), which, W0, H0,
                                            W[q].double().cpu().numpy(),
                                            H[q].double().cpu().numpy(), "f32",
                                            label="group") <= 1.0, (q, it, which)
                    if which == 0:
                        half = o.h_half_step(V64[q], Wr, Hr)
                        mask, _ = replay_choice(half, ch, "f32")
                        Wr, Hr, _ = o.dna_step_h(V64[q], Wr, Hr, choice=mask)
                    else:
                        half = o.w_half_step(V64[q], Wr, Hr)
                        mask, _ = replay_choice(half, ch, "f32")
                        Wr, Hr, _ = o.dna_step_w(V64[q], Wr, Hr, choice=mask)
                    ref[q] = (Wr, Hr)
                    Wg = W[q].double().cpu().numpy()
                    Hg = H[q].double().cpu().numpy()
                    assert rel_fro(Wg, Wr) < 1e-4 and rel_fro(Hg, Hr) < 1e-4, (q, it, which)
                    assert rel_elem(Wg, Wr, "group W") < ELEM_TOL["f32"], (q, it, which)
                    assert rel_elem(Hg, Hr, "group H") < ELEM_TOL["f32"], (q, it, which)
        kl = dna.dna_group_kl(g, len(probs))
        for q, (Wr, Hr) in enumerate(ref):
            kr = o.kl_divergence(V64[q], Wr @ Hr)
            assert abs(kl[q] - kr) <= 1e-4 * max(kr, 1.0), (q, kl[q], kr)
    finally:
        dna.dna_group_destroy(g)


def test_group_graph_equals_direct():
    import torch
    outs = []
    for graph in (False, True):
        probs = _problems(1)
        dna, g, V, W, H = _group(probs)
        try:
            dna.dna_group_use_graph(g, graph)
            dna.dna_group_normalize(g, 1)
            dna.dna_group_iterate(g, 3)
            torch.cuda.synchronize()
            outs.append([(w.cpu().numpy().copy(), h.cpu().numpy().copy()) for w, h in zip(W, H)])
            assert dna.dna_group_get_status(g) == 0
        finally:
            dna.dna_group_destroy(g)
    for (w0, h0), (w1, h1) in zip(*outs):
        np.testing.assert_array_equal(w0, w1)
        np.testing.assert_array_equal(h0, h1)


def test_group_autotune_keeps_state():
    import torch
    probs = _problems(2)
    dna, g, V, W, H = _group(probs)
    try:
        dna.dna_group_normalize(g, 1)
        torch.cuda.synchronize()
        before = [(w.cpu().numpy().copy(), h.cpu().numpy().copy()) for w, h in zip(W, H)]
        rows = dna.dna_group_autotune(g, 1)
        assert rows in (256, 512, 1024, 2048, 4096, 1 << 30)
        torch.cuda.synchronize()
        for (w0, h0), w, h in zip(before, W, H):
            np.testing.assert_array_equal(w0, w.cpu().numpy())
            np.testing.assert_array_equal(h0, h.cpu().numpy())
        dna.dna_group_iterate(g, 1)
        assert dna.dna_group_get_status(g) == 0
    finally:
        dna.dna_group_destroy(g)


def test_group_rejects_unsupported():
    import paper_1301_3389_gb300 as dna
    with pytest.raises(dna.DNAError) as e:
        dna.dna_group_create([10], [10], [65])
    assert e.value.code == dna.DNA_ERR_UNSUPPORTED
    for opts in (dna.make_opts(dtype=dna.DNA_F64),
                 dna.make_opts(dtype=dna.DNA_BF16, engine=dna.DNA_ENGINE_SIMT),
                 dna.make_opts(dtype=dna.DNA_F32, engine=dna.DNA_ENGINE_TENSOR)):
        with pytest.raises(dna.DNAError) as e:
            dna.dna_group_create([10], [10], [8], opts)
        assert e.value.code == dna.DNA_ERR_UNSUPPORTED


BF16_TOL = 2e-2   # one BF16 half-step against the oracle from the same state (test_gpu_bf16)


def test_group_bf16_matches_oracle_per_half_step():
    """The BF16 form of the group (tcgen05 passes over the tile table): every problem, after
    each half-step of two iterations, against the FP64 oracle's half-step from the group's
    own state with the group's selections replayed where they differ at near ties: W and H
    within the BF16 form's 2e-2 relative (Frobenius) and its element-wise bound; d_KL of the
    final factors within 1e-4."""
    import torch
    probs = _problems(5)
    dna, g, V, W, H = _group(probs, bf16=True)
    try:
        dna.dna_group_normalize(g, 1)
        V64 = [p.V.astype(np.float64) for p in probs]
        for it in range(2):
            for which in (0, 1):
                torch.cuda.synchronize()
                before = [(w.double().cpu().numpy(), h.double().cpu().numpy()) for w, h in zip(W, H)]
                (dna.dna_group_step_H if which == 0 else dna.dna_group_step_W)(g)
                torch.cuda.synchronize()
                assert dna.dna_group_get_status(g) == 0
                for q, p in enumerate(probs):
                    n = p.V.shape[1] if which == 0 else p.V.shape[0]
                    ch = dna.dna_group_get_choice(g, q, which, n)
                    W0, H0 = before[q]
                    one = (o.h_half_step if which == 0 else o.w_half_step)(V64[q], W0, H0)
                    m1, _ = replay_choice(one, ch, "bf16")
                    Wg = W[q].double().cpu().numpy()
                    Hg = H[q].double().cpu().numpy()
                    assert step_elementwise(dataclasses.replace(one, choice=m1), which, W0, H0,
                                            Wg, Hg, "bf16", label="group-bf16") <= 1.0, (q, it, which)
                    step = o.dna_step_h if which == 0 else o.dna_step_w
                    Wr, Hr, _ = step(V64[q], W0, H0, choice=m1)
                    assert rel_fro(Wg, Wr) < BF16_TOL and rel_fro(Hg, Hr) < BF16_TOL, (q, it, which)
        kl = dna.dna_group_kl(g, len(probs))
        for q, p in enumerate(probs):
            kr = o.kl_divergence(V64[q], W[q].double().cpu().numpy() @ H[q].double().cpu().numpy())
            assert abs(kl[q] - kr) <= 1e-4 * max(kr, 1.0), (q, kl[q], kr)
    finally:
        dna.dna_group_destroy(g)


def test_group_bf16_graph_autotune():
    """BF16 group: graph replay equals direct launches bit for bit; the autotuner picks a
    split size and a pass-2 tile size, restores W and H, and the group keeps iterating."""
    import torch
    outs = []
    for graph in (False, True):
        probs = _problems(6)
        dna, g, V, W, H = _group(probs, bf16=True)
        try:
            dna.dna_group_use_graph(g, graph)
            dna.dna_group_normalize(g, 1)
            dna.dna_group_iterate(g, 3)
            torch.cuda.synchronize()
            outs.append([(w.cpu().numpy().copy(), h.cpu().numpy().copy()) for w, h in zip(W, H)])
            assert dna.dna_group_get_status(g) == 0
            if graph:
                before = outs[-1]
                rows = dna.dna_group_autotune(g, 1)
                r2, units = dna.dna_group_tile_config(g)
                assert rows == r2 and rows in (256, 512, 1024, 2048, 4096, 1 << 30)
                assert units in (4, 8, 16, 32, 64, 128)
                torch.cuda.synchronize()
                for (w0, h0), w, h in zip(before, W, H):
                    np.testing.assert_array_equal(w0, w.cpu().numpy())
                    np.testing.assert_array_equal(h0, h.cpu().numpy())
                dna.dna_group_iterate(g, 1)
                assert dna.dna_group_get_status(g) == 0
        finally:
            dna.dna_group_destroy(g)
    for (w0, h0), (w1, h1) in zip(*outs):
        np.testing.assert_array_equal(w0, w1)
        np.testing.assert_array_equal(h0, h1)


def test_group_bf16_fused_rescale_equals_half_steps():
    """dna_group_iterate (whose H half-step rescale also writes the W half-step's bf16
    operands) equals separate dna_group_step_H / dna_group_step_W calls bit for bit."""
    import torch
    outs = []
    for fused in (True, False):
        probs = _problems(7)
        dna, g, V, W, H = _group(probs, bf16=True)
        try:
            dna.dna_group_normalize(g, 1)
            for _ in range(2):
                if fused:
                    dna.dna_group_iterate(g, 1)
                else:
                    dna.dna_group_step_H(g)
                    dna.dna_group_step_W(g)
            torch.cuda.synchronize()
            assert dna.dna_group_get_status(g) == 0
            outs.append([(w.cpu().numpy().copy(), h.cpu().numpy().copy()) for w, h in zip(W, H)])
        finally:
            dna.dna_group_destroy(g)
    for (w0, h0), (w1, h1) in zip(*outs):
        np.testing.assert_array_equal(w0, w1)
        np.testing.assert_array_equal(h0, h1)


@pytest.mark.parametrize("kind", ["f32", "bf16"])
def test_group_regularised(kind):
    """The group with lambda, rho > 0 and non-default eps, alpha (eq. 2, Section 2.3), in both
    forms: every problem's half-steps against the oracle's from the group's own state, the
    group's selections replayed at near ties; the element-wise bound of the form, and its
    Frobenius tolerance (FP32 1e-4, BF16 2e-2)."""
    import torch
    probs = _problems(8)[:6]
    reg = dict(eps=0.05, alpha=1.5, rho=0.2, lam=0.3)
    tol = BF16_TOL if kind == "bf16" else 1e-4
    dna, g, V, W, H = _group(probs, bf16=(kind == "bf16"), **reg)
    try:
        dna.dna_group_normalize(g, 1)
        V64 = [p.V.astype(np.float64) for p in probs]
        for which in (0, 1, 0, 1):
            torch.cuda.synchronize()
            before = [(w.double().cpu().numpy(), h.double().cpu().numpy()) for w, h in zip(W, H)]
            (dna.dna_group_step_H if which == 0 else dna.dna_group_step_W)(g)
            torch.cuda.synchronize()
            assert dna.dna_group_get_status(g) == 0
            for q, p in enumerate(probs):
                n = p.V.shape[1] if which == 0 else p.V.shape[0]
                ch = dna.dna_group_get_choice(g, q, which, n)
                W0, H0 = before[q]
                if which == 0:
                    one = o.h_half_step(V64[q], W0, H0, reg["eps"], reg["alpha"], reg["lam"])
                else:
                    one = o.w_half_step(V64[q], W0, H0, reg["eps"], reg["alpha"], reg["rho"])
                m1, _ = replay_choice(one, ch, kind)
                Wg = W[q].double().cpu().numpy()
                Hg = H[q].double().cpu().numpy()
                assert step_elementwise(dataclasses.replace(one, choice=m1), which, W0, H0, Wg, Hg,
                                        kind, reg["eps"], reg["alpha"],
                                        reg["rho"] if which == 0 else reg["lam"],
                                        label=f"group-{kind}-reg") <= 1.0, (q, which)
                step = o.dna_step_h if which == 0 else o.dna_step_w
                Wr, Hr, _ = step(V64[q], W0, H0, reg["eps"], reg["alpha"], reg["rho"], reg["lam"],
                                 choice=m1)
                assert rel_fro(Wg, Wr) < tol and rel_fro(Hg, Hr) < tol, (q, which)
    finally:
        dna.dna_group_destroy(g)
