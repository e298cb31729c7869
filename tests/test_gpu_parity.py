"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: FP32 form, W and H within 1e-4 relative (Frobenius) after each of the
first 5 iterations and final d_KL within 1e-3 relative after 50; FP64 form, 1e-10.
The FP32 form runs on the CUDA cores ("f32") and on the tensor cores with split hi + lo
bf16 operands ("f32t"), both held to the FP32 tolerances.
Selections may differ only at near ties (gpu_helpers.NEAR_TIE); the oracle then
replays the GPU's choice so rounding near a tie cannot grow into a different
trajectory.
"""
import numpy as np
import pytest

import workloads
from gpu_helpers import ELEM_TOL, SPLIT_LARGE_R_TOL, GpuProblem, rel_elem, rel_fro, step_pair
from oracle import dna as o

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f32t": 1e-4, "f64": 1e-10}


def _trajectory(p, kind, iters, mu=False, **opts):
    V = p.V.astype(np.float64)
    tol = SPLIT_LARGE_R_TOL if (kind == "f32t" and p.W.shape[1] > 300) else TOL[kind]
    with GpuProblem(p.V, p.W, p.H, kind, **{k: v for k, v in opts.items()}) as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        W, H = o.normalize_w_columns(p.W, p.H, opts.get("lam", 0.0))
        Wg, Hg = gp.WH()
        assert rel_fro(Wg, W) < tol and rel_fro(Hg, H) < tol
        flips = 0
        oopts = {"eps": opts.get("eps", o.EPS), "alpha": opts.get("alpha", o.ALPHA),
                 "rho": opts.get("rho", 0.0), "lam": opts.get("lam", 0.0)}
        for it in range(iters):
            for which in (0, 1):
                W, H, nf = step_pair(gp, W, H, which, mu=mu, opts=oopts)
                flips += nf
                Wg, Hg = gp.WH()
                ew, eh = rel_fro(Wg, W), rel_fro(Hg, H)
                assert ew < tol and eh < tol, (it, which, ew, eh)
                xw = rel_elem(Wg, W, f"{kind} W it{it}.{which}")
                xh = rel_elem(Hg, H, f"{kind} H it{it}.{which}")
                assert xw < ELEM_TOL[kind] and xh < ELEM_TOL[kind], (it, which, xw, xh)
        kl_gpu = gp.dna.dna_kl(gp.ctx)
        kl_ref = o.kl_divergence(V, W @ H)
        assert abs(kl_gpu - kl_ref) <= tol * abs(kl_ref), (kl_gpu, kl_ref)
    return flips


@pytest.mark.parametrize("kind", ["f32", "f32t", "f64"])
def test_plain_small_first_iterations(kind):
    """N=256 T=512 R=16: W and H after each of the first 5 DNA iterations."""
    _trajectory(workloads.plain_small(0), kind, 5)


@pytest.mark.parametrize("kind", ["f32", "f32t", "f64"])
def test_plain_small_mu_iterations(kind):
    _trajectory(workloads.plain_small(1), kind, 5, mu=True)


@pytest.mark.parametrize("kind", ["f32", "f32t", "f64"])
def test_mu_iterate_matches_oracle(kind):
    """mu_iterate (MU iterations with each half-step preparing the next) against the oracle's
    MU (eq. 11 then steps 16 / 29), and against the same iterations by mu_step.  Chained
    half-steps take the next eq. 7 / 14 denominators from the step 16 / 29 sums (the sum of a
    rescaled row is its old sum over the normaliser) instead of summing the rescaled factor
    again, so the two agree to rounding: 1e-6 (FP32) or 1e-13 (FP64) relative."""
    p = workloads.custom(150, 333, 12, seed=31)
    V = p.V.astype(np.float64)
    W, H = o.normalize_w_columns(p.W, p.H)
    for _ in range(4):
        W, H = o.mu_iteration(V, W, H)
    outs = []
    for chained in (True, False):
        with GpuProblem(p.V, p.W, p.H, kind) as gp:
            gp.dna.dna_normalize(gp.ctx, 1)
            if chained:
                gp.dna.mu_iterate(gp.ctx, 4)
            else:
                for _ in range(4):
                    gp.dna.mu_step(gp.ctx, 0)
                    gp.dna.mu_step(gp.ctx, 1)
            outs.append(gp.WH())
    Wg, Hg = outs[0]
    assert rel_fro(Wg, W) < TOL[kind] and rel_fro(Hg, H) < TOL[kind]
    assert rel_elem(Wg, W, "mu W") < ELEM_TOL[kind] and rel_elem(Hg, H, "mu H") < ELEM_TOL[kind]
    same = 1e-13 if kind == "f64" else 1e-6
    assert rel_fro(outs[0][0], outs[1][0]) < same and rel_fro(outs[0][1], outs[1][1]) < same


@pytest.mark.parametrize("kind", ["f32", "f32t", "f64"])
def test_plain_small_final_kl_free_running(kind):
    """50 free-running DNA iterations: final d_KL within 1e-3 relative (FP32)."""
    p = workloads.plain_small(0)
    _, _, costs = o.run(p.V, p.W, p.H, 50, "dna")
    with GpuProblem(p.V, p.W, p.H, kind) as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        kl0 = gp.dna.dna_kl(gp.ctx)
        assert abs(kl0 - costs[0]) <= 1e-6 * costs[0]
        prev = kl0
        for _ in range(50):
            gp.dna.dna_iterate(gp.ctx, 1)
            kl = gp.dna.dna_kl(gp.ctx)
            assert kl <= prev * (1 + 1e-6), (kl, prev)      # non-increasing (Section 2.4)
            prev = kl
    tol = 1e-3 if kind in ("f32", "f32t") else 1e-9
    assert abs(prev - costs[-1]) <= tol * costs[-1], (prev, costs[-1])


SHAPES = [(1, 1, 1), (3, 5, 2), (67, 131, 17), (130, 70, 33), (129, 200, 64),
          (200, 300, 129), (65, 129, 300), (40, 70, 512), (70, 513, 8)]


@pytest.mark.parametrize("kind", ["f32", "f32t", "f64"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_ragged_shapes(shape, kind):
    """Odd sizes: several tiles plus ragged tails in N, T and R (R up to 512, padded to 64,
    128, 256 or 512 on the tensor cores)."""
    N, T, R = shape
    p = workloads.custom(N, T, R, seed=N * 7 + T * 3 + R)
    _trajectory(p, kind, 2)


@pytest.mark.parametrize("kind", ["f32", "f32t", "f64"])
def test_regularised_and_limits(kind):
    """lambda, rho > 0 and non-default eps, alpha (eq. 2, Section 2.3)."""
    p = workloads.custom(90, 150, 12, seed=5)
    _trajectory(p, kind, 3, eps=0.05, alpha=1.5, rho=0.2, lam=0.3)


def test_regularised_large_rank_split():
    """lambda, rho > 0 and non-default eps, alpha through the split form's rank-512 kernels
    (R = 300: ratios + contraction pass 1, K-sliced pass 2)."""
    p = workloads.custom(257, 400, 300, seed=15)
    _trajectory(p, "f32t", 2, eps=0.05, alpha=1.5, rho=0.2, lam=0.3)


def test_costs_match_oracle():
    """Per-column and per-row candidate costs (steps 9, 14, 22, 27) against the oracle."""
    p = workloads.custom(100, 180, 10, seed=9)
    with GpuProblem(p.V, p.W, p.H, "f64") as gp:
        V = p.V.astype(np.float64)
        half = o.h_half_step(V, p.W, p.H)
        gp.dna.dna_step_H(gp.ctx)
        dm, dd = gp.costs(0)
        np.testing.assert_allclose(dm, half.d_mu, rtol=1e-11)
        np.testing.assert_allclose(dd, half.d_dna, rtol=1e-11)
        np.testing.assert_array_equal(gp.choice(0), half.choice)


def test_zero_rows_and_columns():
    """All-zero columns and rows of V: q = 0, the column goes to 0, MU kept on the tie."""
    p = workloads.custom(50, 60, 5, seed=2)
    V = p.V.copy()
    V[:, 7] = 0
    V[11, :] = 0
    _ = _trajectory(workloads.Problem("z", V, p.W0, p.H0, p.W, p.H, 0), "f64", 2)


@pytest.mark.parametrize("kind", ["f32", "f32t", "bf16", "bf16_r300"])
@pytest.mark.parametrize("fault", ["zero_w", "nan_h"])
def test_nonfinite_reported(kind, fault):
    """z = 0 where v > 0 (a zero factor) or a NaN entry is reported as DNA_ERR_NONFINITE
    after the half-step, not hidden (pass 1 checks for z = 0 where v > 0, pass 2 the
    finiteness of the cost sums); bf16_r300: the BF16 passes at padded rank 512."""
    import paper_1301_3389_gb300 as dna
    R = 300 if kind == "bf16_r300" else 4
    kind = "bf16" if kind == "bf16_r300" else kind
    p = workloads.custom(40, 50, R, seed=3)
    W, H = p.W.copy(), p.H.copy()
    if fault == "zero_w":
        W[:] = 0.0
    else:
        H[1, 7] = np.nan
    with GpuProblem(p.V, W, H, kind) as gp:
        gp.dna.dna_step_H(gp.ctx)
        assert gp.dna.dna_get_status(gp.ctx) == dna.DNA_ERR_NONFINITE


@pytest.mark.parametrize("kind", ["f32", "f32t"])
def test_run_host_matches_device_path(kind):
    """dna_run_host (host buffers, copies inside) equals the device-buffer path, with V in
    pageable memory (copied in) and in pinned memory (read across the host link by the
    transpose kernel, which writes the device copy), twice on one context."""
    import torch

    import paper_1301_3389_gb300 as dna
    p = workloads.custom(120, 200, 9, seed=4)
    with GpuProblem(p.V, p.W, p.H, kind) as gp:
        gp.dna.dna_iterate(gp.ctx, 3)
        kl_dev = gp.dna.dna_kl(gp.ctx)
        Wd, Hd = gp.WH()
    eng = dna.DNA_ENGINE_TENSOR if kind == "f32t" else dna.DNA_ENGINE_AUTO
    ctx = dna.dna_create(120, 200, 9, dna.make_opts(dtype=dna.DNA_F32, engine=eng))
    try:
        for pinned in (False, True, True):
            if pinned:
                V = torch.from_numpy(p.V).pin_memory()
                W = torch.from_numpy(p.W.copy()).pin_memory()
                H = torch.from_numpy(p.H.copy()).pin_memory()
            else:
                V, W, H = p.V, p.W.copy(), p.H.copy()
            kl = dna.dna_run_host(ctx, V, W, H, 3)
            Wn = W.numpy() if pinned else W
            Hn = H.numpy() if pinned else H
            assert kl == kl_dev, pinned
            np.testing.assert_array_equal(Wn, Wd.astype(np.float32))
            np.testing.assert_array_equal(Hn, Hd.astype(np.float32))
    finally:
        dna.dna_destroy(ctx)


def test_deterministic():
    """Two runs give bit-identical W and H (fixed-order reductions, no float atomics)."""
    p = workloads.custom(300, 500, 20, seed=6)
    outs = []
    for _ in range(2):
        with GpuProblem(p.V, p.W, p.H, "f32") as gp:
            gp.dna.dna_iterate(gp.ctx, 3)
            outs.append(gp.WH())
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


COST_RTOL = {"f32": 1e-5, "f32t": 1e-4, "f64": 1e-11}


@pytest.mark.parametrize("kind", ["f32", "f32t", "f64"])
def test_regularised_selection_costs(kind):
    """lambda = rho = 2 (eq. 2-5): from the GPU's own state at each half-step, the costs the
    GPU compares are the oracle's eq. 5 (eq. 4) costs d' + lambda sum_r h (rho sum_r w), and
    its selections are the oracle's except at near ties."""
    from gpu_helpers import NEAR_TIE
    p = workloads.custom(60, 140, 6, seed=21)
    V = p.V.astype(np.float64)
    reg = 2.0
    with GpuProblem(p.V, p.W, p.H, kind, rho=reg, lam=reg) as gp:
        gp.dna.dna_normalize(gp.ctx, 1)
        for _ in range(3):
            for which in (0, 1):
                W, H = gp.WH()
                if which == 0:
                    half = o.h_half_step(V, W, H, lam=reg)
                    gp.dna.dna_step_H(gp.ctx)
                else:
                    half = o.w_half_step(V, W, H, rho=reg)
                    gp.dna.dna_step_W(gp.ctx)
                dm, dd = gp.costs(which)
                np.testing.assert_allclose(dm, half.d_mu, rtol=COST_RTOL[kind])
                np.testing.assert_allclose(dd, half.d_dna, rtol=COST_RTOL[kind])
                diff = np.asarray(gp.choice(which), bool) != half.choice
                if diff.any():
                    assert half.margin[diff].max() < NEAR_TIE[kind]


def test_wait_timeout_reported_and_context_usable():
    """A bounded device wait that runs out (on a barrier nothing completes, nothing else in
    flight) is reported as DNA_ERR_TIMEOUT; the CUDA context stays usable and a context made
    afterwards runs a tensor-core iteration with a clean status."""
    import paper_1301_3389_gb300 as dna
    assert dna.LIB.dna_check_wait_timeout(2_000_000) == dna.DNA_ERR_TIMEOUT
    p = workloads.custom(120, 200, 16, seed=12)
    with GpuProblem(p.V, p.W, p.H, "f32t") as gp:
        gp.dna.dna_iterate(gp.ctx, 2)
        assert gp.dna.dna_get_status(gp.ctx) == dna.DNA_OK
    assert dna.LIB.dna_check_wait_timeout(0) == dna.DNA_ERR_ARG


@pytest.mark.parametrize("kind", ["f32", "f32t", "f64", "bf16"])
def test_iterate_graph_equals_direct(kind):
    """dna_use_graph: dna_iterate replays one captured iteration (after forming the first
    H half-step's operands from the current factors); W and H equal those of the direct
    launches bit for bit, across calls (the second call replays the same graph) and after
    a rebind (a new capture)."""
    import torch
    p = workloads.custom(150, 260, 20, seed=41)
    outs = []
    for graph in (False, True):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            with GpuProblem(p.V, p.W, p.H, kind) as gp:
                gp.dna.dna_set_stream(gp.ctx, stream)
                gp.dna.dna_use_graph(gp.ctx, graph)
                gp.dna.dna_normalize(gp.ctx, 1)
                gp.dna.dna_iterate(gp.ctx, 2)
                gp.dna.dna_iterate(gp.ctx, 1)
                gp.dna.dna_bind(gp.ctx, gp.V, gp.W, gp.H)
                gp.dna.dna_iterate(gp.ctx, 2)
                stream.synchronize()
                assert gp.dna.dna_get_status(gp.ctx) == 0
                outs.append(gp.WH())
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
