"""Helpers for the GPU parity tests: a problem bound to the CUDA library, and comparisons
with the FP64 oracle."""
from __future__ import annotations

import os

import numpy as np

from oracle import dna as o

# Tolerances (written in the tests that use them):
#  * W and H after each of the first iterations: 1e-4 relative (Frobenius) in FP32,
#    1e-10 in FP64 (only the summation order differs).
#  * final d_KL: 1e-3 relative in FP32.
#  * selection: a column (row) may differ from the oracle only where the oracle's
#    |d_dna - d_mu| / |d_mu| is below NEAR_TIE; the oracle then replays the GPU's choice.
#  * "f32t" is the FP32 form on the tensor cores (split hi + lo bf16 products, relative
#    error per product below about 2^-15): the same W, H and d_KL tolerances as "f32",
#    near ties up to 1e-4.
NEAR_TIE = {"f32": 1e-5, "f32t": 1e-4, "f64": 1e-12}

# Element-wise check beside every Frobenius one: the largest |x - x_ref| / |x_ref| over
# the entries with |x_ref| > ELEM_FLOOR * max |x_ref| (smaller entries carry no relative
# accuracy worth testing: they are the ones an eps floor or a strong MU decrease has
# driven towards zero, and their absolute error is already bounded by the Frobenius
# check).  ELEM_TOL per form; derivation in the module docstring of test_gpu_parity.py.
ELEM_FLOOR = 1e-6
ELEM_TOL = {"f32": 2e-3, "f32t": 5e-3, "f64": 1e-8}


def rel_fro(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a - b))


def rel_elem(a, b, label: str = "", floor: float = ELEM_FLOOR) -> float:
    """max |a - b| / |b| over the entries of b above floor * max |b| (see ELEM_FLOOR).

    With DNA_PARITY_LOG set, each value is also appended to that file (label, value), so a
    run can report the measured element-wise errors."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = float(np.abs(b).max()) if b.size else 0.0
    if m == 0.0:
        val = float(np.abs(a).max()) if a.size else 0.0
    else:
        sel = np.abs(b) > floor * m
        val = float((np.abs(a[sel] - b[sel]) / np.abs(b[sel])).max())
    path = os.environ.get("DNA_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(f"{os.environ.get('PYTEST_CURRENT_TEST', '?').split(' ')[0]} {label} {val:.3e}\n")
    return val


class GpuProblem:
    """V, W, H on the GPU, bound to a library context."""

    def __init__(self, V, W, H, dtype="f32", **opts):
        import torch

        import paper_1301_3389_gb300 as dna
        self.dna = dna
        self.torch = torch
        self.kind = dtype
        code = {"f64": dna.DNA_F64, "f32": dna.DNA_F32, "f32t": dna.DNA_F32,
                "bf16": dna.DNA_BF16}[dtype]
        if dtype == "f32t":
            opts.setdefault("engine", dna.DNA_ENGINE_TENSOR)
        self.tdt = torch.float64 if dtype == "f64" else torch.float32
        self.N, self.T = V.shape
        self.R = W.shape[1]
        self.V = torch.from_numpy(np.ascontiguousarray(V)).to("cuda", self.tdt)
        self.W = torch.from_numpy(np.ascontiguousarray(W)).to("cuda", self.tdt)
        self.H = torch.from_numpy(np.ascontiguousarray(H)).to("cuda", self.tdt)
        self.ctx = dna.dna_create(self.N, self.T, self.R, dna.make_opts(dtype=code, **opts))
        dna.dna_set_stream(self.ctx)
        dna.dna_bind(self.ctx, self.V, self.W, self.H)

    def WH(self):
        self.torch.cuda.synchronize()
        return (self.W.double().cpu().numpy(), self.H.double().cpu().numpy())

    def choice(self, which):
        return self.dna.dna_get_choice(self.ctx, which, self.N if which else self.T)

    def costs(self, which):
        return self.dna.dna_get_costs(self.ctx, which, self.N if which else self.T)

    def close(self):
        if self.ctx:
            self.dna.dna_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def replay_choice(half, gpu_choice, kind):
    """Check the GPU selection against the oracle's and return the mask to replay.

    Where they differ, the oracle's relative cost margin must be a near tie.
    """
    gpu_choice = np.asarray(gpu_choice, dtype=bool)
    diff = gpu_choice != half.choice
    if np.any(diff):
        worst = float(half.margin[diff].max())
        assert worst < NEAR_TIE[kind], (
            f"{int(diff.sum())} selections differ from the oracle with margin up to {worst:.3e}")
    return gpu_choice, int(diff.sum())


def step_pair(gp: GpuProblem, W, H, which, mu=False, opts=None):
    """Run one GPU half-step (or MU step) and the matching oracle step (replaying the
    GPU selection).  Returns (W_ref, H_ref, n_flipped)."""
    opts = opts or {}
    dna = gp.dna
    eps = opts.get("eps", o.EPS)
    alpha = opts.get("alpha", o.ALPHA)
    rho = opts.get("rho", 0.0)
    lam = opts.get("lam", 0.0)
    if mu:
        dna.mu_step(gp.ctx, which)
        if which == 0:
            W2, H2 = o.mu_step_h(gp_V(gp), W, H, rho, lam)
        else:
            W2, H2 = o.mu_step_w(gp_V(gp), W, H, rho, lam)
        return W2, H2, 0
    V = gp_V(gp)
    if which == 0:
        dna.dna_step_H(gp.ctx)
        half = o.h_half_step(V, W, H, eps, alpha, lam)
        mask, nflip = replay_choice(half, gp.choice(0), gp.kind)
        W2, H2, _ = o.dna_step_h(V, W, H, eps, alpha, rho, lam, choice=mask)
    else:
        dna.dna_step_W(gp.ctx)
        half = o.w_half_step(V, W, H, eps, alpha, rho)
        mask, nflip = replay_choice(half, gp.choice(1), gp.kind)
        W2, H2, _ = o.dna_step_w(V, W, H, eps, alpha, rho, lam, choice=mask)
    return W2, H2, nflip


def gp_V(gp):
    if not hasattr(gp, "_V64"):
        gp._V64 = gp.V.double().cpu().numpy()
    return gp._V64
