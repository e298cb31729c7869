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
NEAR_TIE = {"f32": 1e-5, "f32t": 1e-4, "f64": 1e-12, "bf16": 1e-2}
# Trajectory tolerance (Frobenius, relative) of the split FP32 form for R > 300, in place of
# the FP32 forms' 1e-4.  Its hi + lo operands carry about 17 significant bits (relative
# representation error up to 2^-17) against 24 for float32: in an FP64 emulation of that
# representation alone, the W, H trajectory of a (520, 640, 512) problem leaves the exact
# one by 5.2e-5 after 2 iterations (9.2e-5 after 5), on top of the float32 rounding that
# the CUDA-core form shows there (3.6e-5 after 2 iterations, 6.7e-5 after 5); the bound is
# that sum with a factor of 2.  The one-step element-wise bound is unchanged.
SPLIT_LARGE_R_TOL = 2e-4

# Element-wise check beside every Frobenius one: the largest |x - x_ref| / |x_ref| over
# the entries with |x_ref| > ELEM_FLOOR * max |x_ref| (smaller entries carry no relative
# accuracy worth testing: they are the ones an eps floor or a strong MU decrease has
# driven towards zero, and their absolute error is already bounded by the Frobenius
# check).  ELEM_TOL per form; derivation in the module docstring of test_gpu_parity.py.
ELEM_FLOOR = 1e-6
# free-running trajectories (errors of earlier steps carried along): measured maxima over
# the parity tests 1.4e-3 (f32), 8.6e-3 (f32t at R <= 128), 5e-12 (f64), about 3x margin;
# the split form at R = 300 and 512 reaches 7.7e-3 and 1.7e-2 (its operand representation
# error grows with R, see SPLIT_LARGE_R_TOL), inside the same bound
ELEM_TOL = {"f32": 5e-3, "f32t": 2e-2, "f64": 1e-9}


def rel_fro(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a - b))


# Relative error of the contractions (1 + a) = (W^t q) / c and b per form, for the
# element-wise bound of step_elementwise (which widens it by ELEM_K): bf16 operands 4u = 2^-7 (z: two rounded
# operands, q rounded again, w rounded); split bf16 products about 2^-15 each, with the
# tensor pipe's truncating float32 accumulation, 2^-13; CUDA-core float32 sums of up to
# 2^14 terms, 2^-16; float64, 2^-40.
DELTA = {"bf16": 2.0 ** -7, "f32t": 2.0 ** -13, "f32": 2.0 ** -16, "f64": 2.0 ** -40}
ELEM_K = 4.0


def _newton_error(X0, A, B, X_dna, c, eps, alpha, kd):
    """Per entry (R x O orientation), a bound on the error of the Newton candidate when
    (1 + a) and b carry relative errors up to kd.

    The candidate of eq. 15 / 17 with its floor and cap is non-decreasing in a (the gain
    x b / (x b - a) rises with a, the step a / b too, and both branches give x at a = 0),
    and monotone in b within each branch, so over the box a' in a +- kd |1 + a|,
    b' in b (1 +- kd) its extremes lie at the four corners: their largest distance from
    the centre bounds the error, kinks (the sign of a, the eps floor, the alpha cap)
    included.  Eq. 10 then scales the column by s / sum_r c_r x'_r: each entry also moves
    by kd of itself and by the column's c-weighted error relative to its c-weighted mass."""
    raw = o.newton_candidate(X0, A, B, eps, alpha)
    da = kd * np.abs(1.0 + A)
    D = np.zeros_like(raw)
    for sa in (-1.0, 1.0):
        for sb in (-1.0, 1.0):
            corner = o.newton_candidate(X0, A + sa * da, B * (1.0 + sb * kd), eps, alpha)
            D = np.maximum(D, np.abs(corner - raw))
    scale = np.where(raw > 0, X_dna / np.where(raw > 0, raw, 1.0), 1.0)
    D = D * np.abs(scale)
    mass = c @ np.abs(X_dna)
    col = np.where(mass > 0, (c @ D) / np.where(mass > 0, mass, 1.0), 0.0)
    # the deviation is scaled by the implementation's own eq. 10 factor, off by kd + col
    return D * (1.0 + kd + col[None, :]) + np.abs(X_dna) * (kd + col[None, :])


def step_elementwise(half, which, W0, H0, Wg, Hg, kind, eps=o.EPS, alpha=o.ALPHA, reg_norm=0.0,
                     label="", sig=None, check_y=True):
    """Element-wise check of one GPU half-step against the oracle's half-step `half` taken
    from the same state (W0, H0), with the GPU's selections replayed in `half.choice`.

    Bound per entry, with kd = ELEM_K * DELTA[kind]: the chosen candidate's error E (the
    Newton candidate: _newton_error; the MU candidate x (1 + a): kd |x|, as accurate as
    (1 + a)), plus |x| rho_r, rho_r = sum_o E / sum_o |x| over the row that the step 16 / 29
    normalisation divides by its sum.  Returns the largest |x_gpu - x_ref| / bound over W
    and H (<= 1 passes)."""
    delta = DELTA[kind]
    kd = ELEM_K * delta
    if which == 0:     # H step: R x T orientation
        X0, A, B, Xd, Xm, ch = H0, half.A, half.B, half.X_dna, half.X_mu, half.choice[None, :]
    else:              # W step: transpose to R x N
        X0, A, B, Xd, Xm, ch = W0.T, half.A.T, half.B.T, half.X_dna.T, half.X_mu.T, half.choice[None, :]
    Bc = np.where(ch, _newton_error(X0, A, B, Xd, half.c, eps, alpha, kd), kd * np.abs(Xm))
    Xc = np.where(ch, Xd, Xm)
    rs = np.abs(Xc).sum(axis=1)
    rho = np.where(rs > 0, Bc.sum(axis=1) / np.where(rs > 0, rs, 1.0), 0.0)
    if sig is None:   # the step 16 / 29 normaliser of the oracle's own stepped factor
        sig = Xc.sum(axis=1) + reg_norm
        sig = np.where(sig == 0, 1.0, sig)
    else:             # a normaliser given (read from the GPU: sampled columns or rows)
        rho = np.zeros_like(rho)
    x_ref = Xc / sig[:, None]                       # step 16 / 29 on the stepped factor
    x_bnd = (Bc + np.abs(Xc) * rho[:, None]) / np.abs(sig)[:, None]
    if which == 0:
        y_ref = W0 * sig[None, :]
        y_bnd = np.abs(y_ref) * (rho[None, :] + kd)
        xg, yg = Hg, Wg
    else:
        x_ref, x_bnd = x_ref.T, x_bnd.T
        y_ref = H0 * sig[:, None]
        y_bnd = np.abs(y_ref) * (rho[:, None] + kd)
        xg, yg = Wg, Hg
    # entries below ELEM_FLOOR of the largest carry no relative accuracy (see ELEM_FLOOR)
    x_bnd = x_bnd + delta * ELEM_FLOOR * float(np.abs(x_ref).max(initial=0.0)) + 1e-300
    y_bnd = y_bnd + delta * ELEM_FLOOR * float(np.abs(y_ref).max(initial=0.0)) + 1e-300
    worst = float(np.max(np.abs(xg - x_ref) / x_bnd, initial=0.0))
    if check_y:
        worst = max(worst, float(np.max(np.abs(yg - y_ref) / y_bnd, initial=0.0)))
    path = os.environ.get("DNA_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(f"{os.environ.get('PYTEST_CURRENT_TEST', '?').split(' ')[0]} bound-{kind} "
                    f"{label} {worst:.3e}\n")
    return worst


def log_value(label: str, val: float) -> float:
    """Append (test, label, value) to the DNA_PARITY_LOG file, if that variable is set."""
    path = os.environ.get("DNA_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(f"{os.environ.get('PYTEST_CURRENT_TEST', '?').split(' ')[0]} {label} {val:.3e}\n")
    return val


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
        selection = opts.pop("selection", None)
        self.tdt = torch.float64 if dtype == "f64" else torch.float32
        self.N, self.T = V.shape
        self.R = W.shape[1]
        self.V = torch.from_numpy(np.ascontiguousarray(V)).to("cuda", self.tdt)
        self.W = torch.from_numpy(np.ascontiguousarray(W)).to("cuda", self.tdt)
        self.H = torch.from_numpy(np.ascontiguousarray(H)).to("cuda", self.tdt)
        self.ctx = dna.dna_create(self.N, self.T, self.R, dna.make_opts(dtype=code, **opts))
        dna.dna_set_stream(self.ctx)
        dna.dna_bind(self.ctx, self.V, self.W, self.H)
        if selection == "descent":
            dna.dna_set_selection(self.ctx, dna.DNA_SELECT_DESCENT)

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


def one_step_check(gp: GpuProblem, which, W0, H0, opts=None, label=""):
    """After a GPU DNA half-step taken from the state (W0, H0) (read before the step): the
    oracle's half-step from the same state with the GPU's selections replayed, checked
    element-wise by step_elementwise.  Returns the worst ratio (<= 1 passes)."""
    import dataclasses
    opts = opts or {}
    eps = opts.get("eps", o.EPS)
    alpha = opts.get("alpha", o.ALPHA)
    rho = opts.get("rho", 0.0)
    lam = opts.get("lam", 0.0)
    V = gp_V(gp)
    sel = opts.get("selection", "paper")
    if which == 0:
        half = o.h_half_step(V, W0, H0, eps, alpha, lam, selection=sel)
    else:
        half = o.w_half_step(V, W0, H0, eps, alpha, rho, selection=sel)
    mask, _ = replay_choice(half, gp.choice(which), gp.kind)
    half = dataclasses.replace(half, choice=mask)
    Wg, Hg = gp.WH()
    return step_elementwise(half, which, W0, H0, Wg, Hg, gp.kind, eps, alpha,
                            rho if which == 0 else lam, label)


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
    sel = opts.get("selection", "paper")
    Wg0, Hg0 = gp.WH()            # the GPU's state before the step, for the one-step check
    if which == 0:
        dna.dna_step_H(gp.ctx)
        half = o.h_half_step(V, W, H, eps, alpha, lam, selection=sel)
        mask, nflip = replay_choice(half, gp.choice(0), gp.kind)
        W2, H2, _ = o.dna_step_h(V, W, H, eps, alpha, rho, lam, choice=mask)
    else:
        dna.dna_step_W(gp.ctx)
        half = o.w_half_step(V, W, H, eps, alpha, rho, selection=sel)
        mask, nflip = replay_choice(half, gp.choice(1), gp.kind)
        W2, H2, _ = o.dna_step_w(V, W, H, eps, alpha, rho, lam, choice=mask)
    ratio = one_step_check(gp, which, Wg0, Hg0, opts, "step")
    assert ratio <= 1.0, f"element-wise error above its bound (ratio {ratio:.3g})"
    return W2, H2, nflip


def gp_V(gp):
    if not hasattr(gp, "_V64"):
        gp._V64 = gp.V.double().cpu().numpy()
    return gp._V64


class SparseGpuProblem(GpuProblem):
    """A sparse-V problem (workloads.SparseProblem, CSR) bound to a dna_create_sparse context;
    the same interface as GpuProblem, with the dense V kept for the oracle."""

    def __init__(self, sp, dtype="f32", V_dense=None, **opts):
        import torch

        import paper_1301_3389_gb300 as dna
        self.dna = dna
        self.torch = torch
        self.kind = dtype
        code = {"f64": dna.DNA_F64, "f32": dna.DNA_F32}[dtype]
        self.tdt = torch.float64 if dtype == "f64" else torch.float32
        self.N, self.T = sp.N, sp.T
        self.R = sp.W.shape[1]
        self.rp = torch.from_numpy(sp.row_ptr).cuda()
        self.ci = torch.from_numpy(sp.col_idx).cuda()
        self.vals = torch.from_numpy(sp.vals).to("cuda", self.tdt)
        self.W = torch.from_numpy(np.ascontiguousarray(sp.W)).to("cuda", self.tdt)
        self.H = torch.from_numpy(np.ascontiguousarray(sp.H)).to("cuda", self.tdt)
        self.ctx = dna.dna_create_sparse(self.N, self.T, self.R, sp.nnz,
                                         dna.make_opts(dtype=code, **opts))
        dna.dna_set_stream(self.ctx)
        dna.dna_bind_csr(self.ctx, self.rp, self.ci, self.vals, self.W, self.H)
        if V_dense is not None:
            self._V64 = np.asarray(V_dense, dtype=np.float64)
