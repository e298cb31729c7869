"""FP64 CPU oracle for the Diagonalized Newton Algorithm (DNA) for KL-NMF.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
it is used by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg
of ``bench.py``.  It shares no code with the CUDA library.

It is plain NumPy in float64, written from the paper (H. Van hamme, "The Diagonalized
Newton Algorithm for Non-negative Matrix Factorization"), following Algorithm 1
(Section 3) in the paper's order and notation.  Matrix products use ``@`` (a library
primitive); there is no blocking, fusion or reordering beyond what Algorithm 1 states.

Notation (Section 2): V is N x T, W is N x R, H is R x T, Z = W H.  One DNA iteration
is an H half-step (Algorithm 1 steps 4-16) followed by a W half-step (steps 17-29).

Readings taken where the paper is silent, ambiguous or garbled (each is tested):

* Newton gain for a < 0: eq. 15, gain = h b / (h b - a), floored at eps (the listing of
  step 11 drops the factor h, which eq. 15's derivation requires).
* a >= 0: eq. 17, h + a / b, with the multiplicative gain capped at 1 + alpha, i.e.
  h + min(a / b, alpha h) (Section 2.3 "ceiling the multiplicative gain").
* a = 0 takes the additive branch (step 11 writes "A >= 0").
* The floor [x]_eps = max(x, eps) applies to the gain of the a < 0 branch only.
* "EM" in steps 15 and 28 is the MU candidate.
* Selection: the Newton candidate is kept iff d_DNA < d_MU; ties keep MU (step 15).
* The per-column cost compared in steps 9 and 14 is the eq. 5 sub-problem cost of that
  column minus a candidate-independent constant:
  d' = sum_{v>0} (-v log z) + sum z + lambda sum_r h_r, i.e. eq. 1 restricted to the
  column, plus the eq. 5 penalty lambda 1^t h, minus sum v log v - sum v.  Per row of W
  (steps 22, 27) the penalty is rho sum_r w_r (eq. 4).  Under eq. 9,
  sum z + lambda sum h = sum v for both candidates, so this orders them exactly as
  steps 9/14 do (1^t (V log Q)), and it stays a true cost comparison when eq. 9 holds only
  up to rounding.  (At lambda > 0, sum z alone differs between the candidates by
  -lambda sum h, so the penalty term cannot be dropped.)
* Zeros in V (note after Algorithm 1): q = v/z and v/z^2 are 0 where v = 0, and such
  entries add only z to the cost.
* z <= 0 where v > 0 cannot happen with positive factors; it raises NonFiniteError.
* Eq. 10 renormalisation with a zero denominator leaves the column unscaled.
* Descent selection (an optional variant; the paper's closing remark that refined step
  damping could avoid cost evaluations): keep the Newton candidate iff its eq. 5 cost is
  below that of the column the half-step starts from, else the MU candidate.  MU never
  increases the eq. 5 cost ([20], Section 2.1), so the kept candidate never does either
  (the guarantee of Section 2.4), and only the Newton candidate's cost is evaluated.
* The denominators of eq. 7 and eq. 14 are always the explicit (W^t 1)_r + lambda
  (H-step) and (H 1)_r + rho (W-step); steps 1, 16 and 29 normalise as written.
* A factor sum that is exactly zero (an all-zero column of W or row of H with no
  regularisation; Section 2 assumes this does not happen) is replaced by 1, in the
  eq. 7 / 14 denominators and in the step 1 / 16 / 29 normalisers alike.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

EPS = 0.01     # Section 4: epsilon = 0.01
ALPHA = 4.0    # Section 4: alpha = 4


class NonFiniteError(FloatingPointError):
    """z <= 0 at an entry with v > 0 (the cost would be infinite)."""


def f64(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float64)


def nonzero_sum(s: np.ndarray) -> np.ndarray:
    """A factor sum, with an exact zero replaced by 1 (module docstring)."""
    return np.where(s == 0, 1.0, s)


# ----------------------------------------------------------------------------- cost
def kl_divergence(V, Z) -> float:
    """Eq. 1: sum v log(v/z) - sum v + sum z, with v log(v/z) = 0 where v = 0."""
    V, Z = f64(V), f64(Z)
    pos = V > 0
    if np.any(Z[pos] <= 0):
        raise NonFiniteError("z <= 0 where v > 0")
    return float(np.sum(V[pos] * np.log(V[pos] / Z[pos])) - V.sum() + Z.sum())


def _neg_v_log_z(V, Z) -> np.ndarray:
    pos = V > 0
    if np.any(Z[pos] <= 0):
        raise NonFiniteError("z <= 0 where v > 0")
    out = np.zeros_like(Z)
    out[pos] = -V[pos] * np.log(Z[pos])
    return out


def column_cost(V, Z) -> np.ndarray:
    """Per-column cost d'_t = sum_n [v>0](-v log z) + sum_n z (steps 9 and 14)."""
    V, Z = f64(V), f64(Z)
    return _neg_v_log_z(V, Z).sum(axis=0) + Z.sum(axis=0)


def row_cost(V, Z) -> np.ndarray:
    """Per-row cost d'_n = sum_t [v>0](-v log z) + sum_t z (steps 22 and 27)."""
    V, Z = f64(V), f64(Z)
    return _neg_v_log_z(V, Z).sum(axis=1) + Z.sum(axis=1)


def ratio(V, Z, power: int) -> np.ndarray:
    """Q = V / Z (power 1, step 3) or Qbar = V / (Z * Z) (power 2, step 10); 0 where v = 0."""
    V, Z = f64(V), f64(Z)
    pos = V > 0
    if np.any(Z[pos] <= 0):
        raise NonFiniteError("z <= 0 where v > 0")
    out = np.zeros_like(Z)
    out[pos] = V[pos] / Z[pos] ** power
    return out


def kl_gradient(V, W, H):
    """Gradient of eq. 1 at Z = W H: (dW, dH, dV) = ((1 - Q) H^t, W^t (1 - Q), log(V / Z)),
    with Q = V / Z (0 where v = 0) and dV = 0 where v = 0 (derivative of v log(v/z) - v)."""
    V, W, H = f64(V), f64(W), f64(H)
    Z = W @ H
    Q = ratio(V, Z, 1)
    G = 1.0 - Q
    dV = np.zeros_like(Z)
    pos = V > 0
    dV[pos] = np.log(V[pos] / Z[pos])
    return G @ H.T, W.T @ G, dV


# ---------------------------------------------------------------------- normalisation
def normalize_w_columns(W, H, lam: float = 0.0):
    """Steps 1 and 29: divide column r of W by sum_n w_nr + lambda, multiply row r of H."""
    W, H = f64(W), f64(H)
    s = nonzero_sum(W.sum(axis=0) + lam)
    return W / s[None, :], H * s[:, None]


def normalize_h_rows(W, H, rho: float = 0.0):
    """Step 16: divide row r of H by sum_t h_rt + rho, multiply column r of W."""
    W, H = f64(W), f64(H)
    s = nonzero_sum(H.sum(axis=1) + rho)
    return W * s[None, :], H / s[:, None]


# ------------------------------------------------------------------------ candidates
def newton_candidate(X, A, B, eps: float = EPS, alpha: float = ALPHA) -> np.ndarray:
    """Element-wise diagonal-Newton update of steps 11 / 24.

    a < 0:  x * max(x b / (x b - a), eps)          (eq. 15 with the eps floor)
    a >= 0: x + min(a / b, alpha x)                (eq. 17 with the gain capped at 1+alpha)
    """
    X, A, B = f64(X), f64(A), f64(B)
    out = np.empty_like(X)
    neg = A < 0
    xb = X[neg] * B[neg]
    out[neg] = X[neg] * np.maximum(xb / (xb - A[neg]), eps)     # xb - a > 0 when a < 0
    nn = ~neg
    step = np.zeros_like(X[nn])
    bpos = B[nn] > 0
    step[bpos] = A[nn][bpos] / B[nn][bpos]
    out[nn] = X[nn] + np.minimum(step, alpha * X[nn])
    return out


@dataclass
class HalfStep:
    X: np.ndarray        # updated factor (before step 16 / 29 normalisation)
    X_mu: np.ndarray     # MU candidate (steps 6 / 19)
    X_dna: np.ndarray    # Newton candidate after eq. 10 renormalisation (steps 11 / 24)
    A: np.ndarray        # eq. 7 a, for every entry
    B: np.ndarray        # eq. 14 b, for every entry
    c: np.ndarray        # denominators (W^t 1 + lambda) or (H 1 + rho)
    d_mu: np.ndarray     # per-column (row) eq. 5 (eq. 4) cost of the MU candidate, less a constant
    d_dna: np.ndarray    # the same for the Newton candidate
    choice: np.ndarray   # True where the Newton candidate is kept
    margin: np.ndarray   # |d_dna - d_ref| / max(|d_ref|, tiny), d_ref the compared cost
    d_cur: np.ndarray = None   # eq. 5 cost of the starting factor (descent selection)


def h_half_step(V, W, H, eps: float = EPS, alpha: float = ALPHA, lam: float = 0.0,
                choice=None, selection: str = "paper") -> HalfStep:
    """Algorithm 1 steps 2-15 for H (W fixed).

    ``choice`` (bool per column) replaces the step-15 comparison when given: it lets a
    test replay another implementation's selection near ties.  ``selection="descent"``
    compares the Newton candidate with the starting column instead of with the MU
    candidate (module docstring).
    """
    V, W, H = f64(V), f64(W), f64(H)
    c = nonzero_sum(W.sum(axis=0) + lam)          # (W^t 1)_r + lambda   (eq. 7, 14)
    Z = W @ H                                     # step 2
    Q = ratio(V, Z, 1)                            # step 3
    W2 = W * W                                    # step 4
    A = (W.T @ Q) / c[:, None] - 1.0              # step 5 (eq. 7)
    H_mu = H + A * H                              # step 6 (eq. 11)
    Z_mu = W @ H_mu                               # step 7
    d_mu = column_cost(V, Z_mu) + lam * H_mu.sum(axis=0)     # steps 8-9, eq. 5 cost
    Qb = ratio(V, Z, 2)                           # step 10
    B = (W2.T @ Qb) / c[:, None]                  #         (eq. 14)
    H_dna = newton_candidate(H, A, B, eps, alpha)  # step 11 (eq. 15, 17)
    s = V.sum(axis=0)                             # 1^t V
    den = c @ H_dna                               # h^t (W^t 1 + lambda)   (eq. 10)
    scale = np.ones_like(s)
    ok = den > 0
    scale[ok] = s[ok] / den[ok]
    H_dna = H_dna * scale[None, :]
    Z_dna = W @ H_dna                             # step 12
    d_dna = column_cost(V, Z_dna) + lam * H_dna.sum(axis=0)  # steps 13-14, eq. 5 cost
    d_cur = column_cost(V, Z) + lam * H.sum(axis=0)          # starting column, eq. 5 cost
    d_ref = d_cur if selection == "descent" else d_mu
    if choice is None:
        choice = d_dna < d_ref                    # step 15, ties keep MU
    choice = np.asarray(choice, dtype=bool)
    H_new = np.where(choice[None, :], H_dna, H_mu)
    margin = np.abs(d_dna - d_ref) / np.maximum(np.abs(d_ref), 1e-300)
    return HalfStep(H_new, H_mu, H_dna, A, B, c, d_mu, d_dna, choice, margin, d_cur)


def w_half_step(V, W, H, eps: float = EPS, alpha: float = ALPHA, rho: float = 0.0,
                choice=None, selection: str = "paper") -> HalfStep:
    """Algorithm 1 steps 17-28 for W (H fixed); selection per row of W."""
    V, W, H = f64(V), f64(W), f64(H)
    c = nonzero_sum(H.sum(axis=1) + rho)          # (H 1)_r + rho
    Z = W @ H                                     # carried Z of step 15 (WH is unchanged by step 16)
    Q = ratio(V, Z, 1)
    H2 = H * H                                    # step 17
    A = (Q @ H.T) / c[None, :] - 1.0              # step 18
    W_mu = W + A * W                              # step 19
    Z_mu = W_mu @ H                               # step 20
    d_mu = row_cost(V, Z_mu) + rho * W_mu.sum(axis=1)        # steps 21-22, eq. 4 cost
    Qb = ratio(V, Z, 2)                           # step 23
    B = (Qb @ H2.T) / c[None, :]
    W_dna = newton_candidate(W, A, B, eps, alpha)  # step 24
    s = V.sum(axis=1)                             # V 1
    den = W_dna @ c
    scale = np.ones_like(s)
    ok = den > 0
    scale[ok] = s[ok] / den[ok]
    W_dna = W_dna * scale[:, None]
    Z_dna = W_dna @ H                             # step 25
    d_dna = row_cost(V, Z_dna) + rho * W_dna.sum(axis=1)     # steps 26-27, eq. 4 cost
    d_cur = row_cost(V, Z) + rho * W.sum(axis=1)             # starting row, eq. 4 cost
    d_ref = d_cur if selection == "descent" else d_mu
    if choice is None:
        choice = d_dna < d_ref                    # step 28, ties keep MU
    choice = np.asarray(choice, dtype=bool)
    W_new = np.where(choice[:, None], W_dna, W_mu)
    margin = np.abs(d_dna - d_ref) / np.maximum(np.abs(d_ref), 1e-300)
    return HalfStep(W_new, W_mu, W_dna, A, B, c, d_mu, d_dna, choice, margin, d_cur)


# ----------------------------------------------------------------------- full steps
def dna_step_h(V, W, H, eps=EPS, alpha=ALPHA, rho=0.0, lam=0.0, choice=None,
               selection="paper"):
    """Steps 4-16: H half-step then the step-16 normalisation.  Returns (W, H, HalfStep)."""
    hs = h_half_step(V, W, H, eps, alpha, lam, choice, selection)
    W2, H2 = normalize_h_rows(W, hs.X, rho)
    return W2, H2, hs


def dna_step_w(V, W, H, eps=EPS, alpha=ALPHA, rho=0.0, lam=0.0, choice=None,
               selection="paper"):
    """Steps 17-29: W half-step then the step-29 normalisation.  Returns (W, H, HalfStep)."""
    ws = w_half_step(V, W, H, eps, alpha, rho, choice, selection)
    W2, H2 = normalize_w_columns(ws.X, H, lam)
    return W2, H2, ws


def dna_iteration(V, W, H, eps=EPS, alpha=ALPHA, rho=0.0, lam=0.0,
                  choice_h=None, choice_w=None, selection="paper"):
    """One DNA iteration (steps 4-29).  Returns (W, H, HalfStep_H, HalfStep_W)."""
    W, H, hs = dna_step_h(V, W, H, eps, alpha, rho, lam, choice_h, selection)
    W, H, ws = dna_step_w(V, W, H, eps, alpha, rho, lam, choice_w, selection)
    return W, H, hs, ws


def mu_h(V, W, H, lam: float = 0.0) -> np.ndarray:
    """Eq. 11 for every column: h <- h (W^t q) / (W^t 1 + lambda)."""
    V, W, H = f64(V), f64(W), f64(H)
    c = nonzero_sum(W.sum(axis=0) + lam)
    Q = ratio(V, W @ H, 1)
    return H * (W.T @ Q) / c[:, None]


def mu_w(V, W, H, rho: float = 0.0) -> np.ndarray:
    """Eq. 11 transposed (Section 2 symmetry): w <- w (q H^t) / (H 1 + rho)."""
    V, W, H = f64(V), f64(W), f64(H)
    c = nonzero_sum(H.sum(axis=1) + rho)
    Q = ratio(V, W @ H, 1)
    return W * (Q @ H.T) / c[None, :]


def mu_step_h(V, W, H, rho=0.0, lam=0.0):
    """MU steps 5-6 then step 16.  Returns (W, H)."""
    return normalize_h_rows(W, mu_h(V, W, H, lam), rho)


def mu_step_w(V, W, H, rho=0.0, lam=0.0):
    """MU steps 18-19 then step 29.  Returns (W, H)."""
    return normalize_w_columns(mu_w(V, W, H, rho), H, lam)


def mu_iteration(V, W, H, rho=0.0, lam=0.0):
    W, H = mu_step_h(V, W, H, rho, lam)
    return mu_step_w(V, W, H, rho, lam)


def run(V, W, H, iters: int, algo: str = "dna", eps=EPS, alpha=ALPHA, rho=0.0, lam=0.0,
        log_cost: bool = True):
    """Step 1 then ``iters`` iterations of DNA, DNA with descent selection ("dna_descent")
    or MU.  Returns (W, H, costs)."""
    W, H = normalize_w_columns(W, H, lam)
    costs = [kl_divergence(V, W @ H)] if log_cost else []
    for _ in range(iters):
        if algo == "dna":
            W, H, _, _ = dna_iteration(V, W, H, eps, alpha, rho, lam)
        elif algo == "dna_descent":
            W, H, _, _ = dna_iteration(V, W, H, eps, alpha, rho, lam, selection="descent")
        elif algo == "mu":
            W, H = mu_iteration(V, W, H, rho, lam)
        else:
            raise ValueError(algo)
        if log_cost:
            costs.append(kl_divergence(V, W @ H))
    return W, H, costs
