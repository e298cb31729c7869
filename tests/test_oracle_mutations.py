"""Planted mistakes in the oracle (on the CPU): every one must trip at least one pin.

Each mutation is a textual change to a copy of ``oracle/dna.py`` (a dropped term, a wrong
sign or index, a transposed operand, a missing limit), loaded as a separate module.  The
pins of ``pins.py`` are then run against that copy.
"""
import importlib.util
import os

import pytest

import pins
from oracle import dna as oracle_dna

SRC_PATH = oracle_dna.__file__

MUTATIONS = {
    "newton_gain_as_listed": ("xb / (xb - A[neg])", "B[neg] / (B[neg] - A[neg])"),
    "a_wrong_sign": ("A = (W.T @ Q) / c[:, None] - 1.0", "A = 1.0 - (W.T @ Q) / c[:, None]"),
    "b_without_square": ("B = (W2.T @ Qb) / c[:, None]", "B = (W.T @ Qb) / c[:, None]"),
    "qbar_power_one": ("Qb = ratio(V, Z, 2)                           # step 10",
                       "Qb = ratio(V, Z, 1)"),
    "no_renorm_h": ("H_dna = H_dna * scale[None, :]", "H_dna = H_dna"),
    "no_renorm_w": ("W_dna = W_dna * scale[:, None]", "W_dna = W_dna"),
    "no_alpha_cap": ("np.minimum(step, alpha * X[nn])", "step"),
    "no_eps_floor": ("np.maximum(xb / (xb - A[neg]), eps)", "(xb / (xb - A[neg]))"),
    "cost_without_sum_z": ("_neg_v_log_z(V, Z).sum(axis=0) + Z.sum(axis=0)",
                           "_neg_v_log_z(V, Z).sum(axis=0)"),
    "log_without_v": ("out[pos] = -V[pos] * np.log(Z[pos])", "out[pos] = -np.log(Z[pos])"),
    "kl_without_sum_z": ("- V.sum() + Z.sum())", "- V.sum())"),
    "w_b_without_square": ("B = (Qb @ H2.T) / c[None, :]", "B = (Qb @ H.T) / c[None, :]"),
    "w_a_missing_denominator": ("A = (Q @ H.T) / c[None, :] - 1.0", "A = (Q @ H.T) - 1.0"),
    "mu_h_missing_denominator": ("return H * (W.T @ Q) / c[:, None]", "return H * (W.T @ Q)"),
    "h_denominator_without_lambda": ("c = nonzero_sum(W.sum(axis=0) + lam)          # (W^t 1)_r",
                                     "c = nonzero_sum(W.sum(axis=0))          # (W^t 1)_r"),
    "step16_multiplies_h": ("return W * s[None, :], H / s[:, None]",
                            "return W / s[None, :], H * s[:, None]"),
    "selection_inverted": ("choice = d_dna < d_ref                    # step 15",
                           "choice = d_dna > d_ref                    # step 15"),
    "descent_compares_mu": ("d_ref = d_cur if selection == \"descent\" else d_mu\n    if choice is None:\n        choice = d_dna < d_ref                    # step 15",
                            "d_ref = d_mu\n    if choice is None:\n        choice = d_dna < d_ref                    # step 15"),
    "descent_cost_without_lambda": ("d_cur = column_cost(V, Z) + lam * H.sum(axis=0)",
                                    "d_cur = column_cost(V, Z)"),
    "descent_w_cost_without_rho": ("d_cur = row_cost(V, Z) + rho * W.sum(axis=1)",
                                   "d_cur = row_cost(V, Z)"),
    "renorm_uses_row_sums": ("s = V.sum(axis=0)                             # 1^t V",
                             "s = V.sum()                             # 1^t V"),
    "h_cost_without_lambda_term": ("column_cost(V, Z_mu) + lam * H_mu.sum(axis=0)",
                                   "column_cost(V, Z_mu)"),
    "h_dna_cost_without_lambda_term": ("column_cost(V, Z_dna) + lam * H_dna.sum(axis=0)",
                                       "column_cost(V, Z_dna)"),
    "w_cost_without_rho_term": ("row_cost(V, Z_mu) + rho * W_mu.sum(axis=1)",
                                "row_cost(V, Z_mu)"),
    "w_dna_cost_without_rho_term": ("row_cost(V, Z_dna) + rho * W_dna.sum(axis=1)",
                                    "row_cost(V, Z_dna)"),
}

EXTRA = [lambda: pins.check_a_b_finite_differences(lam=0.3),
         lambda: pins.check_w_a_b_finite_differences(rho=0.2),
         lambda: pins.check_transpose_symmetry(reg=0.15)]


def _mutant(name, old, new):
    src = open(SRC_PATH).read()
    assert src.count(old) == 1, f"mutation {name}: pattern found {src.count(old)} times"
    spec = importlib.util.spec_from_loader(f"oracle_mutant_{name}", loader=None)
    mod = importlib.util.module_from_spec(spec)
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, monkeypatch):
    mod = _mutant(name, *MUTATIONS[name])
    monkeypatch.setattr(pins, "o", mod)
    caught = []
    for check in list(pins.ALL) + EXTRA:
        try:
            check()
        except Exception as e:          # an assertion or a crash both expose the mistake
            caught.append((getattr(check, "__name__", "extra"), type(e).__name__))
    assert caught, f"no pin detects the planted mistake {name}"


def test_unmutated_passes_everything():
    for check in list(pins.ALL) + EXTRA:
        check()
