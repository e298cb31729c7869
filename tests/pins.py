"""Checks that pin the FP64 oracle to what the paper and the mathematics fix.

Each ``check_*`` raises AssertionError on failure.  They are run as tests in
``test_oracle_pins.py`` and, against deliberately broken copies of the oracle, in
``test_oracle_mutations.py`` (which shows that a plausible mistake trips at least one).
"""
from __future__ import annotations

import os

import numpy as np
from scipy import optimize, special

from oracle import dna as o

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rand_problem(N, T, R, seed, zeros=0.3, scale=1.0):
    g = np.random.default_rng(seed)
    W = g.uniform(0.1, 1.0, (N, R))
    H = g.uniform(0.1, 1.0, (R, T))
    V = g.poisson(scale * 2.0, (N, T)).astype(np.float64)
    V *= g.random((N, T)) >= zeros
    V[:, 0] += 1.0          # no all-zero column / row
    V[0, :] += 1.0
    return V, W, H


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "V":
                rows = " ".join(vals).split("/")
                out[key] = np.array([[float(x) for x in r.split()] for r in rows])
            else:
                out[key] = np.array([float(x) for x in vals])
    return out


# -------------------------------------------------------------------------- the cost
def check_kl_definition():
    """Eq. 1 against SciPy's element-wise kl_div, >= 0, and 0 at an exact factorisation."""
    V, W, H = rand_problem(9, 7, 3, 1)
    Z = W @ H
    ref = float(np.sum(special.kl_div(V, Z)))           # x log(x/y) - x + y, 0 log 0 = 0
    got = o.kl_divergence(V, Z)
    assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)
    assert got > 0
    g = np.random.default_rng(2)
    W0, H0 = g.gamma(0.5, 1.0, (9, 3)), g.gamma(0.5, 1.0, (3, 7))
    D = g.uniform(0.5, 2.0, 3)
    V0 = W0 @ H0
    exact = o.kl_divergence(V0, (W0 * D) @ (H0 / D[:, None]))
    assert abs(exact) <= 1e-12 * V0.sum(), exact


def check_costs_sum_to_kl():
    """Per-column and per-row costs plus the constant sum v log v - sum v give eq. 1."""
    V, W, H = rand_problem(8, 6, 3, 3)
    Z = W @ H
    pos = V > 0
    const = float(np.sum(V[pos] * np.log(V[pos])) - V.sum())
    kl = float(np.sum(special.kl_div(V, Z)))
    assert abs(o.column_cost(V, Z).sum() + const - kl) <= 1e-11 * abs(kl)
    assert abs(o.row_cost(V, Z).sum() + const - kl) <= 1e-11 * abs(kl)
    cols = o.column_cost(V, Z)
    for t in range(V.shape[1]):
        v, z = V[:, t], Z[:, t]
        ref = float(np.sum(special.kl_div(v, z))) - float(np.sum(v[v > 0] * np.log(v[v > 0]))) + v.sum()
        assert abs(cols[t] - ref) <= 1e-11 * max(1.0, abs(ref))


# --------------------------------------------------------------- a and b (eq. 7, 14)
def _obj_h(V, W, h, t, lam):
    return o.kl_divergence(V[:, t:t + 1], W @ h[:, None]) + lam * h.sum()


def check_a_b_finite_differences(lam=0.0):
    """a_r = -(d cost / d h_r) / c_r and b_r = -d a_r / d h_r (eq. 6, 7, 14)."""
    V, W, H = rand_problem(7, 4, 3, 5)
    hs = o.h_half_step(V, W, H, lam=lam)
    c = W.sum(axis=0) + lam
    d = 1e-6
    for t in range(V.shape[1]):
        for r in range(W.shape[1]):
            hp, hm = H[:, t].copy(), H[:, t].copy()
            hp[r] += d
            hm[r] -= d
            g = (_obj_h(V, W, hp, t, lam) - _obj_h(V, W, hm, t, lam)) / (2 * d)
            a_fd = -g / c[r]
            assert abs(hs.A[r, t] - a_fd) <= 1e-6 * max(1.0, abs(a_fd)), (r, t, hs.A[r, t], a_fd)
            Hp, Hm = H.copy(), H.copy()
            Hp[r, t] += d
            Hm[r, t] -= d
            ap = o.h_half_step(V, W, Hp, lam=lam).A[r, t]
            am = o.h_half_step(V, W, Hm, lam=lam).A[r, t]
            b_fd = -(ap - am) / (2 * d)
            assert abs(hs.B[r, t] - b_fd) <= 1e-5 * max(1.0, abs(b_fd)), (r, t, hs.B[r, t], b_fd)


def check_w_a_b_finite_differences(rho=0.0):
    """The W-step a and b are minus the scaled gradient and its diagonal derivative in W."""
    V, W, H = rand_problem(5, 6, 3, 6)
    ws = o.w_half_step(V, W, H, rho=rho)
    c = H.sum(axis=1) + rho
    d = 1e-6

    def obj(Wx):
        return o.kl_divergence(V, Wx @ H) + rho * Wx.sum()

    for n in range(V.shape[0]):
        for r in range(W.shape[1]):
            Wp, Wm = W.copy(), W.copy()
            Wp[n, r] += d
            Wm[n, r] -= d
            a_fd = -(obj(Wp) - obj(Wm)) / (2 * d) / c[r]
            assert abs(ws.A[n, r] - a_fd) <= 1e-6 * max(1.0, abs(a_fd)), (n, r)
            b_fd = -(o.w_half_step(V, Wp, H, rho=rho).A[n, r] -
                     o.w_half_step(V, Wm, H, rho=rho).A[n, r]) / (2 * d)
            assert abs(ws.B[n, r] - b_fd) <= 1e-5 * max(1.0, abs(b_fd)), (n, r)


# ---------------------------------------------------------------- closed forms
def check_r1_golden():
    """Hand-worked rank-1 H half-step (tests/golden/r1_closed_form.txt)."""
    g = read_golden("r1_closed_form.txt")
    W = g["W"][:, None]
    H = g["H"][None, :]
    V = g["V"]
    hs = o.h_half_step(V, W, H)
    np.testing.assert_allclose(hs.A[0], g["A"], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(hs.B[0], g["B"], rtol=1e-14)
    np.testing.assert_allclose(o.newton_candidate(H, hs.A, hs.B)[0], g["H_dna_before_renorm"],
                               rtol=1e-14)
    np.testing.assert_allclose(hs.X_mu[0], g["H_after_half_step"], rtol=1e-14)
    np.testing.assert_allclose(hs.X_dna[0], g["H_after_half_step"], rtol=1e-14)
    np.testing.assert_allclose(hs.X[0], g["H_after_half_step"], rtol=1e-14)
    W2, H2, _ = o.dna_step_h(V, W, H)
    np.testing.assert_allclose(H2[0], g["H_after_step16"], rtol=1e-14)
    np.testing.assert_allclose(W2[:, 0], g["W_after_step16"], rtol=1e-14)


def check_r1_random():
    """At R = 1 one H half-step returns h* = sum v / sum w per column (and mirror for W)."""
    V, W, H = rand_problem(11, 9, 1, 7)
    hs = o.h_half_step(V, W, H)
    hstar = V.sum(axis=0) / W.sum()
    np.testing.assert_allclose(hs.X_mu[0], hstar, rtol=1e-12)
    np.testing.assert_allclose(hs.X_dna[0], hstar, rtol=1e-12)
    ws = o.w_half_step(V, W, H)
    wstar = V.sum(axis=1) / H.sum()
    np.testing.assert_allclose(ws.X_mu[:, 0], wstar, rtol=1e-12)
    np.testing.assert_allclose(ws.X_dna[:, 0], wstar, rtol=1e-12)
    np.testing.assert_allclose(o.mu_h(V, W, H)[0], hstar, rtol=1e-12)      # eq. 11
    np.testing.assert_allclose(o.mu_w(V, W, H)[:, 0], wstar, rtol=1e-12)


def check_step_limits_golden():
    """Hand-worked eps floor and alpha cap (tests/golden/step_limits.txt)."""
    rows = []
    with open(os.path.join(GOLDEN, "step_limits.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    x, a, b, want = (np.array(col) for col in zip(*rows))
    got = o.newton_candidate(x, a, b, eps=0.01, alpha=4.0)
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)


# -------------------------------------------------------------------- invariants
def check_eq9_invariant():
    """After a half-step, sum_r c_r h_rt = sum_n v_nt for every column (eq. 9), both candidates."""
    V, W, H = rand_problem(12, 10, 4, 8)
    hs = o.h_half_step(V, W, H)
    s = V.sum(axis=0)
    for X in (hs.X_mu, hs.X_dna, hs.X):
        np.testing.assert_allclose(hs.c @ X, s, rtol=1e-12)
    ws = o.w_half_step(V, W, H)
    s = V.sum(axis=1)
    for X in (ws.X_mu, ws.X_dna, ws.X):
        np.testing.assert_allclose(X @ ws.c, s, rtol=1e-12)


def check_monotone(iters=25):
    """Per-column (H-step) and per-row (W-step) cost never increases, for DNA and MU (Section 2.4)."""
    V, W, H = rand_problem(16, 12, 4, 9)
    W, H = o.normalize_w_columns(W, H)
    Wm, Hm = W.copy(), H.copy()
    for _ in range(iters):
        before = o.column_cost(V, W @ H)
        W, H, hs = o.dna_step_h(V, W, H)
        after = o.column_cost(V, W @ H)
        assert np.all(after <= before + 1e-12 * np.abs(before)), "DNA H-step increased a column cost"
        assert np.all(np.minimum(hs.d_mu, hs.d_dna) <= hs.d_mu)
        before = o.row_cost(V, W @ H)
        W, H, ws = o.dna_step_w(V, W, H)
        after = o.row_cost(V, W @ H)
        assert np.all(after <= before + 1e-12 * np.abs(before)), "DNA W-step increased a row cost"
        before = o.column_cost(V, Wm @ Hm)
        Wm, Hm = o.mu_step_h(V, Wm, Hm)
        assert np.all(o.column_cost(V, Wm @ Hm) <= before + 1e-12 * np.abs(before)), "MU H"
        before = o.row_cost(V, Wm @ Hm)
        Wm, Hm = o.mu_step_w(V, Wm, Hm)
        assert np.all(o.row_cost(V, Wm @ Hm) <= before + 1e-12 * np.abs(before)), "MU W"


def _eq5_cost_columns(V, W, X, lam):
    """Eq. 5 per column, evaluated directly: sum kl_div(v, W h) + lambda 1^t h."""
    return np.array([float(np.sum(special.kl_div(V[:, t], W @ X[:, t]))) + lam * X[:, t].sum()
                     for t in range(V.shape[1])])


def check_regularised_selection(reg=2.0, seeds=range(8), iters=3):
    """At lambda, rho > 0 the selection orders the candidates by the eq. 5 (eq. 4) cost.

    For every column (row) of several H (W) half-steps, the Newton candidate is kept iff
    its sub-problem cost d_KL + lambda 1^t h (per row: + rho 1^t w), evaluated here directly
    with SciPy's kl_div, is below the MU candidate's (Section 2.4; ties and rounding-level
    margins are skipped), and the kept candidate's cost is not above that of the factor the
    half-step started from (MU never increases it, [20])."""
    for seed in seeds:
        V, W, H = rand_problem(12, 30, 4, 100 + seed)
        W, H = o.normalize_w_columns(W, H, reg)
        for _ in range(iters):
            hs = o.h_half_step(V, W, H, lam=reg)
            e_mu = _eq5_cost_columns(V, W, hs.X_mu, reg)
            e_dna = _eq5_cost_columns(V, W, hs.X_dna, reg)
            clear = np.abs(e_dna - e_mu) > 1e-10 * np.abs(e_mu)
            assert np.array_equal(hs.choice[clear], (e_dna < e_mu)[clear]), \
                f"H-step selection disagrees with the eq. 5 cost (seed {seed})"
            e_old = _eq5_cost_columns(V, W, H, reg)
            e_new = _eq5_cost_columns(V, W, hs.X, reg)
            assert np.all(e_new <= e_old + 1e-10 * np.abs(e_old)), "eq. 5 cost increased"
            W, H, _ = o.dna_step_h(V, W, H, rho=reg, lam=reg)
            ws = o.w_half_step(V, W, H, rho=reg)
            e_mu = _eq5_cost_columns(V.T, H.T, ws.X_mu.T, reg)
            e_dna = _eq5_cost_columns(V.T, H.T, ws.X_dna.T, reg)
            clear = np.abs(e_dna - e_mu) > 1e-10 * np.abs(e_mu)
            assert np.array_equal(ws.choice[clear], (e_dna < e_mu)[clear]), \
                f"W-step selection disagrees with the eq. 4 cost (seed {seed})"
            e_old = _eq5_cost_columns(V.T, H.T, W.T, reg)
            e_new = _eq5_cost_columns(V.T, H.T, ws.X.T, reg)
            assert np.all(e_new <= e_old + 1e-10 * np.abs(e_old)), "eq. 4 cost increased"
            W, H, _ = o.dna_step_w(V, W, H, rho=reg, lam=reg)


def check_descent_selection(reg_values=(0.0, 1.5), seeds=range(6), iters=3):
    """Descent selection: the Newton candidate is kept iff its eq. 5 (eq. 4) cost, evaluated
    directly with SciPy, is below that of the starting column (row), so the kept candidate
    never raises it; and every column the paper's rule gives to Newton, descent does too
    (d_DNA < d_MU <= d_start, MU being non-increasing)."""
    for reg in reg_values:
        for seed in seeds:
            V, W, H = rand_problem(12, 30, 4, 300 + seed)
            W, H = o.normalize_w_columns(W, H, reg)
            for _ in range(iters):
                hs = o.h_half_step(V, W, H, lam=reg, selection="descent")
                paper = o.h_half_step(V, W, H, lam=reg)
                e_cur = _eq5_cost_columns(V, W, H, reg)
                e_dna = _eq5_cost_columns(V, W, hs.X_dna, reg)
                clear = np.abs(e_dna - e_cur) > 1e-10 * np.abs(e_cur)
                assert np.array_equal(hs.choice[clear], (e_dna < e_cur)[clear]), "H descent"
                e_new = _eq5_cost_columns(V, W, hs.X, reg)
                assert np.all(e_new <= e_cur + 1e-10 * np.abs(e_cur)), "descent raised a cost"
                assert np.all(hs.choice[paper.choice]), "paper's Newton columns must stay Newton"
                W, H, _ = o.dna_step_h(V, W, H, rho=reg, lam=reg, selection="descent")
                ws = o.w_half_step(V, W, H, rho=reg, selection="descent")
                e_cur = _eq5_cost_columns(V.T, H.T, W.T, reg)
                e_dna = _eq5_cost_columns(V.T, H.T, ws.X_dna.T, reg)
                clear = np.abs(e_dna - e_cur) > 1e-10 * np.abs(e_cur)
                assert np.array_equal(ws.choice[clear], (e_dna < e_cur)[clear]), "W descent"
                W, H, _ = o.dna_step_w(V, W, H, rho=reg, lam=reg, selection="descent")


def check_sparse_identities():
    """On a sparse term-count V (the paper's second workload, Section 4.2), the oracle's
    quantities are sums over the stored non-zeros only (the note after Algorithm 1): A and
    B of eq. 7 / 14 recomputed entry by entry over the non-zeros of each column, and each
    column cost over the non-zeros plus sum_n z = sum_r (sum_n w_nr) h_r."""
    import workloads
    sp = workloads.sparse_custom(40, 60, 3, 0.08, seed=4)
    V = sp.dense().astype(np.float64)
    W, H = sp.W.astype(np.float64), sp.H.astype(np.float64)
    hs = o.h_half_step(V, W, H)
    c = W.sum(axis=0)
    rows = np.repeat(np.arange(sp.N), np.diff(sp.row_ptr))
    A = np.zeros_like(H)
    B = np.zeros_like(H)
    cost = (c @ hs.X_mu).copy()                   # sum_n z of the MU candidate
    for k in range(sp.nnz):
        n, t, v = rows[k], sp.col_idx[k], float(sp.vals[k])
        z = float(W[n] @ H[:, t])
        A[:, t] += W[n] * v / z
        B[:, t] += W[n] ** 2 * v / z ** 2
        cost[t] -= v * np.log(float(W[n] @ hs.X_mu[:, t]))
    np.testing.assert_allclose(hs.A, A / c[:, None] - 1.0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(hs.B, B / c[:, None], rtol=1e-12)
    np.testing.assert_allclose(hs.d_mu, cost, rtol=1e-12)


def check_fixed_point():
    """At an exact factorisation a = 0, so MU and DNA leave W and H unchanged (Section 2.1-2.2)."""
    g = np.random.default_rng(10)
    W0, H0 = g.gamma(0.5, 1.0, (10, 3)) + 0.05, g.gamma(0.5, 1.0, (3, 8)) + 0.05
    V = W0 @ H0
    W, H = o.normalize_w_columns(W0, H0)
    W1, H1, _, _ = o.dna_iteration(V, W, H)
    np.testing.assert_allclose(W1, W, rtol=1e-10)
    np.testing.assert_allclose(H1, H, rtol=1e-10)
    W2, H2 = o.mu_iteration(V, W, H)
    np.testing.assert_allclose(W2, W, rtol=1e-10)
    np.testing.assert_allclose(H2, H, rtol=1e-10)


def check_transpose_symmetry(reg=0.0):
    """The W half-step equals the H half-step on (V^t, H^t, W^t), transposed (Section 2)."""
    V, W, H = rand_problem(9, 13, 3, 11)
    ws = o.w_half_step(V, W, H, rho=reg)
    hs = o.h_half_step(V.T, H.T, W.T, lam=reg)
    np.testing.assert_allclose(ws.X, hs.X.T, rtol=1e-12)
    np.testing.assert_allclose(ws.A, hs.A.T, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(ws.B, hs.B.T, rtol=1e-12)
    np.testing.assert_array_equal(ws.choice, hs.choice)


def check_scale_equivariance():
    """W D, D^-1 H gives D^-1 times the updated H (eq. 7, 11, 14, 15, 17, 10 are scale-covariant)."""
    V, W, H = rand_problem(10, 9, 3, 12)
    D = np.array([0.25, 3.0, 1.7])
    a = o.h_half_step(V, W, H)
    b = o.h_half_step(V, W * D, H / D[:, None])
    np.testing.assert_allclose(b.X, a.X / D[:, None], rtol=1e-11)
    np.testing.assert_array_equal(a.choice, b.choice)


def check_normalisation_steps():
    """Steps 1/29 and 16 leave W H unchanged and make column (row) sums equal to 1."""
    V, W, H = rand_problem(6, 5, 3, 13)
    W1, H1 = o.normalize_w_columns(W, H)
    np.testing.assert_allclose(W1.sum(axis=0), 1.0, rtol=1e-14)
    np.testing.assert_allclose(W1 @ H1, W @ H, rtol=1e-13)
    W2, H2 = o.normalize_h_rows(W, H)
    np.testing.assert_allclose(H2.sum(axis=1), 1.0, rtol=1e-14)
    np.testing.assert_allclose(W2 @ H2, W @ H, rtol=1e-13)


# ------------------------------------------------------------------- brute force
def brute_force_column(v, W):
    """Minimum of eq. 5 (lambda = 0) for R = 2 by 1-D bounded search on the eq. 9 segment."""
    c = W.sum(axis=0)
    s = v.sum()

    def f(u):                       # h = (s - c1 u) / c0, u in [0, s / c1]
        h = np.array([(s - c[1] * u) / c[0], u])
        return float(np.sum(special.kl_div(v, W @ h)))

    hi = s / c[1]
    grid = np.linspace(0.0, hi, 2001)
    vals = [f(u) for u in grid]
    k = int(np.argmin(vals))
    lo_b, hi_b = grid[max(k - 1, 0)], grid[min(k + 1, len(grid) - 1)]
    res = optimize.minimize_scalar(f, bounds=(lo_b, hi_b), method="bounded",
                                   options={"xatol": 1e-13 * max(hi, 1.0)})
    u = res.x if res.fun <= min(vals) else grid[k]
    return np.array([(s - c[1] * u) / c[0], u]), min(res.fun, min(vals))


def _brute_force_case(W, V, H, steps):
    for _ in range(steps):
        H = o.h_half_step(V, W, H).X
    for t in range(V.shape[1]):
        h_bf, f_bf = brute_force_column(V[:, t], W)
        f = float(np.sum(special.kl_div(V[:, t], W @ H[:, t])))
        assert f <= f_bf + 1e-9 * max(1.0, f_bf), (t, f, f_bf)
        assert abs(f - f_bf) <= 1e-9 * max(1.0, f_bf), (t, f, f_bf)
        np.testing.assert_allclose(H[:, t], h_bf, rtol=1e-4, atol=1e-6)
    hs = o.h_half_step(V, W, H)
    kkt = np.abs(hs.A * H)
    assert kkt.max() <= 1e-8, kkt.max()
    assert np.all(hs.A[H < 1e-12] <= 1e-8)


def check_brute_force_tiny():
    """Repeated DNA H half-steps at fixed W reach the brute-force optimum of eq. 5 and its KKT point.

    Well-separated W columns: the diagonal Hessian of eq. 14 is a good model and 60 steps
    suffice.  Nearly collinear columns: eq. 13's off-diagonal terms are large, the diagonal
    Newton step converges only linearly (about 0.93 per step here), so 700 steps are run.
    """
    g = np.random.default_rng(14)
    V = g.poisson(3.0, (4, 5)).astype(np.float64) + np.array([[1, 0, 0, 2, 0]] * 4)
    W_sep = np.array([[1.0, 0.1], [0.9, 0.2], [0.1, 1.0], [0.2, 0.8]])
    _brute_force_case(W_sep, V, g.uniform(0.1, 1.0, (2, 5)), 60)
    W_col = g.uniform(0.1, 1.0, (4, 2))
    _brute_force_case(W_col, V, g.uniform(0.1, 1.0, (2, 5)), 700)


ALL = [check_kl_definition, check_costs_sum_to_kl, check_a_b_finite_differences,
       check_w_a_b_finite_differences, check_r1_golden, check_r1_random,
       check_step_limits_golden, check_eq9_invariant, check_monotone, check_fixed_point,
       check_transpose_symmetry, check_scale_equivariance, check_normalisation_steps,
       check_brute_force_tiny, check_regularised_selection, check_sparse_identities,
       check_descent_selection]
