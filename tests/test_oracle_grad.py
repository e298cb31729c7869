"""Pins for the differentiation-form references (CPU): the analytic d_KL gradient and the
autograd gradient of the unrolled H solve, both against central finite differences."""
import numpy as np
import torch

import pins
from oracle import dna as o
from oracle import unrolled as u


def test_kl_gradient_finite_differences():
    V, W, H = pins.rand_problem(6, 5, 3, 21)
    dW, dH, dV = o.kl_gradient(V, W, H)
    d = 1e-6
    for M, G in ((W, dW), (H, dH), (V, dV)):
        for idx in [(0, 0), (1, 2), (M.shape[0] - 1, M.shape[1] - 1)]:
            if M is V and V[idx] == 0:
                continue
            Mp, Mm = M.copy(), M.copy()
            Mp[idx] += d
            Mm[idx] -= d
            args_p = [Mp if X is M else X for X in (V, W, H)]
            args_m = [Mm if X is M else X for X in (V, W, H)]
            fd = (o.kl_divergence(args_p[0], args_p[1] @ args_p[2]) -
                  o.kl_divergence(args_m[0], args_m[1] @ args_m[2])) / (2 * d)
            assert abs(G[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (idx, G[idx], fd)


def test_torch_step_matches_numpy_oracle():
    V, W, H = pins.rand_problem(12, 9, 4, 22)
    hs = o.h_half_step(V, W, H)
    Hn, ch = u.h_step(torch.tensor(V), torch.tensor(W), torch.tensor(H))
    np.testing.assert_allclose(Hn.numpy(), hs.X, rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(ch.numpy(), hs.choice)
    hs2 = o.h_half_step(V, W, H, eps=0.3, alpha=0.5, lam=0.2)
    Hn2, _ = u.h_step(torch.tensor(V), torch.tensor(W), torch.tensor(H), eps=0.3, alpha=0.5, lam=0.2)
    np.testing.assert_allclose(Hn2.numpy(), hs2.X, rtol=1e-12, atol=1e-14)


def test_unrolled_gradient_finite_differences():
    V, W, H0 = pins.rand_problem(9, 7, 3, 23)
    K, mu = 4, 1e-2
    loss, gV, gH, used = u.loss_and_grads(V, W, H0, K, mu)
    d = 1e-6
    checked = 0
    for M, G, which in ((H0, gH, "H"), (V, gV, "V")):
        for idx in [(0, 0), (1, 3), (2, 6), (M.shape[0] - 1, 1), (3, 2), (4, 4)]:
            if idx[0] >= M.shape[0] or idx[1] >= M.shape[1]:
                continue
            if which == "V" and V[idx] == 0:
                continue   # v log v is not differentiable at v = 0
            Mp, Mm = M.copy(), M.copy()
            Mp[idx] += d
            Mm[idx] -= d
            lp, _, _, up = u.loss_and_grads(Mp if which == "V" else V, W, Mp if which == "H" else H0, K, mu)
            lm, _, _, um = u.loss_and_grads(Mm if which == "V" else V, W, Mm if which == "H" else H0, K, mu)
            if any((a != b).any() for a, b in zip(up, used)) or any((a != b).any() for a, b in zip(um, used)):
                continue   # a selection changes inside +-d: not a smooth point
            fd = (lp - lm) / (2 * d)
            assert abs(G[idx] - fd) <= 1e-5 * max(1.0, abs(fd)), (which, idx, G[idx], fd)
            checked += 1
    assert checked >= 5


def test_unrolled_w_gradient_finite_differences():
    """dL/dW through the unrolled solve (every step's Z, A, B and column sums, plus the
    loss's own Z = W H_K) against central differences of the forward, with lambda = 0 and
    lambda > 0 (eq. 7's denominators), at points where no selection, floor or cap flips."""
    checked = 0
    for lam, seed in ((0.0, 24), (0.3, 25)):
        V, W, H0 = pins.rand_problem(9, 7, 3, seed)
        K, mu = 4, 1e-2
        loss, gV, gW, gH, used = u.loss_and_grads_vwh(V, W, H0, K, mu, lam=lam)
        # the V and H0 gradients are those of loss_and_grads (W's being a variable adds
        # nothing to them)
        if lam == 0.0:
            _, gV2, gH2, _ = u.loss_and_grads(V, W, H0, K, mu)
            np.testing.assert_allclose(gV, gV2, rtol=1e-12, atol=1e-14)
            np.testing.assert_allclose(gH, gH2, rtol=1e-12, atol=1e-14)
        d = 1e-6
        for idx in [(0, 0), (1, 2), (4, 1), (8, 2), (6, 0), (3, 1)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += d
            Wm[idx] -= d
            lp, _, _, _, up = u.loss_and_grads_vwh(V, Wp, H0, K, mu, lam=lam)
            lm, _, _, _, um = u.loss_and_grads_vwh(V, Wm, H0, K, mu, lam=lam)
            if any((a != b).any() for a, b in zip(up, used)) or any((a != b).any() for a, b in zip(um, used)):
                continue
            fd = (lp - lm) / (2 * d)
            assert abs(gW[idx] - fd) <= 1e-5 * max(1.0, abs(fd)), (lam, idx, gW[idx], fd)
            checked += 1
    assert checked >= 8


def test_step_vjp_chain_matches_unrolled_autograd():
    """Chaining step_vjp over the oracle's own states gives loss_and_grads_vwh's gradients."""
    V, W, H0 = pins.rand_problem(9, 7, 3, 26)
    K, mu = 4, 1e-2
    loss, gV, gW, gH, used = u.loss_and_grads_vwh(V, W, H0, K, mu)
    Vt, Wt = torch.tensor(V, dtype=torch.float64), torch.tensor(W, dtype=torch.float64)
    states = [torch.tensor(H0, dtype=torch.float64)]
    for k in range(K):
        states.append(u.h_step(Vt, Wt, states[-1], choice=torch.tensor(used[k]))[0])
    # the loss's own gradients at H_K
    Vl = Vt.clone().requires_grad_(True)
    Wl = Wt.clone().requires_grad_(True)
    HK = states[-1].clone().requires_grad_(True)
    lk = u.kl(Vl, Wl @ HK) + 0.5 * mu * (HK * HK).sum()
    hb, vb, wb = (g.numpy() for g in torch.autograd.grad(lk, (HK, Vl, Wl)))
    for k in reversed(range(K)):
        hb, dv, dw = u.step_vjp(V, W, states[k].numpy(), used[k], hb)
        vb, wb = vb + dv, wb + dw
    np.testing.assert_allclose(hb, gH, rtol=1e-10, atol=1e-12 * np.abs(gH).max())
    np.testing.assert_allclose(vb, gV, rtol=1e-10, atol=1e-12 * np.abs(gV).max())
    np.testing.assert_allclose(wb, gW, rtol=1e-10, atol=1e-12 * np.abs(gW).max())
