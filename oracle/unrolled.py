"""Reference for the differentiation form: K DNA H half-steps at fixed W, in plain PyTorch
float64 CPU ops so that torch.autograd gives the reference gradient.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Each step is Algorithm 1 steps 2-15
(eq. 7, 10, 11, 14, 15, 17, selection of Section 2.4) without the step-16 normalisation,
written with the same readings as oracle/dna.py (which its forward is tested against).
The selection, the eps floor and the alpha cap are piecewise choices: autograd
differentiates the branch that was taken.  ``choices`` replays given selections.
Derivatives at v = 0: q = v / z is smooth there (derivative 1 / z); the loss term
v log(v / z) - v is not, and its derivative is taken as 0 (as dna_kl_backward does).
"""
from __future__ import annotations

import torch

EPS = 0.01
ALPHA = 4.0


def h_step(V, W, H, eps=EPS, alpha=ALPHA, lam=0.0, choice=None):
    """One H half-step (steps 2-15) at fixed W.  Returns (H_new, choice)."""
    c = W.sum(dim=0) + lam
    c = torch.where(c == 0, torch.ones_like(c), c)
    Z = W @ H                                              # step 2
    pos = V > 0
    # q = v / z and qbar = v / z^2 (0 where v = 0); as functions of v they are smooth at
    # v = 0, so their derivative there is 1 / z (resp. 1 / z^2): divide wherever z > 0
    Zs = torch.where(Z > 0, Z, torch.ones_like(Z))
    Q = V / Zs                                             # step 3
    Qb = V / (Zs * Zs)
    A = (W.t() @ Q) / c[:, None] - 1.0                     # step 5 (eq. 7)
    B = ((W * W).t() @ Qb) / c[:, None]                    # step 10 (eq. 14)
    H_mu = H + A * H                                       # step 6 (eq. 11)
    neg = A < 0
    xb = H * B
    den = torch.where(neg, xb - A, torch.ones_like(A))
    gain = torch.where(neg, xb / den, torch.ones_like(A))
    g_neg = H * torch.where(gain > eps, gain, torch.full_like(gain, eps))   # eq. 15, floor
    Bs = torch.where(B > 0, B, torch.ones_like(B))
    step = torch.where(B > 0, A / Bs, torch.zeros_like(A))
    cap = alpha * H
    g_pos = H + torch.where(step < cap, step, cap)         # eq. 17, cap
    H_dna = torch.where(neg, g_neg, g_pos)                 # step 11
    s = V.sum(dim=0)
    D = (c[:, None] * H_dna).sum(dim=0)                    # eq. 10
    scale = torch.where(D > 0, s / torch.where(D > 0, D, torch.ones_like(D)), torch.ones_like(D))
    H_dna = H_dna * scale[None, :]
    if choice is None:
        def cost(Zc):                                      # steps 9, 14 (reading of the cost)
            Zp = torch.where(pos, Zc, torch.ones_like(Zc))
            return torch.where(pos, -V * torch.log(Zp), torch.zeros_like(Zc)).sum(0) + Zc.sum(0)
        with torch.no_grad():
            choice = cost(W @ H_dna) < cost(W @ H_mu)      # step 15, ties keep MU
    H_new = torch.where(choice[None, :], H_dna, H_mu)
    return H_new, choice


def unrolled(V, W, H0, K, eps=EPS, alpha=ALPHA, lam=0.0, choices=None):
    """K steps from H0; returns (H_K, list of choices)."""
    H = H0
    used = []
    for k in range(K):
        H, ch = h_step(V, W, H, eps, alpha, lam, None if choices is None else choices[k])
        used.append(ch)
    return H, used


def kl(V, Z):
    """Eq. 1 in torch (for losses), as sum_{v>0} (v log(v/z) - v) + sum z: the same value,
    with the derivative in v taken as 0 where v = 0 (v log v - v is not differentiable
    there), the reading of dna_kl_backward."""
    pos = V > 0
    Zp = torch.where(pos, Z, torch.ones_like(Z))
    Vp = torch.where(pos, V, torch.ones_like(V))
    return torch.where(pos, V * torch.log(Vp / Zp) - V, torch.zeros_like(Z)).sum() + Z.sum()


def loss_and_grads_vwh(V, W, H0, K, mu, choices=None, lam=0.0):
    """As loss_and_grads, with W a variable of the solve too (and lambda >= 0 in eq. 7):
    (loss, dL/dV, dL/dW, dL/dH0, choices).  dL/dW collects every path by which W enters:
    the loss's Z = W H_K and, in every step, Z = W H, A = W^t Q, B = (W o W)^t Qbar and the
    column sums c = W^t 1 + lambda (eq. 7, 10, 14)."""
    V = torch.as_tensor(V, dtype=torch.float64).clone().requires_grad_(True)
    W = torch.as_tensor(W, dtype=torch.float64).clone().requires_grad_(True)
    H0 = torch.as_tensor(H0, dtype=torch.float64).clone().requires_grad_(True)
    HK, used = unrolled(V, W, H0, K, lam=lam, choices=choices)
    loss = kl(V, W @ HK) + 0.5 * mu * (HK * HK).sum()
    gV, gW, gH = torch.autograd.grad(loss, (V, W, H0))
    return float(loss.detach()), gV.numpy(), gW.numpy(), gH.numpy(), [u.numpy() for u in used]


def step_vjp(V, W, Hk, choice, Hbar_next, lam=0.0):
    """Vector-Jacobian product of one step at a GIVEN state Hk (with the selection held):
    (dL/dH_k, the step's share of dL/dV, the step's share of dL/dW) for
    dL/dH_{k+1} = Hbar_next, by autograd of h_step in float64.  Chaining these over the
    states of another run (e.g. a float32 solve) gives the exact gradient along that run's
    own trajectory, which separates the accuracy of an adjoint from that of the forward."""
    V = torch.as_tensor(V, dtype=torch.float64).clone().requires_grad_(True)
    W = torch.as_tensor(W, dtype=torch.float64).clone().requires_grad_(True)
    Hk = torch.as_tensor(Hk, dtype=torch.float64).clone().requires_grad_(True)
    Hn, _ = h_step(V, W, Hk, lam=lam, choice=torch.as_tensor(choice, dtype=torch.bool))
    gH, gV, gW = torch.autograd.grad(Hn, (Hk, V, W),
                                     grad_outputs=torch.as_tensor(Hbar_next, dtype=torch.float64))
    return gH.numpy(), gV.numpy(), gW.numpy()


def loss_and_grads(V, W, H0, K, mu, choices=None):
    """Loss d_KL(V, W H_K) + (mu / 2) |H_K|^2 and its gradients w.r.t. V and H0 (float64)."""
    V = torch.as_tensor(V, dtype=torch.float64).clone().requires_grad_(True)
    W = torch.as_tensor(W, dtype=torch.float64)
    H0 = torch.as_tensor(H0, dtype=torch.float64).clone().requires_grad_(True)
    HK, used = unrolled(V, W, H0, K, choices=choices)
    loss = kl(V, W @ HK) + 0.5 * mu * (HK * HK).sum()
    gV, gH = torch.autograd.grad(loss, (V, H0))
    return float(loss.detach()), gV.numpy(), gH.numpy(), [u.numpy() for u in used]
