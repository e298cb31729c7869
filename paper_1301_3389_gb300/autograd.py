"""torch.autograd wrappers over the C ABI (argument marshalling only).

* ``KLDiv.apply(V, W, H)``: d_KL(V, W H) of eq. 1; the backward pass is
  ``dna_kl_backward`` (dW = (1 - Q) H^t, dH = W^t (1 - Q), dV = log(V / Z)).
* ``UnrolledDNAH.apply(V, W, H0, K, every)``: K DNA H half-steps with W held fixed by the
  solve (``dna_step_H_fixed``), returning H_K; the backward pass runs
  ``dna_step_H_adjoint_w`` in reverse, recomputing the states of each segment from
  checkpoints kept every ``every`` steps.  Gradients flow to V, H0 and, when W requires
  one, to W (through every step's Z = W H, A = W^t Q, B = (W o W)^t Qbar and the column
  sums W^t 1 + lambda).

Tensors are CUDA float32 (F32 form) or float64 (F64 form), contiguous, row-major.

Library contexts (their device workspace) are kept per thread and per (N, T, R, form,
device) and bound afresh to the call's tensors each time (``dna_bind`` prepares
everything from them), so repeated calls allocate nothing; a call that fails destroys its
context.  ``release_contexts()`` frees the calling thread's contexts.
"""
from __future__ import annotations

import threading

import torch

from . import _lib as L

_local = threading.local()


def _pool() -> dict:
    pool = getattr(_local, "pool", None)
    if pool is None:
        pool = _local.pool = {}
    return pool


def release_contexts() -> None:
    """Destroy the library contexts this thread keeps for the autograd wrappers."""
    pool = _pool()
    for ctx in pool.values():
        L.dna_destroy(ctx)
    pool.clear()


class _Ctx:
    """A pooled context bound to (V, W, H) for the duration of a ``with`` block."""

    def __init__(self, V, W, H):
        N, T = V.shape
        R = W.shape[1]
        dtype = L.DNA_F64 if V.dtype == torch.float64 else L.DNA_F32
        self.key = (N, T, R, dtype, V.device.index)
        pool = _pool()
        ctx = pool.pop(self.key, None)   # taken out while in use (re-entrant calls get their own)
        if ctx is None:
            ctx = L.dna_create(N, T, R, L.make_opts(dtype=dtype))
        self.ctx = ctx
        try:
            L.dna_set_stream(ctx)
            L.dna_bind(ctx, V, W, H)
        except BaseException:
            L.dna_destroy(ctx)
            raise

    def __enter__(self):
        return self.ctx

    def __exit__(self, exc_type, exc, tb):
        pool = _pool()
        if exc_type is None and self.key not in pool:
            pool[self.key] = self.ctx
        else:
            L.dna_destroy(self.ctx)
        return False


class KLDiv(torch.autograd.Function):
    @staticmethod
    def forward(fctx, V, W, H):
        V, W, H = V.contiguous(), W.contiguous(), H.contiguous()
        with _Ctx(V, W, H) as ctx:
            kl = L.dna_kl(ctx)
        fctx.save_for_backward(V, W, H)
        return torch.tensor(kl, dtype=torch.float64, device=V.device)

    @staticmethod
    def backward(fctx, grad):
        V, W, H = fctx.saved_tensors
        need_v, need_w, need_h = fctx.needs_input_grad
        dV = torch.empty_like(V) if need_v else None
        dW = torch.empty_like(W) if need_w else None
        dH = torch.empty_like(H) if need_h else None
        with _Ctx(V, W, H) as ctx:
            L.dna_kl_backward(ctx, float(grad), dW, dH, dV)
            torch.cuda.current_stream().synchronize()
        return dV, dW, dH


class UnrolledDNAH(torch.autograd.Function):
    @staticmethod
    def forward(fctx, V, W, H0, K: int, every: int = 5):
        V, W = V.contiguous(), W.contiguous()
        H = H0.detach().clone().contiguous()
        T = V.shape[1]
        choices = torch.empty((K, T), dtype=torch.uint8, device=V.device)
        ckpts = []
        with _Ctx(V, W, H) as ctx:
            for k in range(K):
                if k % every == 0:
                    ckpts.append(H.clone())
                L.dna_step_H_fixed(ctx, choices[k])
            torch.cuda.current_stream().synchronize()
        fctx.K, fctx.every = K, every
        fctx.save_for_backward(V, W, choices, *ckpts)
        return H

    @staticmethod
    def backward(fctx, grad_HK):
        V, W, choices, *ckpts = fctx.saved_tensors
        K, every = fctx.K, fctx.every
        need_v, need_w = fctx.needs_input_grad[0], fctx.needs_input_grad[1]
        Hbar = grad_HK.contiguous().clone()
        Vbar = torch.zeros_like(V) if need_v else None
        Wbar = torch.zeros_like(W) if need_w else None
        Hrun = ckpts[0].clone()
        with _Ctx(V, W, Hrun) as ctx:
            for seg in reversed(range(len(ckpts))):
                k0, k1 = seg * every, min(seg * every + every, K)
                Hrun.copy_(ckpts[seg])
                states = [ckpts[seg]]
                for _ in range(k0, k1 - 1):           # recompute this segment's states
                    L.dna_step_H_fixed(ctx, None)
                    states.append(Hrun.clone())
                for k in reversed(range(k0, k1)):
                    out = torch.empty_like(Hbar)
                    L.dna_step_H_adjoint_w(ctx, states[k - k0], choices[k], Hbar, out, Vbar,
                                           Wbar)
                    Hbar = out
            torch.cuda.current_stream().synchronize()
        return Vbar, Wbar, Hbar, None, None
