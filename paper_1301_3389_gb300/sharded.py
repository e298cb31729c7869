"""Column-sharded DNA iterations over several GPUs (the dna_shard_* calls of the C ABI).

A problem V (N x T) is split into column blocks; each block has its own library context
(V[:, block], H[:, block] and a full copy of W) on its rank's GPU.  The H half-step
separates over columns (Section 2, eq. 5); the W half-step and the normalisations of
Algorithm 1 need sums over all columns.  ``ShardedDNA`` runs the library's phases on every
local block in lockstep and, at each exchange point, makes every block's buffer hold the
total over all blocks: the sum over the blocks of this process, then ``all_reduce``
(a callable summing a device tensor over processes in place, e.g.
``torch.distributed.all_reduce`` over NCCL; None when one process holds every block).
The arithmetic of the method runs in the library's kernels; this module only orders the
calls and moves the exchanged buffers.
"""
from __future__ import annotations

from . import _lib


class ShardedDNA:
    """One process's column blocks of a sharded problem.

    ``contexts``: library contexts, one per local block, bound to that block's V and H and
    to a full W (all blocks must hold the same W, e.g. after the same dna_normalize).
    ``R``, ``N``: rank and rows of the problem; ``dtype``: the contexts' element type as a
    torch dtype (float32 or float64).  ``lib`` defaults to this package's C binding."""

    def __init__(self, contexts, N: int, R: int, dtype, all_reduce=None, lib=None, device=None):
        import torch
        self.torch = torch
        self.lib = lib or _lib
        self.ctx = list(contexts)
        self.all_reduce = all_reduce
        dev = device or torch.device("cuda", torch.cuda.current_device())
        f64 = torch.float64
        n = len(self.ctx)
        self.rowsum = [torch.empty(N, dtype=f64, device=dev) for _ in range(n)]
        self.rsum = [torch.empty(R, dtype=f64, device=dev) for _ in range(n)]
        self.hsum = [torch.empty(R, dtype=f64, device=dev) for _ in range(n)]
        self.AB = [torch.empty(2 * R * N, dtype=dtype, device=dev) for _ in range(n)]
        self.cost = [torch.empty(2 * N, dtype=f64, device=dev) for _ in range(n)]
        for c, b in zip(self.ctx, self.rowsum):
            self.lib.dna_shard_rowsums(c, b)
        self._reduce(self.rowsum)
        for c, b in zip(self.ctx, self.rowsum):
            self.lib.dna_shard_set_rowsums(c, b)

    def _reduce(self, bufs):
        """Every buffer of ``bufs`` becomes the sum over all blocks of all processes."""
        total = bufs[0]
        if len(bufs) > 1:
            total = bufs[0].clone()
            for b in bufs[1:]:
                total += b
        if self.all_reduce is not None:
            self.all_reduce(total)
        for b in bufs:
            if b is not total:
                b.copy_(total)

    def step_H(self) -> None:
        """Algorithm 1 steps 4-16 on every block (one exchange: step 16's row sums)."""
        for c, b in zip(self.ctx, self.rsum):
            self.lib.dna_shard_H_begin(c, b)
        self._reduce(self.rsum)
        for c, b in zip(self.ctx, self.rsum):
            self.lib.dna_shard_H_end(c, b)

    def step_W(self) -> None:
        """Algorithm 1 steps 17-29 (exchanges: H's row sums, the eq. 7 / 14 sums, the costs)."""
        for c, b in zip(self.ctx, self.hsum):
            self.lib.dna_shard_W_begin(c, b)
        self._reduce(self.hsum)
        for c, h, ab in zip(self.ctx, self.hsum, self.AB):
            self.lib.dna_shard_W_pass1(c, h, ab)
        self._reduce(self.AB)
        for c, ab, d in zip(self.ctx, self.AB, self.cost):
            self.lib.dna_shard_W_pass2(c, ab, d)
        self._reduce(self.cost)
        for c, d in zip(self.ctx, self.cost):
            self.lib.dna_shard_W_end(c, d)

    def iterate(self, iters: int) -> None:
        for _ in range(iters):
            self.step_H()
            self.step_W()

    def kl(self) -> float:
        """d_KL (eq. 1) of the whole problem: the blocks' shares (dna_kl), summed."""
        t = self.torch.tensor([sum(self.lib.dna_kl(c) for c in self.ctx)], dtype=self.torch.float64,
                              device=self.rsum[0].device)
        if self.all_reduce is not None:
            self.all_reduce(t)
        return float(t.item())
