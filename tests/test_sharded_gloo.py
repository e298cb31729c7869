"""The column-sharded driver (paper_1301_3389_gb300.sharded.ShardedDNA) on two CPU ranks
over gloo, with a stand-in for the library's dna_shard_* calls built from the FP64
oracle's steps (the same split of Algorithm 1 at the same exchange points).  Two ranks of
one column block each, and one rank holding two blocks, must both give the oracle's
iteration on the whole problem (1e-12): this checks the order of the calls and of the
exchanges, and that every exchanged buffer is summed over all blocks of all ranks."""
import os
import socket

import numpy as np
import pytest

from oracle import dna as o


class _Block:
    """One column block: V[:, a:b], H[:, a:b] and a full W, as a library context holds."""

    def __init__(self, V, W, H, rho=0.0, lam=0.0):
        self.V, self.W, self.H = V.copy(), W.copy(), H.copy()
        self.rho, self.lam = rho, lam


class FakeShardLib:
    """dna_shard_* and dna_kl on _Block objects and CPU float64 tensors."""

    @staticmethod
    def dna_shard_rowsums(b, out):
        out.copy_(_t(b.V.sum(axis=1)))

    @staticmethod
    def dna_shard_set_rowsums(b, buf):
        b.rowsum = buf.numpy().copy()

    @staticmethod
    def dna_shard_H_begin(b, rsum):
        hs = o.h_half_step(b.V, b.W, b.H, lam=b.lam)
        b.Hnew = hs.X
        rsum.copy_(_t(hs.X.sum(axis=1)))

    @staticmethod
    def dna_shard_H_end(b, rsum):
        f = o.nonzero_sum(rsum.numpy() + b.rho)
        b.H = b.Hnew / f[:, None]
        b.W = b.W * f[None, :]

    @staticmethod
    def dna_shard_W_begin(b, hsum):
        hsum.copy_(_t(b.H.sum(axis=1)))

    @staticmethod
    def dna_shard_W_pass1(b, hsum, AB):
        b.c = o.nonzero_sum(hsum.numpy() + b.rho)
        Z = b.W @ b.H
        A = o.ratio(b.V, Z, 1) @ b.H.T                       # N x R raw sums over the block
        B = o.ratio(b.V, Z, 2) @ (b.H * b.H).T
        AB.copy_(_t(np.concatenate([A.T.ravel(), B.T.ravel()])))

    @staticmethod
    def dna_shard_W_pass2(b, AB, cost):
        N, R = b.W.shape
        ab = AB.numpy()
        A = ab[:R * N].reshape(R, N).T / b.c[None, :] - 1.0
        Bm = ab[R * N:].reshape(R, N).T / b.c[None, :]
        b.Wmu = b.W + A * b.W
        Wd = o.newton_candidate(b.W, A, Bm)
        den = Wd @ b.c
        sc = np.where(den > 0, b.rowsum / np.where(den > 0, den, 1.0), 1.0)
        b.Wdna = Wd * sc[:, None]
        cost.copy_(_t(np.concatenate([o.row_cost(b.V, b.Wmu @ b.H), o.row_cost(b.V, b.Wdna @ b.H)])))

    @staticmethod
    def dna_shard_W_end(b, cost):
        N = b.W.shape[0]
        d = cost.numpy()
        dm = d[:N] + b.rho * b.Wmu.sum(axis=1)
        dd = d[N:] + b.rho * b.Wdna.sum(axis=1)
        W = np.where((dd < dm)[:, None], b.Wdna, b.Wmu)
        f = o.nonzero_sum(W.sum(axis=0) + b.lam)
        b.W = W / f[None, :]
        b.H = b.H * f[:, None]

    @staticmethod
    def dna_kl(b):
        return o.kl_divergence(b.V, b.W @ b.H)


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))


def _problem():
    g = np.random.default_rng(5)
    N, T, R = 14, 23, 3
    V = g.poisson(2.0, (N, T)).astype(np.float64)
    V[:, 0] += 1
    W = g.uniform(0.1, 1.0, (N, R))
    H = g.uniform(0.1, 1.0, (R, T))
    return V, *o.normalize_w_columns(W, H, 0.2)


def _reference(iters, rho, lam):
    V, W, H = _problem()
    for _ in range(iters):
        W, H, _, _ = o.dna_iteration(V, W, H, rho=rho, lam=lam)
    return W, H, o.kl_divergence(V, W @ H)


def _blocks_for(rank, world, per_rank, rho, lam):
    V, W, H = _problem()
    cuts = np.linspace(0, V.shape[1], world * per_rank + 1).astype(int)
    ids = range(rank * per_rank, (rank + 1) * per_rank)
    return [_Block(V[:, cuts[i]:cuts[i + 1]], W, H[:, cuts[i]:cuts[i + 1]], rho, lam) for i in ids]


def _rank(rank, world, port, out_dir, per_rank, rho, lam):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1301_3389_gb300.sharded import ShardedDNA
    blocks = _blocks_for(rank, world, per_rank, rho, lam)
    sh = ShardedDNA(blocks, blocks[0].W.shape[0], blocks[0].W.shape[1], torch.float64,
                    all_reduce=dist.all_reduce, lib=FakeShardLib, device=torch.device("cpu"))
    sh.iterate(2)
    kl = sh.kl()
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            {"W": [b.W for b in blocks], "H": [b.H for b in blocks], "kl": kl}, allow_pickle=True)
    dist.destroy_process_group()


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("per_rank", [1, 2])
def test_sharded_driver_two_ranks(tmp_path, per_rank):
    import torch.multiprocessing as mp
    rho, lam = 0.1, 0.2
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path), per_rank, rho, lam), nprocs=2, join=True)
    W, H, kl = _reference(2, rho, lam)
    Hs, Ws, kls = [], [], []
    for r in range(2):
        d = np.load(tmp_path / f"r{r}.npy", allow_pickle=True).item()
        Hs += d["H"]
        Ws += d["W"]
        kls.append(d["kl"])
    for Wb in Ws:
        np.testing.assert_allclose(Wb, W, rtol=1e-12)
    np.testing.assert_allclose(np.concatenate(Hs, axis=1), H, rtol=1e-12)
    assert kls[0] == kls[1] and abs(kls[0] - kl) <= 1e-12 * kl
