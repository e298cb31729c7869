"""Multi-rank paths on CPU ranks (torch.distributed, gloo, world size 2).

* The bench's N > 1 path: every rank times its own problem; the job's time is the slowest
  rank's (all-reduce MAX) and its rate counts every rank's iterations.
* The column-sharded iteration a multi-GPU run of one problem would use: V and H split
  by columns across ranks, W replicated.  The H half-step needs no exchange (columns are
  independent, Section 2); the step-16 row sums of H, the W half-step's A and B sums over
  t (eq. 7, 14), the row sums of V (eq. 10) and the per-row costs (steps 22, 27) are
  all-reduced.  One iteration on two ranks must equal the FP64 oracle's on the whole
  problem to rounding (1e-12).
"""
import os
import socket

import numpy as np
import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(fn, world, *args):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(fn, args=(world, port) + args, nprocs=world, join=True)


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _aggregation_rank(rank, world, port, out_dir):
    import torch
    import bench
    dist = _init(rank, world, port)
    ms = 10.0 + 5.0 * rank                       # rank 1 is the slower one
    ms_max = bench.max_over_ranks(torch, dist, ms, torch.device("cpu"))
    rate = bench.job_rate(world, 7, ms_max)
    np.save(os.path.join(out_dir, f"agg{rank}.npy"), np.array([ms_max, rate]))
    dist.destroy_process_group()


def test_bench_rank_aggregation(tmp_path):
    _run(_aggregation_rank, 2, str(tmp_path))
    for r in range(2):
        ms_max, rate = np.load(tmp_path / f"agg{r}.npy")
        assert ms_max == 15.0
        assert rate == pytest.approx(2 * 7 / 0.015)


def _allreduce(dist, x):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def _sharded_rank(rank, world, port, out_dir):
    import workloads
    from oracle import dna as o
    dist = _init(rank, world, port)
    p = workloads.custom(48, 90, 5, seed=77)
    V, W, H = o.f64(p.V), o.f64(p.W), o.f64(p.H)
    cols = np.array_split(np.arange(V.shape[1]), world)[rank]
    Vg, Hg = V[:, cols], H[:, cols]
    W, _ = o.normalize_w_columns(W, H)           # step 1 (W replicated, column sums local)
    Hg = H[:, cols] * o.nonzero_sum(o.f64(p.W).sum(axis=0))[:, None]
    # H half-step on the local columns: no exchange
    hs = o.h_half_step(Vg, W, Hg)
    # step 16: row sums of H over all columns
    srow = o.nonzero_sum(_allreduce(dist, hs.X.sum(axis=1)))
    W, Hg = W * srow[None, :], hs.X / srow[:, None]
    # W half-step: sums over t are all-reduced
    c = o.nonzero_sum(_allreduce(dist, Hg.sum(axis=1)))          # (H 1)_r
    Z = W @ Hg
    A = _allreduce(dist, o.ratio(Vg, Z, 1) @ Hg.T) / c[None, :] - 1.0
    B = _allreduce(dist, o.ratio(Vg, Z, 2) @ (Hg * Hg).T) / c[None, :]
    W_mu = W + A * W
    W_dna = o.newton_candidate(W, A, B)
    s = _allreduce(dist, Vg.sum(axis=1))                            # V 1
    den = W_dna @ c
    W_dna = W_dna * np.where(den > 0, s / np.where(den > 0, den, 1.0), 1.0)[:, None]
    d_mu = _allreduce(dist, o.row_cost(Vg, W_mu @ Hg))
    d_dna = _allreduce(dist, o.row_cost(Vg, W_dna @ Hg))
    Wn = np.where((d_dna < d_mu)[:, None], W_dna, W_mu)
    W, Hg = o.normalize_w_columns(Wn, Hg)        # step 29 (W replicated)
    np.save(os.path.join(out_dir, f"W{rank}.npy"), W)
    np.save(os.path.join(out_dir, f"H{rank}.npy"), Hg)
    dist.destroy_process_group()


def test_column_sharded_iteration_matches_oracle(tmp_path):
    import workloads
    from oracle import dna as o
    world = 2
    _run(_sharded_rank, world, str(tmp_path))
    p = workloads.custom(48, 90, 5, seed=77)
    W, H = o.normalize_w_columns(p.W, p.H)
    W, H, _, _ = o.dna_iteration(p.V, W, H)
    cols = np.array_split(np.arange(p.V.shape[1]), world)
    for r in range(world):
        np.testing.assert_allclose(np.load(tmp_path / f"W{r}.npy"), W, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(np.load(tmp_path / f"H{r}.npy"), H[:, cols[r]], rtol=1e-12,
                                   atol=1e-300)
