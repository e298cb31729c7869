"""The trajectory tolerance of the split FP32 form for R > 300 (SPLIT_LARGE_R_TOL), checked
against its derivation on the CPU.

The split form carries every tensor-core operand as x_hi + x_lo with x_hi = bf16(x) and
x_lo = bf16(x - x_hi): about 17 significant bits.  This test runs the oracle's DNA
iterations twice from the same state, exactly and with that representation applied to
every operand of the O(NRT) products (W and H in Z = W H and in A = W^t Q,
B = (W o W)^t Qbar; q and qbar), everything else in FP64 with the exact run's selections
replayed, and measures how far the W, H trajectories part.  The GPU tolerance is that
separation plus the CUDA-core FP32 form's measured rounding, times 2; this test checks
that the representation alone stays within half of it.
"""
import numpy as np

import workloads
from gpu_helpers import SPLIT_LARGE_R_TOL
from oracle import dna as o


def bf16(x):
    """Round-to-nearest-even to bfloat16 (the top 16 bits of a float32)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def split(x):
    x32 = np.asarray(x, dtype=np.float32)
    hi = bf16(x32)
    return hi.astype(np.float64) + bf16(x32 - hi).astype(np.float64)


def h_step_split(V, W, H, choice):
    """The H half-step with split operands in the O(NRT) products (selection given)."""
    c = W.sum(axis=0)
    Ws, Hs = split(W), split(H)
    Z = Ws @ Hs
    Q, Qb = split(o.ratio(V, Z, 1)), split(o.ratio(V, Z, 2))
    A = (Ws.T @ Q) / c[:, None] - 1.0
    B = (split(Ws * Ws).T @ Qb) / c[:, None]
    H_mu = H + A * H
    H_dna = o.newton_candidate(H, A, B, o.EPS, o.ALPHA)
    H_dna = H_dna * (V.sum(axis=0) / (c @ H_dna))[None, :]
    return np.where(choice[None, :], H_dna, H_mu)


def separation(N, T, R, iters):
    p = workloads.custom(N, T, R, seed=N + 3 * T + 7 * R)
    V = p.V.astype(np.float64)
    We, He = o.normalize_w_columns(p.W, p.H)
    Ws, Hs = We.copy(), He.copy()
    out = []
    for _ in range(iters):
        hs = o.h_half_step(V, We, He)
        We, He = o.normalize_h_rows(We, hs.X)
        Ws, Hs = o.normalize_h_rows(Ws, h_step_split(V, Ws, Hs, hs.choice))
        ws = o.w_half_step(V, We, He)
        We, He = o.normalize_w_columns(ws.X, He)
        Ws, Hs = o.normalize_w_columns(h_step_split(V.T, Hs.T, Ws.T, ws.choice).T, Hs)
        out.append(max(np.linalg.norm(Ws - We) / np.linalg.norm(We),
                       np.linalg.norm(Hs - He) / np.linalg.norm(He)))
    return out


def test_split_rounding():
    x = np.array([1.0, 1.0 + 2.0 ** -9, 3.14159265, -2.5e-7, 1e30], dtype=np.float32)
    assert np.all(np.abs(split(x) - x.astype(np.float64)) <= 2.0 ** -16 * np.abs(x))
    # bf16 spacing at 1 is 2^-7: 1 + 2^-8 is a tie and goes to the even neighbour 1;
    # 1 + 3 * 2^-8 is a tie between 1 + 2^-7 and 1 + 2^-6 and goes to 1 + 2^-6
    t = bf16(np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7], dtype=np.float32))
    assert t.tolist() == [1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7]


def test_representation_within_half_the_tolerance():
    sep = separation(520, 640, 512, 2)
    assert 0.0 < sep[-1] < 0.5 * SPLIT_LARGE_R_TOL, sep
