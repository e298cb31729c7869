"""dna_kl_noalloc: the d_KL entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (their device memory belongs to another framework's
pool allocator, or their latency budget cannot absorb cudaMalloc or the device
synchronisation of cudaFree).  dna_kl_noalloc keeps its scratch in a static device array
inside the library.  This test calls it through the C ABI and checks it against the
context-based dna_kl and against the FP64 oracle on the same inputs, on calls in a row
(a later call must not see an earlier call's leftovers), over every rank class of its
kernel (R up to 512), a padded V (ldv > T) and a size whose sum over n is split across
CTAs.  It is collected last so a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import dna as o

REL = 1e-6          # against dna_kl: the same float32 products, the same float64 sums
REL_ORACLE = 1e-4   # against the FP64 oracle: the FP32 form's d_KL tolerance

# (N, T, R, pad): rank classes 32 (R=24), 64 (R=48), 128 (R=129 and 512: several
# 128-row pieces); pad > 0 gives V a leading dimension T + pad; N=2048 T=128 makes the
# kernel split the sum over n across CTAs (few column blocks for 152 SMs)
CASES = [(300, 700, 24, 0), (67, 131, 129, 0), (90, 200, 48, 0), (40, 70, 512, 0),
         (120, 333, 16, 7), (2048, 128, 20, 0)]


def _tensors(torch, p, pad):
    N, T = p.V.shape
    Vfull = torch.zeros((N, T + pad), dtype=torch.float32, device="cuda")
    Vfull[:, :T] = torch.from_numpy(p.V).cuda()
    V = Vfull[:, :T]
    return V, torch.from_numpy(p.W).cuda(), torch.from_numpy(p.H).cuda()


def _kl_context(dna, V, W, H):
    N, T = V.shape
    ctx = dna.dna_create(N, T, W.shape[1], dna.make_opts(dtype=dna.DNA_F32))
    try:
        dna.dna_set_stream(ctx)
        dna.dna_bind(ctx, V, W, H)
        return dna.dna_kl(ctx)
    finally:
        dna.dna_destroy(ctx)


def _kl_noalloc(dna, torch, V, W, H, out):
    """Straight through the C ABI (ctypes), no Python wrapper."""
    N, T = V.shape
    code = dna.LIB.dna_kl_noalloc(
        ctypes.c_void_p(V.data_ptr()), V.stride(0), ctypes.c_void_p(W.data_ptr()),
        ctypes.c_void_p(H.data_ptr()), N, T, W.shape[1], ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == dna.DNA_OK, dna.dna_strerror(code)
    torch.cuda.synchronize()
    return float(out.item())


@pytest.mark.gpu
def test_noalloc_matches_dna_kl_and_oracle():
    import torch

    import paper_1301_3389_gb300 as dna
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    last = None
    for i, (N, T, R, pad) in enumerate(CASES):      # calls in a row, sizes and data differ
        p = workloads.custom(N, T, R, seed=11 + i)
        V, W, H = _tensors(torch, p, pad)
        ref = _kl_context(dna, V, W, H)
        got = _kl_noalloc(dna, torch, V, W, H, out)
        assert abs(got - ref) <= REL * abs(ref), (N, T, R, pad, got, ref)
        kl64 = o.kl_divergence(p.V, p.W.astype(np.float64) @ p.H.astype(np.float64))
        assert abs(got - kl64) <= REL_ORACLE * abs(kl64), (N, T, R, pad, got, kl64)
        last = (V, W, H, got)
    # the same inputs again right after: identical answer
    V, W, H, got = last
    assert _kl_noalloc(dna, torch, V, W, H, out) == got
    # and once through the Python wrapper (argument checks, then the same C call)
    out2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    dna.dna_kl_noalloc(V, W, H, out2)
    torch.cuda.synchronize()
    assert float(out2.item()) == got


@pytest.mark.gpu
def test_noalloc_limits_and_infinite_cost():
    import torch

    import paper_1301_3389_gb300 as dna
    T = dna.DNA_KL_NOALLOC_MAX_PARTIALS + 1
    code = dna.LIB.dna_kl_noalloc(ctypes.c_void_p(16), T, ctypes.c_void_p(16),
                                  ctypes.c_void_p(16), 4, T, 4, ctypes.c_void_p(16), None)
    assert code == dna.DNA_ERR_LIMIT            # rejected on the host, nothing queued
    p = workloads.custom(40, 50, 4, seed=3)
    V = torch.from_numpy(p.V).cuda()
    W = torch.zeros((40, 4), dtype=torch.float32, device="cuda")   # z = 0 where v > 0
    H = torch.from_numpy(p.H).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert np.isinf(_kl_noalloc(dna, torch, V, W, H, out))
    # and a finite call right after is not affected by the flag of the previous one
    W = torch.from_numpy(p.W).cuda()
    ref = _kl_context(dna, V, W, H)
    assert abs(_kl_noalloc(dna, torch, V, W, H, out) - ref) <= REL * abs(ref)
    # the wrapper rejects layouts the C call cannot take, before any work is queued
    with pytest.raises(dna.DNAError):
        dna.dna_kl_noalloc(V, W.t().contiguous().t(), H, out)       # W not row-major
    with pytest.raises(dna.DNAError):
        dna.dna_kl_noalloc(V, W, H.double(), out)                   # H not float32
