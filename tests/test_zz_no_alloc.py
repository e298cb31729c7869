"""dna_kl_noalloc: the d_KL entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (their device memory belongs to another framework's
pool allocator, or their latency budget cannot absorb cudaMalloc or the device
synchronisation of cudaFree).  dna_kl_noalloc keeps its scratch in a static device array
inside the library.  This test calls it through the C ABI and checks it against the
context-based dna_kl on the same inputs, on two calls in a row (the second call must not
see the first call's leftovers).  It is collected last so a failure here comes after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

import workloads

REL = 1e-6   # stricter than the 1e-4 relative d_KL tolerance of the parity tests


def _kl_context(dna, torch, V, W, H):
    N, T = V.shape
    ctx = dna.dna_create(N, T, W.shape[1], dna.make_opts(dtype=dna.DNA_F32))
    try:
        dna.dna_set_stream(ctx)
        dna.dna_bind(ctx, V, W, H)
        return dna.dna_kl(ctx)
    finally:
        dna.dna_destroy(ctx)


def _kl_noalloc(dna, torch, V, W, H, out):
    N, T = V.shape
    code = dna.LIB.dna_kl_noalloc(
        ctypes.c_void_p(V.data_ptr()), V.stride(0), ctypes.c_void_p(W.data_ptr()),
        ctypes.c_void_p(H.data_ptr()), N, T, W.shape[1], ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == dna.DNA_OK, dna.dna_strerror(code)
    torch.cuda.synchronize()
    return float(out.item())


@pytest.mark.gpu
def test_noalloc_matches_dna_kl_twice():
    import torch

    import paper_1301_3389_gb300 as dna
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cases = [workloads.custom(300, 700, 24, seed=11), workloads.custom(67, 131, 129, seed=12)]
    for p in cases:                       # two calls in a row, different sizes and data
        V = torch.from_numpy(p.V).cuda()
        W = torch.from_numpy(p.W).cuda()
        H = torch.from_numpy(p.H).cuda()
        ref = _kl_context(dna, torch, V, W, H)
        got = _kl_noalloc(dna, torch, V, W, H, out)
        assert abs(got - ref) <= REL * abs(ref), (got, ref)
    # the same inputs again right after: identical answer
    again = _kl_noalloc(dna, torch, V, W, H, out)
    assert again == got


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
    ref = _kl_context(dna, torch, V, W, H)
    assert abs(_kl_noalloc(dna, torch, V, W, H, out) - ref) <= REL * abs(ref)
