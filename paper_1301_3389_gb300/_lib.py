"""ctypes binding of libdna.so (include/dna.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Device buffers are torch
CUDA tensors (their data pointers are passed); the stream is torch's current stream
unless one is given.  There is no fallback: if libdna.so is missing or fails to load,
importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdna.so")

DNA_OK = 0
DNA_ERR_ARG = -1
DNA_ERR_CUDA = -2
DNA_ERR_NONFINITE = -3
DNA_ERR_TIMEOUT = -4
DNA_ERR_UNSUPPORTED = -5
DNA_ERR_ALLOC = -6
DNA_ERR_LIMIT = -7
DNA_KL_NOALLOC_MAX_PARTIALS = 1 << 20

DNA_F64, DNA_F32, DNA_BF16 = 0, 1, 2
PHASES = ("pass1", "candidates", "pass2", "select", "sums", "kl", "prepare", "operands")
DNA_ENGINE_AUTO, DNA_ENGINE_SIMT, DNA_ENGINE_TENSOR = 0, 1, 2


class dna_opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("alpha", ctypes.c_double),
                ("rho", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("dtype", ctypes.c_int32), ("engine", ctypes.c_int32)]


class DNAError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {dna_strerror(code)} ({code})")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdna.so not built ({LIB_PATH}); run "
                          "`python paper_1301_3389_gb300/build.py` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "dna_default_opts": (None, [ctypes.POINTER(dna_opts)]),
        "dna_create": (I, [I64, I64, I64, ctypes.POINTER(dna_opts), ctypes.POINTER(P)]),
        "dna_bind": (I, [P, P, I64, P, P]),
        "dna_set_stream": (I, [P, P]),
        "dna_normalize": (I, [P, I]),
        "dna_step_H": (I, [P]),
        "dna_step_W": (I, [P]),
        "dna_iterate": (I, [P, I]),
        "dna_use_graph": (I, [P, I]),
        "mu_step": (I, [P, I]),
        "mu_iterate": (I, [P, I]),
        "dna_create_sparse": (I, [I64, I64, I64, I64, ctypes.POINTER(dna_opts), ctypes.POINTER(P)]),
        "dna_bind_csr": (I, [P, P, P, P, P, P]),
        "dna_shard_rowsums": (I, [P, P]),
        "dna_check_wait_timeout": (I, [I64]),
        "dna_set_selection": (I, [P, I]),
        "dna_shard_set_rowsums": (I, [P, P]),
        "dna_shard_H_begin": (I, [P, P]),
        "dna_shard_H_end": (I, [P, P]),
        "dna_shard_W_begin": (I, [P, P]),
        "dna_shard_W_pass1": (I, [P, P, P]),
        "dna_shard_W_pass2": (I, [P, P, P]),
        "dna_shard_W_end": (I, [P, P]),
        "dna_kl": (I, [P, ctypes.POINTER(D)]),
        "dna_get_choice": (I, [P, I, P, I64]),
        "dna_get_costs": (I, [P, I, P, P, I64]),
        "dna_get_status": (I, [P]),
        "dna_run_host": (I, [P, P, P, P, I, ctypes.POINTER(D)]),
        "dna_profile": (I, [P, I]),
        "dna_profile_phases": (I, [P, ctypes.c_uint]),
        "dna_phase_times": (I, [P, P, P, I]),
        "dna_kl_noalloc": (I, [P, I64, P, P, I64, I64, I64, P, P]),
        "dna_kl_backward": (I, [P, D, P, P, P]),
        "dna_step_H_fixed": (I, [P, P]),
        "dna_step_H_adjoint": (I, [P, P, P, P, P, P]),
        "dna_step_H_adjoint_w": (I, [P, P, P, P, P, P, P]),
        "dna_group_create": (I, [I, P, P, P, ctypes.POINTER(dna_opts), ctypes.POINTER(P)]),
        "dna_group_bind": (I, [P, P, P, P, P]),
        "dna_group_set_stream": (I, [P, P]),
        "dna_group_normalize": (I, [P, I]),
        "dna_group_step_H": (I, [P]),
        "dna_group_step_W": (I, [P]),
        "dna_group_iterate": (I, [P, I]),
        "dna_group_use_graph": (I, [P, I]),
        "dna_group_autotune": (I, [P, I, P]),
        "dna_group_tile_config": (I, [P, P, P]),
        "dna_group_kl": (I, [P, P]),
        "dna_group_get_status": (I, [P]),
        "dna_group_get_choice": (I, [P, I, I, P, I64]),
        "dna_group_launches_per_iteration": (I64, [P]),
        "dna_group_destroy": (None, [P]),
        "dna_destroy": (None, [P]),
        "dna_strerror": (ctypes.c_char_p, [I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()


def _check(code: int, where: str) -> None:
    if code != DNA_OK:
        raise DNAError(code, where)


def _ptr(t) -> int:
    """Device (or host) address of a torch tensor or a NumPy array."""
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def dna_strerror(code: int) -> str:
    return LIB.dna_strerror(int(code)).decode()


def dna_default_opts() -> dna_opts:
    o = dna_opts()
    LIB.dna_default_opts(ctypes.byref(o))
    return o


def make_opts(eps=None, alpha=None, rho=None, lam=None, dtype=None, engine=None) -> dna_opts:
    o = dna_default_opts()
    if eps is not None:
        o.eps = eps
    if alpha is not None:
        o.alpha = alpha
    if rho is not None:
        o.rho = rho
    if lam is not None:
        o.lambda_ = lam
    if dtype is not None:
        o.dtype = dtype
    if engine is not None:
        o.engine = engine
    return o


def dna_create(N: int, T: int, R: int, opts: dna_opts | None = None) -> int:
    h = ctypes.c_void_p()
    _check(LIB.dna_create(N, T, R, ctypes.byref(opts) if opts is not None else None,
                          ctypes.byref(h)), "dna_create")
    return h.value


def dna_create_sparse(N: int, T: int, R: int, nnz: int, opts: dna_opts | None = None) -> int:
    h = ctypes.c_void_p()
    _check(LIB.dna_create_sparse(N, T, R, nnz, ctypes.byref(opts) if opts is not None else None,
                                 ctypes.byref(h)), "dna_create_sparse")
    return h.value


def dna_bind_csr(ctx: int, row_ptr, col_idx, vals, W, H) -> None:
    """row_ptr int64 (N + 1), col_idx int32 (nnz), vals (nnz), W, H: device tensors."""
    _check(LIB.dna_bind_csr(ctx, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(W), _ptr(H)),
           "dna_bind_csr")


def dna_bind(ctx: int, V, W, H, ldv: int | None = None) -> None:
    if ldv is None:
        ldv = V.stride(0) if hasattr(V, "stride") else V.shape[1]
    _check(LIB.dna_bind(ctx, _ptr(V), ldv, _ptr(W), _ptr(H)), "dna_bind")


def dna_set_stream(ctx: int, stream=None) -> None:
    _check(LIB.dna_set_stream(ctx, _stream(stream)), "dna_set_stream")


def dna_normalize(ctx: int, which: int) -> None:
    _check(LIB.dna_normalize(ctx, which), "dna_normalize")


def dna_step_H(ctx: int) -> None:
    _check(LIB.dna_step_H(ctx), "dna_step_H")


def dna_step_W(ctx: int) -> None:
    _check(LIB.dna_step_W(ctx), "dna_step_W")


def dna_iterate(ctx: int, iters: int) -> None:
    _check(LIB.dna_iterate(ctx, iters), "dna_iterate")


def dna_use_graph(ctx: int, enable: bool) -> None:
    _check(LIB.dna_use_graph(ctx, int(bool(enable))), "dna_use_graph")


def mu_step(ctx: int, which: int) -> None:
    _check(LIB.mu_step(ctx, which), "mu_step")


def mu_iterate(ctx: int, iters: int) -> None:
    _check(LIB.mu_iterate(ctx, iters), "mu_iterate")


def dna_kl(ctx: int) -> float:
    out = ctypes.c_double()
    _check(LIB.dna_kl(ctx, ctypes.byref(out)), "dna_kl")
    return out.value


def dna_kl_backward(ctx: int, scale: float, dW=None, dH=None, dV=None) -> None:
    _check(LIB.dna_kl_backward(ctx, float(scale), _ptr(dW) if dW is not None else None,
                               _ptr(dH) if dH is not None else None,
                               _ptr(dV) if dV is not None else None), "dna_kl_backward")


def dna_step_H_fixed(ctx: int, choice_out=None) -> None:
    _check(LIB.dna_step_H_fixed(ctx, _ptr(choice_out) if choice_out is not None else None),
           "dna_step_H_fixed")


def dna_step_H_adjoint(ctx: int, Hk, choice, Hbar_next, Hbar_out, Vbar) -> None:
    _check(LIB.dna_step_H_adjoint(ctx, _ptr(Hk), _ptr(choice), _ptr(Hbar_next), _ptr(Hbar_out),
                                  _ptr(Vbar)), "dna_step_H_adjoint")


def dna_step_H_adjoint_w(ctx: int, Hk, choice, Hbar_next, Hbar_out, Vbar=None,
                         Wbar=None) -> None:
    _check(LIB.dna_step_H_adjoint_w(ctx, _ptr(Hk), _ptr(choice), _ptr(Hbar_next),
                                    _ptr(Hbar_out), _ptr(Vbar) if Vbar is not None else None,
                                    _ptr(Wbar) if Wbar is not None else None),
           "dna_step_H_adjoint_w")


def dna_get_choice(ctx: int, which: int, n: int):
    import numpy as np
    out = np.zeros(n, dtype=np.uint8)
    _check(LIB.dna_get_choice(ctx, which, out.ctypes.data, n), "dna_get_choice")
    return out.astype(bool)


def dna_get_costs(ctx: int, which: int, n: int):
    import numpy as np
    dm = np.zeros(n, dtype=np.float64)
    dd = np.zeros(n, dtype=np.float64)
    _check(LIB.dna_get_costs(ctx, which, dm.ctypes.data, dd.ctypes.data, n), "dna_get_costs")
    return dm, dd


def dna_get_status(ctx: int) -> int:
    return LIB.dna_get_status(ctx)


def dna_run_host(ctx: int, V, W, H, iters: int) -> float:
    kl = ctypes.c_double()
    _check(LIB.dna_run_host(ctx, _ptr(V), _ptr(W), _ptr(H), iters, ctypes.byref(kl)),
           "dna_run_host")
    return kl.value


def dna_profile(ctx: int, enable: bool = True) -> None:
    _check(LIB.dna_profile(ctx, 1 if enable else 0), "dna_profile")


def dna_profile_phases(ctx: int, phases) -> None:
    """Record event pairs around the named phases only (an empty list stops recording)."""
    mask = 0
    for p in phases:
        mask |= 1 << PHASES.index(p)
    _check(LIB.dna_profile_phases(ctx, mask), "dna_profile_phases")


def dna_phase_times(ctx: int) -> dict:
    """{phase: (milliseconds, launches)} since the previous call."""
    import numpy as np
    ms = np.zeros(len(PHASES), dtype=np.float64)
    nl = np.zeros(len(PHASES), dtype=np.int64)
    _check(LIB.dna_phase_times(ctx, ms.ctypes.data, nl.ctypes.data, len(PHASES)),
           "dna_phase_times")
    return {p: (float(ms[i]), int(nl[i])) for i, p in enumerate(PHASES)}


def dna_kl_noalloc(V, W, H, out, stream=None, ldv: int | None = None) -> None:
    """d_KL(V, W H) into the one-element float64 device tensor ``out`` (asynchronous).

    Allocates nothing (static scratch inside the library); calls that overlap on the GPU
    race, so keep them ordered on one stream."""
    import torch
    N, T = V.shape
    R = W.shape[1]
    for name, t in (("V", V), ("W", W), ("H", H)):
        if t.dtype != torch.float32 or not t.is_cuda:
            raise DNAError(DNA_ERR_ARG, f"dna_kl_noalloc: {name} must be a float32 CUDA tensor")
    if W.shape[0] != N or tuple(H.shape) != (R, T):
        raise DNAError(DNA_ERR_ARG, "dna_kl_noalloc: shapes must be V (N, T), W (N, R), H (R, T)")
    if not (W.is_contiguous() and H.is_contiguous()) or V.stride(1) != 1:
        raise DNAError(DNA_ERR_ARG, "dna_kl_noalloc: W, H contiguous and V rows contiguous")
    if out.dtype != torch.float64 or not out.is_cuda or out.numel() < 1:
        raise DNAError(DNA_ERR_ARG, "dna_kl_noalloc: out must be a float64 CUDA tensor")
    if ldv is None:
        ldv = V.stride(0)
    _check(LIB.dna_kl_noalloc(_ptr(V), ldv, _ptr(W), _ptr(H), N, T, R, _ptr(out),
                              _stream(stream)), "dna_kl_noalloc")


def _i64_array(vals):
    import numpy as np
    return np.ascontiguousarray(np.asarray(vals, dtype=np.int64))


def _ptr_array(tensors):
    import numpy as np
    return np.ascontiguousarray(np.asarray([_ptr(t) for t in tensors], dtype=np.uint64))


def dna_group_create(N, T, R, opts: dna_opts | None = None) -> int:
    n, t, r = _i64_array(N), _i64_array(T), _i64_array(R)
    h = ctypes.c_void_p()
    _check(LIB.dna_group_create(len(n), n.ctypes.data, t.ctypes.data, r.ctypes.data,
                                ctypes.byref(opts) if opts is not None else None,
                                ctypes.byref(h)), "dna_group_create")
    return h.value


def dna_group_bind(g: int, V, W, H, ldv=None) -> None:
    pv, pw, ph = _ptr_array(V), _ptr_array(W), _ptr_array(H)
    ld = _i64_array(ldv if ldv is not None else [v.stride(0) for v in V])
    _check(LIB.dna_group_bind(g, pv.ctypes.data, ld.ctypes.data, pw.ctypes.data, ph.ctypes.data),
           "dna_group_bind")


def dna_group_set_stream(g: int, stream=None) -> None:
    _check(LIB.dna_group_set_stream(g, _stream(stream)), "dna_group_set_stream")


def dna_group_normalize(g: int, which: int) -> None:
    _check(LIB.dna_group_normalize(g, which), "dna_group_normalize")


def dna_group_step_H(g: int) -> None:
    _check(LIB.dna_group_step_H(g), "dna_group_step_H")


def dna_group_step_W(g: int) -> None:
    _check(LIB.dna_group_step_W(g), "dna_group_step_W")


def dna_group_iterate(g: int, iters: int) -> None:
    _check(LIB.dna_group_iterate(g, iters), "dna_group_iterate")


def dna_group_use_graph(g: int, enable: bool = True) -> None:
    _check(LIB.dna_group_use_graph(g, 1 if enable else 0), "dna_group_use_graph")


def dna_group_autotune(g: int, reps: int = 2) -> int:
    rows = ctypes.c_int64()
    _check(LIB.dna_group_autotune(g, reps, ctypes.byref(rows)), "dna_group_autotune")
    return rows.value


def dna_group_tile_config(g: int):
    """(rows of s per split, pass-2 units per CTA (0 in the FP32 form))."""
    rows, units = ctypes.c_int64(), ctypes.c_int64()
    _check(LIB.dna_group_tile_config(g, ctypes.byref(rows), ctypes.byref(units)),
           "dna_group_tile_config")
    return rows.value, units.value


def dna_group_kl(g: int, count: int):
    import numpy as np
    out = np.zeros(count, dtype=np.float64)
    _check(LIB.dna_group_kl(g, out.ctypes.data), "dna_group_kl")
    return out


def dna_group_get_status(g: int) -> int:
    return LIB.dna_group_get_status(g)


def dna_group_get_choice(g: int, q: int, which: int, n: int):
    import numpy as np
    out = np.zeros(n, dtype=np.uint8)
    _check(LIB.dna_group_get_choice(g, q, which, out.ctypes.data, n), "dna_group_get_choice")
    return out.astype(bool)


def dna_group_launches_per_iteration(g: int) -> int:
    return LIB.dna_group_launches_per_iteration(g)


def dna_group_destroy(g: int) -> None:
    LIB.dna_group_destroy(g)


def dna_destroy(ctx: int) -> None:
    LIB.dna_destroy(ctx)


def _shard_call(name):
    def f(ctx: int, *bufs) -> None:
        _check(getattr(LIB, name)(ctx, *[_ptr(b) for b in bufs]), name)
    f.__name__ = name
    return f


dna_shard_rowsums = _shard_call("dna_shard_rowsums")
dna_shard_set_rowsums = _shard_call("dna_shard_set_rowsums")
dna_shard_H_begin = _shard_call("dna_shard_H_begin")
dna_shard_H_end = _shard_call("dna_shard_H_end")
dna_shard_W_begin = _shard_call("dna_shard_W_begin")
dna_shard_W_pass1 = _shard_call("dna_shard_W_pass1")
dna_shard_W_pass2 = _shard_call("dna_shard_W_pass2")
dna_shard_W_end = _shard_call("dna_shard_W_end")


DNA_SELECT_PAPER = 0
DNA_SELECT_DESCENT = 1


def dna_set_selection(ctx: int, mode: int) -> None:
    _check(LIB.dna_set_selection(ctx, mode), "dna_set_selection")
