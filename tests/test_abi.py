"""The C-ABI library builds, loads and exports every entry point of include/dna.h.

No compute calls here: only host-side validation paths that return before any CUDA work.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*"
                             r"([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, flags=re.M):
            if m.group(1) not in ("if", "return", "sizeof"):
                names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = declared_functions()
    for n in ("dna_create", "dna_step_H", "dna_step_W", "mu_step", "dna_kl", "dna_bind",
              "dna_destroy", "dna_run_host"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_validation():
    import paper_1301_3389_gb300 as dna
    bad = [(0, 4, 4), (4, 0, 4), (4, 4, 0), (4, 4, 513), (-3, 4, 4)]
    for N, T, R in bad:
        with pytest.raises(dna.DNAError) as e:
            dna.dna_create(N, T, R)
        assert e.value.code == dna.DNA_ERR_ARG
    with pytest.raises(dna.DNAError) as e:
        dna.dna_create(8, 8, 2, dna.make_opts(eps=0.0))
    assert e.value.code == dna.DNA_ERR_ARG
    with pytest.raises(dna.DNAError) as e:
        dna.dna_create(8, 8, 2, dna.make_opts(dtype=7))
    assert e.value.code == dna.DNA_ERR_ARG
    # NULL context is rejected before any CUDA work
    for f in (dna.LIB.dna_step_H, dna.LIB.dna_step_W, dna.LIB.dna_get_status):
        assert f(None) == dna.DNA_ERR_ARG
    assert dna.LIB.mu_step(None, 0) == dna.DNA_ERR_ARG
    assert dna.dna_strerror(dna.DNA_ERR_NONFINITE).startswith("non-positive")
    o = dna.dna_default_opts()
    assert (o.eps, o.alpha, o.rho, o.lambda_, o.dtype) == (0.01, 4.0, 0.0, 0.0, dna.DNA_F32)
