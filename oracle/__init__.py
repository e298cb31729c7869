"""FP64 CPU oracle for DNA KL-NMF: test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The CUDA library never does, and this package never imports the
CUDA library.
"""
from . import dna  # noqa: F401
