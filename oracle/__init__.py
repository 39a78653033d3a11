"""Plain FP64 CPU oracle for QMC-CPW Greeks (arXiv 2209.11337).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path (the CUDA library
and its Python binding) never imports, links or runs anything here.
"""
from .oracle import *  # noqa: F401,F403
