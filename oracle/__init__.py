"""Plain FP64 CPU oracle for the Strang-preconditioned BVM/GMRES method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product (the CUDA library and
its Python binding) never imports or calls anything in this package.
"""
from .fde_oracle import *  # noqa: F401,F403
