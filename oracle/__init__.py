"""CPU oracle for Gaussian Wave Splatting: plain FP64 C (``gws_oracle.c``) plus ctypes wrapper.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  It shares no code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
