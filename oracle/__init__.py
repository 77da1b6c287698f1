"""CPU FP64 oracle for the nonlinear ship-wave residual and solve.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py``; never by the product
library.  See ``oracle.py`` for what each function follows in the paper.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build_c  # noqa: F401
