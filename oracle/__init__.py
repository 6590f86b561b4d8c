"""FP64 CPU oracle for partial-sky spin-s synthesis general and its adjoint.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  The product library never imports, links or runs it.
"""
from .oracle import *  # noqa: F401,F403
