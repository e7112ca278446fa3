"""CPU oracle for FP8 Ozaki-II DGEMM emulation (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The CUDA product path does not.
"""
from . import ozaki2  # noqa: F401
