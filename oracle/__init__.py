"""FP64 CPU oracle for the improved random batch Ewald force path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the cpu_baseline / reference leg of
``bench.py`` may import this package. The product library never uses it.
"""
from .oracle import *  # noqa: F401,F403
