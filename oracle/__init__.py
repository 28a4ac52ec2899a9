"""FP64 CPU oracle for the discrete PAT operators (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never imports it.
"""
from .oracle import *  # noqa: F401,F403
