"""FD-CGKS FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
legs may import this package.  It is independent of the CUDA library: the two
share no code, headers or helpers.
"""
from .oracle import *  # noqa: F401,F403
