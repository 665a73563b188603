"""FP64 CPU oracle for the sliding Frank-Wolfe hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA library.
"""

from .oracle import *  # noqa: F401,F403
