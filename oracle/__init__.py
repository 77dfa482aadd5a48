"""FP64 CPU oracle for the rotation-voting hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. The product library never does.
"""
from .oracle import *  # noqa: F401,F403
