"""FP64 CPU oracle (test infrastructure only).

Only the test suite, `__graft_entry__.smoke()` and the benchmark's CPU-baseline
leg import this package.  The CUDA library and its Python binding never do, and
the two share no code.  See oracle.c for the definitions it computes.
"""
from .oracle import (  # noqa: F401
    build, brute, celllist, listset, pairs_within, vjp, energy_moments, num_threads, set_num_threads,
)
