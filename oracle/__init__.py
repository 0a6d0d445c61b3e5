"""FP64 CPU oracle (test infrastructure only).

Only the test suite, `__graft_entry__.smoke()` and the benchmark's CPU-baseline
leg import this package.  The CUDA library and its Python binding never do, and
the two share no code.  See oracle.c (short-range pair sum), ewald.c (exact
reciprocal-space, self and exclusion terms of the Ewald sum) and pme.py
(smooth particle-mesh Ewald in FP64) for what each piece computes.
"""
from .oracle import (  # noqa: F401
    build, brute, celllist, listset, pairs_within, vjp, energy_moments, energy_hist, num_threads, set_num_threads,
    ewald_recip, ewald_excl, ewald_self, ewald_kmax,
)
from .pme import pme, pme_grid  # noqa: F401
