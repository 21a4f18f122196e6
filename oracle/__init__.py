"""FP64 CPU oracle for the explicit finite-difference sweep (TEST INFRASTRUCTURE ONLY).

This package is the slow, plain reference that the CUDA path is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product library never does, and it shares no
code with ``paper_1906_10811_b300`` (its weights, loops, interpolation and
Laplacian are all written independently here).

Contents
--------
weights   exact rational central second-derivative weights (space order so),
          solved from the Taylor moment system in ``fractions.Fraction``.
core      ctypes binding to ``fd_oracle.c`` (plain FP64 C loops): Laplacian,
          diffusion sweep, acoustic sweep with damping, source injection and
          receiver interpolation.
dense     brute force on tiny grids: the operator assembled as a dense matrix
          from Kronecker products, the sparse operators from tent functions.

Parity status: every function here is pinned by tests in ``tests/test_oracle_*``
(closed forms, invariants, brute force, golden values); see the module headers.
"""

from .weights import fd_weights_fraction, fd_weights  # noqa: F401
