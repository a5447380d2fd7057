"""Plain float64 CPU oracle for the CADDeLaG hot path (TEST INFRASTRUCTURE).

This package is the checker, not the product. Only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
or run it. It shares no code with the CUDA path and never calls it.

Contents (each function cites the paper passage it follows):

* ``philox``   - Philox4x32-10 counter-based generator, written from its
                 published definition (Salmon, Moraes, Dror, Shaw, SC'11).
* ``caddelag`` - graph build, random projection, inverse chain and
                 Richardson solve (Alg. 2), exact embedding, commute times
                 (Eq. 1), CAD edge/node scores (Alg. 4).

Parity status of every function is recorded in its docstring; a function
whose result is not pinned by an independent test says "parity unpinned".
"""
from . import philox, caddelag  # noqa: F401
