"""FP64 CPU oracle of the coupled LBM-DEM step (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library never loads it.

Parity pins live in tests/test_oracle_*.py.  Functions whose result the
paper and mathematics do not fix beyond those pins are marked in the
docstrings below.
"""
from .oracle import (Oracle, build, lattice, equilibrium, collide_node, pressure_face, pair_force,  # noqa: F401
                     set_threads, threads)
