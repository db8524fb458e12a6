"""FP64 CPU oracle of the lattice method (test infrastructure; never on the product path).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` and
``--impl reference`` legs) import this package.  See ``oracle/lattice.py``.
"""
from .lattice import *  # noqa: F401,F403
