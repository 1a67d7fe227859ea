"""FP64 CPU oracle of the D3Q27 FPC-LBM (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library never does.
"""
from .oracle import *  # noqa: F401,F403
