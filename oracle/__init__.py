"""CPU oracle for the SuCo query path (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
path (``paper_2411_14754_gb300``) never does; it shares no code with it.
"""
from .suco_oracle import *  # noqa: F401,F403
from . import mlp_oracle  # noqa: F401,E402
