"""CPU oracle of MRCQR -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The library itself never does.
"""
from .mrcqr_oracle import *  # noqa: F401,F403
