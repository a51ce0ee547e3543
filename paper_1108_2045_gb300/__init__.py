"""GB300 (sm_103a) high-occupancy multigrid (HOMG) for Poisson problems, arXiv:1108.2045.

The solver lives in ``lib/libhomg.so`` behind the C ABI of ``include/homg.h``; ``homg`` is its
Python binding and ``inputs`` holds the seeded synthetic right-hand sides.
"""

from . import inputs  # noqa: F401
