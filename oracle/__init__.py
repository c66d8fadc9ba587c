"""FP64 CPU oracle for Reduced Basis Decomposition -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The product library never imports or links it, and it shares no code with the
CUDA path.
"""
from .oracle import (  # noqa: F401
    build,
    load,
    compress,
    project,
    reconstruct,
    grad,
    TOL_MODES,
    RANK_FLOOR,
)
