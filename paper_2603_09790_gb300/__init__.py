"""GB300-native Chebyshev-basis s-step PCG with FGS Gram solves (arXiv 2603.09790).

The solver is the CUDA library ``libsstep.so`` (C ABI in ``include/sstep.h``); ``sstep``
is its thin Python binding (the library is loaded on first use and its absence is an
error) and ``inputs`` the seeded synthetic workload generator.
"""
from . import inputs  # noqa: F401
from . import sstep  # noqa: F401

__all__ = ["inputs", "sstep"]
