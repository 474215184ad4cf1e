"""GB300 (sm_103a) ADER-DG time step on adaptive 3^d spacetree meshes.

The compute path lives in the CUDA library ``libader.so`` (C ABI declared in
``include/ader.h``); ``ader`` is its thin ctypes binding and ``Solver`` a
convenience wrapper that marshals torch tensors and streams.  Importing the
package does not load the library; the first call does, and raises
``RuntimeError`` if it has not been built (``python -m
paper_1806_07984_gb300.build``).  There is no CPU fallback.
"""
from . import ader  # noqa: F401
from .solver import Solver  # noqa: F401
