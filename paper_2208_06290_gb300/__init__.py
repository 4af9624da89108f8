"""GPU (sm_103a) direct solver for HODLR matrices (arXiv 2208.06290).

The compute path is libhodlr (CUDA kernels behind the C ABI in include/hodlr.h);
``binding`` is its thin ctypes binding. Importing ``binding`` builds / loads the
library and raises if it cannot: there is no CPU fallback.
"""

__all__ = ["binding", "build", "costs"]
