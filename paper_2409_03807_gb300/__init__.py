"""GB300-native neural-subspace reduced-order solver (projective Newton in a
Lipschitz-optimisable MLP subspace, arxiv 2409.03807).

The compute path is the CUDA library liblsn (C ABI in include/lsn.h); this
package holds its sources (csrc/), the in-tree build (build.py) and a thin
ctypes binding (_native.py).  There is no CPU fallback: using the solver
without the built library raises.
"""
from ._native import (Context, LsnError, LsnStats, load, exported_symbols, PRECISIONS,
                      LSN_OK, LSN_NOT_CONVERGED, LSN_LS_FAILED, LSN_NOT_SPD,
                      LSN_PRECISION_FLOOR, LSN_SADDLE, OPTIMIZERS)
from .problem import context_from_problem

__all__ = ["Context", "LsnError", "LsnStats", "load", "exported_symbols", "PRECISIONS",
           "context_from_problem", "LSN_OK", "LSN_NOT_CONVERGED", "LSN_LS_FAILED",
           "LSN_NOT_SPD", "LSN_PRECISION_FLOOR", "LSN_SADDLE", "OPTIMIZERS"]
