"""GB300-native solver for tree-structured optimal transport with local entropic
regularisation (bipartite iterative scaling, "A parallel framework for graphical
optimal transport", Sec. 3).

The compute path is the C-ABI library ``libtreeot.so`` (hand-written sm_103a
CUDA kernels); ``treeot`` is its ctypes binding.
"""
from .treeot import (  # noqa: F401
    MLP, Solver, TreeOTError, bipartition, load, options, validate, LIB_PATH, SIGNATURES, OK, NOT_CONVERGED,
)
