"""FP64 CPU oracle for the tree solver (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  The product path (the C-ABI library and its Python
binding) never touches it.
"""
from . import tree_ot  # noqa: F401
