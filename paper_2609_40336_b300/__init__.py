"""B300-native message-passing dual solvers for local relaxation hierarchies.

The compute path is the CUDA library ``liblrh.so`` (C ABI in include/lrh.h);
``Solver`` is its thin Python binding.  Importing this package does not load
the library; constructing a ``Solver`` does, and fails loudly if it is not
built.
"""
from .solver import Solver, marshal  # noqa: F401

__all__ = ["Solver", "marshal"]
