"""Batched primal-dual interior-point solver for many small NLPs on one GB300.

The solver itself is CUDA (csrc/, exposed through the C ABI in include/bipm.h);
``bipm`` is its ctypes binding and ``build`` compiles the library in-tree.
"""

__all__ = ["bipm", "build"]
