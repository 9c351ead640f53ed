"""GB300 adaptive multigrid for the 2D U(1) Wilson-Dirac normal equations.

The compute path is the CUDA library libmg.so (C ABI in include/mg.h); the
Python side (``mg``) only marshals device pointers to it.
"""
from . import mg  # noqa: F401

__all__ = ["mg"]
