"""Randomized block Krylov truncated T-SVD (arXiv 2504.04989) on one GB300.

The compute path is the C-ABI library ``libtsvd`` (hand-written sm_103a CUDA
kernels, declared in include/tsvd.h); this package is its thin Python binding.
Importing the package loads nothing; the first call of an op loads the library
and raises if it is missing.
"""
__all__ = ["workloads"]
