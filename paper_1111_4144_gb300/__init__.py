"""Batched Cholesky factorisation and direct inversion of Hermitian positive-definite
matrices on GB300 (sm_103a), after "Matrix Inversion Using Cholesky Decomposition"
(Krishnamoorthy & Menon, arXiv 1111.4144).

The compute path is the in-tree CUDA library ``lib/libcholinv.so`` behind a C ABI
(``include/cholinv.h``); this package is its thin Python binding.  Importing the
package does not load the library; the first call that needs it does, and raises
if it is missing (there is no CPU fallback).
"""
__all__ = ["workloads"]
