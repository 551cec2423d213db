"""GB300-native sparse determinant-ratio engine for variational Monte Carlo on insulators.

Computes det(A')/det(A) = 1 + u^T A^{-1} e_i for single-electron Metropolis moves on a
sparse Slater matrix with ILUTP-preconditioned GMRES, cheap rank-one preconditioner
updates, geometric reordering and the effective-stability monitor (Ahuja, Clark,
de Sturler, Ceperley, Kim, "Improved Scaling for Quantum Monte Carlo on Insulators").

The compute path is the CUDA library ``libvmc.so`` (sm_103a) behind the C ABI of
``include/vmc.h``; :mod:`.vmc` is its ctypes binding.  Importing this package loads
nothing; :func:`.build.build_library` compiles the library in-tree.
"""
__all__ = ["build", "vmc", "workloads"]
