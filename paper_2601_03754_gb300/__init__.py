"""Block-tridiagonal SPD Cholesky factor + solve on GB300 (sm_103a).

Nested-dissection (multi-stage permutation) block Cholesky: all independent
block eliminations of one dissection level run at once, over about log2(N)
levels, followed by level-wise forward and backward substitution.

The numerical work runs in hand-written CUDA kernels inside the shared library
``libbtc.so`` behind a C ABI (``include/btc.h``); ``btc`` in this package is a
thin ctypes binding with the same names. Importing the package loads nothing;
the library is loaded on first use and an error is raised if it is missing.
"""

__all__ = ["btc", "gen"]
