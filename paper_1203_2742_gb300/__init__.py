"""GB300 (sm_103a) library for the log-det barrier on chordal sparsity patterns.

Andersen, Dahl, Vandenberghe, "Logarithmic barriers for sparse matrix cones":
Cholesky factor, gradient -P(X^{-1}), Hessian products P(X^{-1} Y X^{-1}),
inverse-Hessian products and the maximum-determinant completion (dual
barrier) by supernodal multifrontal FP64 CUDA kernels behind a C ABI
(``include/chordal_barrier.h``).  ``paper_1203_2742_gb300.binding`` is the
Python view of that ABI; importing it loads ``libchordal_barrier.so`` (built
by ``paper_1203_2742_gb300.build.build()``) and fails if the library is
absent.
"""
