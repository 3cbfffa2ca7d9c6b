"""CPU oracle for the log-det barrier on chordal sparsity patterns.

TEST INFRASTRUCTURE ONLY.  Nothing in the library (``paper_1203_2742_gb300``)
imports, links or executes this package; only ``tests/``, the ``smoke()``
check in ``__graft_entry__.py`` and the CPU-baseline leg of ``bench.py`` use
it.  It shares no code with the CUDA path.

Andersen, Dahl, Vandenberghe, "Logarithmic barriers for sparse matrix cones".

Modules
-------
``dense``         -- the definitions, computed densely in FP64 (factor, §2;
                     gradient, Eq. (e-grad-def); Hessian, §1.1 / §5; inverse
                     Hessian, §5.3; completion, Eq. (e-Xhat-eq) and
                     (e-dual-barrier-def)).
``symbolic``      -- filled pattern, elimination tree, monotone degrees,
                     cliques, supernode partitions (§2, §6, Algorithm 6.1).
``factored``      -- the completion with factored update matrices, step by
                     step (Algorithm 4.3 in the supernodal form of §7.2),
                     pinned against ``dense``'s completion.
``multifrontal``  -- the paper's scalar multifrontal algorithms, step by step
                     (Algorithms 3.1, 3.2, 4.1, 4.2, 5.1, 5.2), pinned
                     against ``dense``'s definitions.
``supernodal``    -- the supernodal block algorithms (Algorithms 7.1-7.3 and
                     the block forms of 5.1 and 5.2 the paper omits), pinned
                     against ``dense``'s definitions on several partitions.

Value layout shared with the library API: a symmetric matrix on the pattern V
is stored as the lower-triangular compressed columns (CSC) of V, rows sorted
ascending in each column, the diagonal entry first.  ``colptr`` has n+1
entries (int64), ``rowind`` holds the row indices (int32).

Every function that has no independent pin says "parity unpinned" in its
docstring.  At present every function here is pinned by tests under
``tests/test_oracle_*.py``.
"""
