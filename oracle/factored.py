"""Completion with factored update matrices (test infrastructure only).

TEST INFRASTRUCTURE ONLY: used by ``tests/`` alone; shares no code with the
CUDA path.

Unlike ``oracle.dense``, which computes definitions, this module restates an
algorithm step by step: Algorithm 4.3 (§4.2, "completion with factored
update matrices") in the supernodal form given at the end of §7.2
(Algorithm 7.3 with the factorization V_j = R_j R_j^T propagated instead of
V_j).  Its result is the max-det completion factor, pinned against the
definitions in ``oracle.dense`` (the closed form and Newton's method); its
intermediate factors R_j are pinned by R_j R_j^T = S_{A_j A_j} (§7.2: V_j is
the submatrix of S on the ancestor set).  Library primitives serve as steps:
scipy's RQ decomposition (Householder reflections) for the reduction
C = R Q^T of Eq. (e-mfp-compl-3-factored), and dense triangular solves.

Notation (§6.2, §7): supernode j has the columns N_j (contiguous) and the
ancestor rows A_j; J_j = N_j ∪ A_j.  Supernodes are processed in reverse
topological order of the clique tree (parents first); with supernodes
numbered in a postorder, that is decreasing supernode index.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .dense import reverse_cholesky, to_dense, project


def partition(n, colptr, rowind, snode_ptr):
    """N_j, A_j and the parent of each supernode of a contiguous partition
    of V (the columns of a supernode share the rows A_j of its last column,
    §7): A_j = the rows of column l-1 below the supernode [f, l); the parent
    is the supernode holding min A_j (-1 for a root)."""
    colptr = np.asarray(colptr, dtype=np.int64)
    rows = np.asarray(rowind, dtype=np.int64)
    sp = np.asarray(snode_ptr, dtype=np.int64)
    owner = np.repeat(np.arange(len(sp) - 1), np.diff(sp))
    N, A, par = [], [], []
    for j in range(len(sp) - 1):
        f, l = int(sp[j]), int(sp[j + 1])
        col = rows[colptr[l - 1]:colptr[l]]
        a = col[col >= l]
        N.append(np.arange(f, l, dtype=np.int64))
        A.append(a)
        par.append(int(owner[a[0]]) if len(a) else -1)
    return N, A, np.asarray(par, dtype=np.int64)


def completion_factored(n, colptr, rowind, s, snode_ptr):
    """X-hat with P(X-hat^{-1}) = S by the supernodal completion with
    factored update matrices.

    For each supernode j, parents first, with V_j = R_j R_j^T (R_j upper
    triangular; empty for a root):
      L_{A_j N_j} = -R_j^{-T} R_j^{-1} S_{A_j N_j},
      D_{N_j N_j} = (S_{N_j N_j} + S_{A_j N_j}^T L_{A_j N_j})^{-1}   (Eq. (e-sn-compl-1));
    and for each child i of j, with A_i split into A_i ∩ N_j (first) and
    A_i \\ N_j (rows of A_j):
      A = S on (A_i ∩ N_j)^2,  B = S on (A_i \\ N_j) x (A_i ∩ N_j),
      C = the rows of R_j at the positions of A_i \\ N_j in A_j,
      C = R Q^T (R square upper triangular, Q with orthonormal columns),
      A - B^T R^{-T} R^{-1} B = R~ R~^T (R~ upper triangular),
      R_i = [[R~, (R^{-1} B)^T], [0, R]].
    Then X-hat = L D L^T with L unit lower (identity blocks on N_j x N_j)
    and D block diagonal.

    Returns (x, Rs, deleted): the lower entries of X-hat on V, the list of
    R_j, and per supernode the number of rows of R_parent deleted to form C
    (|A_parent| - |A_i \\ N_parent|; the work of the Householder reduction
    grows with it, §4.2).
    """
    N, A, par = partition(n, colptr, rowind, snode_ptr)
    S = to_dense(n, colptr, rowind, s)
    nsn = len(N)
    ch = [[] for _ in range(nsn)]
    for i in range(nsn):
        if par[i] >= 0:
            ch[par[i]].append(i)
    L = np.eye(n)
    D = np.zeros((n, n))
    Rs = [None] * nsn
    deleted = np.zeros(nsn, dtype=np.int64)
    for j in range(nsn - 1, -1, -1):
        Nj, Aj = N[j], A[j]
        if Rs[j] is None:
            Rs[j] = np.zeros((0, 0))
        Rj = Rs[j]
        S_AN = S[np.ix_(Aj, Nj)]
        S_NN = S[np.ix_(Nj, Nj)]
        if len(Aj):
            L_AN = -sla.solve_triangular(Rj, sla.solve_triangular(Rj, S_AN, lower=False), lower=False, trans="T")
        else:
            L_AN = np.zeros((0, len(Nj)))
        D_NN = np.linalg.inv(S_NN + S_AN.T @ L_AN)
        L[np.ix_(Aj, Nj)] = L_AN
        D[np.ix_(Nj, Nj)] = D_NN
        pos = {int(v): t for t, v in enumerate(Aj)}
        for i in ch[j]:
            Ai = A[i]
            inN = Ai[Ai <= Nj[-1]]  # A_i ∩ N_j: indices of N_j are below those of A_j
            out = Ai[Ai > Nj[-1]]   # A_i \ N_j, a subset of A_j
            deleted[i] = len(Aj) - len(out)
            Amat = S[np.ix_(inN, inN)]
            Bmat = S[np.ix_(out, inN)]
            if len(out):
                C = Rj[[pos[int(v)] for v in out], :]
                R, _ = sla.rq(C, mode="economic")
                W = sla.solve_triangular(R, Bmat, lower=False)  # R^{-1} B
            else:
                R = np.zeros((0, 0))
                W = np.zeros((0, len(inN)))
            Rt = reverse_cholesky(Amat - W.T @ W) if len(inN) else np.zeros((0, 0))
            p, q = len(inN), len(out)
            Ri = np.zeros((p + q, p + q))
            Ri[:p, :p] = Rt
            Ri[:p, p:] = W.T
            Ri[p:, p:] = R
            Rs[i] = Ri
    X = L @ D @ L.T
    return project(n, colptr, rowind, X), Rs, deleted
