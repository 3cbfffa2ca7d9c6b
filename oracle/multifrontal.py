"""Scalar multifrontal algorithms of the paper, step by step (test
infrastructure only).

TEST INFRASTRUCTURE ONLY: used by ``tests/`` alone; shares no code with the
CUDA path.

A second, independent CPU route to the quantities ``oracle.dense`` computes
from their definitions: the paper's own recursions over the vertices of the
elimination tree, one column at a time (§3-§5): Algorithm 3.1 (Cholesky
factorization), 3.2 (Cholesky product), 4.1 (projected inverse), 4.2 (matrix
completion), 5.1 (Hessian evaluation, with V_j = S_{I_j I_j} propagated as
§5.2 suggests after the algorithm) and 5.2 (inverse Hessian evaluation).
The library's supernodal block forms reduce to these when every supernode
has one column, so agreement of the two oracles with each other pins both.

Notation (§2): V is a filled (chordal) pattern in a perfect elimination
order, I_j = the rows i > j of column j of V, the parent of j is min I_j,
I'_j = {j} followed by I_j, and for a child i of j the index set I_i is
contained in I'_j; E_{I'_j I_i} selects the positions of I_i in I'_j.
Topological order (children before parents) is increasing j.  Readings of
garbled passages: the lower-left block of Eq. (e-compl-lin) is T_{I_j j}
(not its transpose), and in Algorithm 5.2 step 3 `K_{I_j}^T` is K_{I_j j}^T.
"""
from __future__ import annotations

import numpy as np

from .dense import to_dense


def structure(n, colptr, rowind):
    """I_j, parent(j) = min I_j (-1 for a root) and children of each vertex."""
    colptr = np.asarray(colptr, dtype=np.int64)
    rows = np.asarray(rowind, dtype=np.int64)
    I, parent = [], np.full(n, -1, dtype=np.int64)
    for j in range(n):
        r = rows[colptr[j]:colptr[j + 1]]
        Ij = np.sort(r[r > j])
        I.append(Ij)
        if len(Ij):
            parent[j] = Ij[0]
    ch = [[] for _ in range(n)]
    for j in range(n):
        if parent[j] >= 0:
            ch[parent[j]].append(j)
    return I, parent, ch


def _positions(I, j, i):
    """Positions of I_i inside I'_j = (j, I_j)."""
    Jp = np.concatenate([[j], I[j]])
    where = {int(v): t for t, v in enumerate(Jp)}
    return np.array([where[int(v)] for v in I[i]], dtype=np.int64)


def cholesky(n, colptr, rowind, x):
    """Algorithm 3.1: L (unit lower, dense) and D (vector) with X = L D L^T.
    Frontal matrix F_j = [X_jj X_Ij^T; X_Ij 0] + sum over children of
    E U_i E^T; D_jj = F11, L_Ij = F21 / D_jj, U_j = F22 - D_jj L_Ij L_Ij^T."""
    X = to_dense(n, colptr, rowind, x)
    I, _, ch = structure(n, colptr, rowind)
    L, D, U = np.eye(n), np.zeros(n), [None] * n
    for j in range(n):
        Ij = I[j]
        m = len(Ij) + 1
        F = np.zeros((m, m))
        F[0, 0] = X[j, j]
        F[1:, 0] = X[Ij, j]
        F[0, 1:] = X[Ij, j]
        for i in ch[j]:
            p = _positions(I, j, i)
            F[np.ix_(p, p)] += U[i]
            U[i] = None
        D[j] = F[0, 0]
        L[Ij, j] = F[1:, 0] / D[j]
        U[j] = F[1:, 1:] - D[j] * np.outer(L[Ij, j], L[Ij, j])
    return L, D


def cholesky_product(n, colptr, rowind, L, D):
    """Algorithm 3.2: X = L D L^T on V from the factors:
    [X_jj X_Ij^T; X_Ij -U_j] = D_jj [1; L_Ij][1; L_Ij]^T - sum E U_i E^T."""
    I, _, ch = structure(n, colptr, rowind)
    X = np.zeros((n, n))
    U = [None] * n
    for j in range(n):
        Ij = I[j]
        v = np.concatenate([[1.0], L[Ij, j]])
        F = D[j] * np.outer(v, v)
        for i in ch[j]:
            p = _positions(I, j, i)
            F[np.ix_(p, p)] -= U[i]
            U[i] = None
        X[j, j] = F[0, 0]
        X[Ij, j] = X[j, Ij] = F[1:, 0]
        U[j] = -F[1:, 1:]
    return X


def _reverse_propagate(n, I, ch, column):
    """Reverse topological order with the update matrices V_j = S_{I_j I_j}:
    column(j, V_j) returns (S_jj, S_Ij); V_i = E^T [S_jj S_Ij^T; S_Ij V_j] E
    for the children i of j."""
    V = [None] * n
    for j in range(n - 1, -1, -1):
        Vj = V[j] if V[j] is not None else np.zeros((0, 0))
        sjj, sIj = column(j, Vj)
        m = len(I[j]) + 1
        Full = np.empty((m, m))
        Full[0, 0] = sjj
        Full[1:, 0] = Full[0, 1:] = sIj
        Full[1:, 1:] = Vj
        for i in ch[j]:
            p = _positions(I, j, i)
            V[i] = Full[np.ix_(p, p)]
        V[j] = None


def projected_inverse(n, colptr, rowind, L, D):
    """Algorithm 4.1: S = P(X^{-1}) from the factors, parents first:
    S_Ij = -V_j L_Ij, S_jj = 1/D_jj - S_Ij^T L_Ij."""
    I, _, ch = structure(n, colptr, rowind)
    S = np.zeros((n, n))

    def column(j, Vj):
        lj = L[I[j], j]
        sI = -Vj @ lj
        sjj = 1.0 / D[j] - sI @ lj
        S[j, j] = sjj
        S[I[j], j] = S[j, I[j]] = sI
        return sjj, sI

    _reverse_propagate(n, I, ch, column)
    return S


def completion(n, colptr, rowind, s):
    """Algorithm 4.2: the factors of X with P(X^{-1}) = S, parents first:
    L_Ij = -V_j^{-1} S_Ij, D_jj = (S_jj + S_Ij^T L_Ij)^{-1}, V from S."""
    Sd = to_dense(n, colptr, rowind, s)
    I, _, ch = structure(n, colptr, rowind)
    L, D = np.eye(n), np.zeros(n)

    def column(j, Vj):
        sI = Sd[I[j], j]
        lj = -np.linalg.solve(Vj, sI) if len(sI) else sI
        L[I[j], j] = lj
        D[j] = 1.0 / (Sd[j, j] + sI @ lj)
        return Sd[j, j], sI

    _reverse_propagate(n, I, ch, column)
    return L, D


def hessian(n, colptr, rowind, L, D, S, y):
    """Algorithm 5.1: T = P(X^{-1} Y X^{-1}) for one Y (dense symmetric S =
    P(X^{-1}) on V, e.g. from projected_inverse).
    1. children first: [K_jj K_Ij^T; K_Ij U'_j] = A (F_j) A^T with
       F_j = [Y_jj Y_Ij^T; Y_Ij 0] + sum E U'_i E^T and A = [1 0; -L_Ij I];
    2. parents first: M_jj = K_jj / D_jj^2, M_Ij = V_j K_Ij / D_jj with
       V_j = S_{I_j I_j} propagated as in Algorithm 4.1;
    3. parents first: [T_jj T_Ij^T; T_Ij V'_j] = B [M_jj M_Ij^T; M_Ij V'_j] B^T,
       B = [1 -L_Ij^T; 0 I], and V'_i = E^T [T_jj T_Ij^T; T_Ij V'_j] E."""
    Y = to_dense(n, colptr, rowind, y)
    I, _, ch = structure(n, colptr, rowind)
    Kjj, KI, Up = np.zeros(n), [None] * n, [None] * n
    for j in range(n):
        Ij = I[j]
        m = len(Ij) + 1
        F = np.zeros((m, m))
        F[0, 0] = Y[j, j]
        F[1:, 0] = F[0, 1:] = Y[Ij, j]
        for i in ch[j]:
            p = _positions(I, j, i)
            F[np.ix_(p, p)] += Up[i]
            Up[i] = None
        lj = L[Ij, j]
        A = np.eye(m)
        A[1:, 0] = -lj
        G = A @ F @ A.T
        Kjj[j], KI[j], Up[j] = G[0, 0], G[1:, 0], G[1:, 1:]
    Mjj, MI = np.zeros(n), [None] * n

    def step2(j, Vj):
        Mjj[j] = Kjj[j] / D[j] ** 2
        MI[j] = Vj @ KI[j] / D[j]
        return S[j, j], S[I[j], j]

    _reverse_propagate(n, I, ch, step2)
    T = np.zeros((n, n))
    Vp = [None] * n
    for j in range(n - 1, -1, -1):
        Ij = I[j]
        m = len(Ij) + 1
        Vj = Vp[j] if Vp[j] is not None else np.zeros((0, 0))
        Mf = np.empty((m, m))
        Mf[0, 0] = Mjj[j]
        Mf[1:, 0] = Mf[0, 1:] = MI[j]
        Mf[1:, 1:] = Vj
        Bm = np.eye(m)
        Bm[0, 1:] = -L[Ij, j]
        Tf = Bm @ Mf @ Bm.T
        T[j, j] = Tf[0, 0]
        T[Ij, j] = T[j, Ij] = Tf[1:, 0]
        for i in ch[j]:
            p = _positions(I, j, i)
            V_ = Tf.copy()
            V_[1:, 1:] = Vj
            Vp[i] = V_[np.ix_(p, p)]
        Vp[j] = None
    return T


def inv_hessian(n, colptr, rowind, L, D, S, t):
    """Algorithm 5.2: Y with P(X^{-1} Y X^{-1}) = T for one T.
    1. parents first: [M_jj M_Ij^T; M_Ij V'_j] = C [T_jj T_Ij^T; T_Ij V'_j] C^T,
       C = [1 L_Ij^T; 0 I], and V'_i = E^T [T_jj T_Ij^T; T_Ij V'_j] E;
    2. K_jj = D_jj^2 M_jj, K_Ij = D_jj S_{I_j I_j}^{-1} M_Ij;
    3. children first: [Y_jj Y_Ij^T; Y_Ij -U'_j] = G [K_jj K_Ij^T; K_Ij 0] G^T
       - sum E U'_i E^T with G = [1 0; L_Ij I]."""
    Tm = to_dense(n, colptr, rowind, t)
    I, _, ch = structure(n, colptr, rowind)
    Mjj, MI = np.zeros(n), [None] * n
    Vp = [None] * n
    for j in range(n - 1, -1, -1):
        Ij = I[j]
        m = len(Ij) + 1
        Vj = Vp[j] if Vp[j] is not None else np.zeros((0, 0))
        Tf = np.empty((m, m))
        Tf[0, 0] = Tm[j, j]
        Tf[1:, 0] = Tf[0, 1:] = Tm[Ij, j]
        Tf[1:, 1:] = Vj
        Cm = np.eye(m)
        Cm[0, 1:] = L[Ij, j]
        Mf = Cm @ Tf @ Cm.T
        Mjj[j], MI[j] = Mf[0, 0], Mf[1:, 0]
        for i in ch[j]:
            p = _positions(I, j, i)
            Vp[i] = Tf[np.ix_(p, p)]
        Vp[j] = None
    Kjj = D ** 2 * Mjj
    KI = [D[j] * np.linalg.solve(S[np.ix_(I[j], I[j])], MI[j]) if len(I[j]) else np.zeros(0) for j in range(n)]
    Y = np.zeros((n, n))
    Up = [None] * n
    for j in range(n):
        Ij = I[j]
        m = len(Ij) + 1
        Kf = np.zeros((m, m))
        Kf[0, 0] = Kjj[j]
        Kf[1:, 0] = Kf[0, 1:] = KI[j]
        Gm = np.eye(m)
        Gm[1:, 0] = L[Ij, j]
        F = Gm @ Kf @ Gm.T
        for i in ch[j]:
            p = _positions(I, j, i)
            F[np.ix_(p, p)] -= Up[i]
            Up[i] = None
        Y[j, j] = F[0, 0]
        Y[Ij, j] = Y[j, Ij] = F[1:, 0]
        Up[j] = -F[1:, 1:]
    return Y
