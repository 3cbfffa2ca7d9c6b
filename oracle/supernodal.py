"""Supernodal (block) multifrontal algorithms, step by step (test
infrastructure only).

TEST INFRASTRUCTURE ONLY: used by ``tests/`` alone; shares no code with the
CUDA path.

The paper gives Algorithms 7.1 (Cholesky factorization), 7.2 (projected
inverse) and 7.3 (matrix completion) for supernodes and omits the block
forms of the Hessian and inverse Hessian (§7).  This module restates the
three in block notation and the two omitted ones in the block form obtained
by linearising the block factorisation exactly as Eq. (e-mf-chol-lin) and
Eq. (e-compl-lin) do for single columns:

  [K_NN K_AN^T; K_AN U'] = [I 0; -L I] (Y-front + sum E U'_i E^T) [I -L^T; 0 I],
  M_NN = D^{-1} K_NN D^{-1},   M_AN = V K_AN D^{-1}   (V = S_{AA}),
  [T_NN T_AN^T; T_AN V'] = [I -L^T; 0 I] [M_NN M_AN^T; M_AN V'] [I 0; -L I],

and the inverse Hessian with the same congruences reversed (K_NN =
D M_NN D, K_AN = V^{-1} M_AN D).  With one column per supernode these are
Algorithms 3.1, 4.1, 4.2, 5.1 and 5.2 (``oracle.multifrontal``); the tests
pin them against the dense definitions on several partitions of the same
pattern.

Notation (§6.2, §7): supernode j has columns N_j and ancestor rows A_j;
J_j = N_j followed by A_j; E selects the positions of a child's A_i inside
its parent's J_j; D_NN is the dense block of the block-diagonal D and L_AN
the block of the unit lower L.
"""
from __future__ import annotations

import numpy as np

from .dense import reverse_cholesky, to_dense
from .factored import partition


def _tree(n, colptr, rowind, snode_ptr):
    N, A, par = partition(n, colptr, rowind, snode_ptr)
    ch = [[] for _ in range(len(N))]
    for i, p in enumerate(par):
        if p >= 0:
            ch[p].append(i)
    return N, A, par, ch


def _pos(N, A, j, i):
    """Positions of A_i inside J_j = (N_j, A_j)."""
    Jj = np.concatenate([N[j], A[j]])
    where = {int(v): t for t, v in enumerate(Jj)}
    return np.array([where[int(v)] for v in A[i]], dtype=np.int64)


def factor(n, colptr, rowind, x, snode_ptr):
    """Algorithm 7.1: D_NN blocks and L_AN blocks, children first:
    F = [X_NN X_AN^T; X_AN 0] + sum E U_i E^T, D_NN = F11, L_AN = F21 F11^{-1},
    U_j = F22 - L_AN D_NN L_AN^T.  Returns dense L (unit lower) and D (block
    diagonal)."""
    X = to_dense(n, colptr, rowind, x)
    N, A, par, ch = _tree(n, colptr, rowind, snode_ptr)
    L, D, U = np.eye(n), np.zeros((n, n)), [None] * len(N)
    for j in range(len(N)):
        Nj, Aj = N[j], A[j]
        nn = len(Nj)
        J = np.concatenate([Nj, Aj])
        F = X[np.ix_(J, J)].copy()
        F[nn:, nn:] = 0.0
        for i in ch[j]:
            p = _pos(N, A, j, i)
            F[np.ix_(p, p)] += U[i]
            U[i] = None
        Dj = F[:nn, :nn]
        Lj = np.linalg.solve(Dj, F[nn:, :nn].T).T
        D[np.ix_(Nj, Nj)] = Dj
        L[np.ix_(Aj, Nj)] = Lj
        U[j] = F[nn:, nn:] - Lj @ Dj @ Lj.T
    return L, D


def _parents_first(N, A, ch, block):
    """Parents first with V_j = S_{A_j A_j}: block(j, V_j) returns the J_j x
    J_j matrix [S_NN S_AN^T; S_AN V_j]; children get V_i = E^T (it) E."""
    V = [None] * len(N)
    for j in range(len(N) - 1, -1, -1):
        Vj = V[j] if V[j] is not None else np.zeros((0, 0))
        Full = block(j, Vj)
        for i in ch[j]:
            p = _pos(N, A, j, i)
            V[i] = Full[np.ix_(p, p)]
        V[j] = None


def projected_inverse(n, colptr, rowind, L, D, snode_ptr):
    """Algorithm 7.2: S = P(X^{-1}), parents first:
    S_AN = -V_j L_AN, S_NN = D_NN^{-1} - S_AN^T L_AN."""
    N, A, par, ch = _tree(n, colptr, rowind, snode_ptr)
    S = np.zeros((n, n))

    def block(j, Vj):
        Nj, Aj = N[j], A[j]
        Lj = L[np.ix_(Aj, Nj)]
        SAN = -Vj @ Lj
        SNN = np.linalg.inv(D[np.ix_(Nj, Nj)]) - SAN.T @ Lj
        S[np.ix_(Nj, Nj)] = SNN
        S[np.ix_(Aj, Nj)] = SAN
        S[np.ix_(Nj, Aj)] = SAN.T
        return np.block([[SNN, SAN.T], [SAN, Vj]])

    _parents_first(N, A, ch, block)
    return S


def completion(n, colptr, rowind, s, snode_ptr):
    """Algorithm 7.3: L and D of X with P(X^{-1}) = S, parents first:
    L_AN = -V_j^{-1} S_AN, D_NN = (S_NN + S_AN^T L_AN)^{-1}, V from S."""
    Sd = to_dense(n, colptr, rowind, s)
    N, A, par, ch = _tree(n, colptr, rowind, snode_ptr)
    L, D = np.eye(n), np.zeros((n, n))

    def block(j, Vj):
        Nj, Aj = N[j], A[j]
        SAN, SNN = Sd[np.ix_(Aj, Nj)], Sd[np.ix_(Nj, Nj)]
        Lj = -np.linalg.solve(Vj, SAN) if len(Aj) else np.zeros((0, len(Nj)))
        L[np.ix_(Aj, Nj)] = Lj
        D[np.ix_(Nj, Nj)] = np.linalg.inv(SNN + SAN.T @ Lj)
        return np.block([[SNN, SAN.T], [SAN, Vj]])

    _parents_first(N, A, ch, block)
    return L, D


def _hessian_step1(Y, L, N, A, ch):
    """Step 1 of the block Hessian, children first: [K_NN K_AN^T; K_AN U'_j]
    = [I 0; -L_AN I] (Y-front + sum E U'_i E^T) [I -L_AN^T; 0 I]."""
    ns = len(N)
    KNN, KAN, Up = [None] * ns, [None] * ns, [None] * ns
    for j in range(ns):
        Nj, Aj = N[j], A[j]
        nn = len(Nj)
        J = np.concatenate([Nj, Aj])
        F = Y[np.ix_(J, J)].copy()
        F[nn:, nn:] = 0.0
        for i in ch[j]:
            p = _pos(N, A, j, i)
            F[np.ix_(p, p)] += Up[i]
            Up[i] = None
        Am = np.eye(len(J))
        Am[nn:, :nn] = -L[np.ix_(Aj, Nj)]
        G = Am @ F @ Am.T
        KNN[j], KAN[j], Up[j] = G[:nn, :nn], G[nn:, :nn], G[nn:, nn:]
    return KNN, KAN


def hessian(n, colptr, rowind, L, D, S, y, snode_ptr):
    """Block form of Algorithm 5.1 (module docstring): T = P(X^{-1} Y X^{-1})."""
    Y = to_dense(n, colptr, rowind, y)
    N, A, par, ch = _tree(n, colptr, rowind, snode_ptr)
    ns = len(N)
    KNN, KAN = _hessian_step1(Y, L, N, A, ch)
    MNN, MAN = [None] * ns, [None] * ns

    def step2(j, Vj):
        Nj, Aj = N[j], A[j]
        Dinv = np.linalg.inv(D[np.ix_(Nj, Nj)])
        MNN[j] = Dinv @ KNN[j] @ Dinv
        MAN[j] = Vj @ KAN[j] @ Dinv
        SAN = S[np.ix_(Aj, Nj)]
        return np.block([[S[np.ix_(Nj, Nj)], SAN.T], [SAN, Vj]])

    _parents_first(N, A, ch, step2)
    T = np.zeros((n, n))

    def step3(j, Vp):
        Nj, Aj = N[j], A[j]
        nn = len(Nj)
        Mf = np.block([[MNN[j], MAN[j].T], [MAN[j], Vp]])
        Bm = np.eye(nn + len(Aj))
        Bm[:nn, nn:] = -L[np.ix_(Aj, Nj)].T
        Tf = Bm @ Mf @ Bm.T
        T[np.ix_(Nj, Nj)] = Tf[:nn, :nn]
        T[np.ix_(Aj, Nj)] = Tf[nn:, :nn]
        T[np.ix_(Nj, Aj)] = Tf[:nn, nn:]
        return Tf

    _parents_first(N, A, ch, step3)
    return T


def inv_hessian(n, colptr, rowind, L, D, S, t, snode_ptr):
    """Block form of Algorithm 5.2 (module docstring): Y with H(Y) = T."""
    Tm = to_dense(n, colptr, rowind, t)
    N, A, par, ch = _tree(n, colptr, rowind, snode_ptr)
    ns = len(N)
    MNN, MAN = [None] * ns, [None] * ns

    def step1(j, Vp):
        Nj, Aj = N[j], A[j]
        nn = len(Nj)
        TAN = Tm[np.ix_(Aj, Nj)]
        Tf = np.block([[Tm[np.ix_(Nj, Nj)], TAN.T], [TAN, Vp]])
        Cm = np.eye(nn + len(Aj))
        Cm[:nn, nn:] = L[np.ix_(Aj, Nj)].T
        Mf = Cm @ Tf @ Cm.T
        MNN[j], MAN[j] = Mf[:nn, :nn], Mf[nn:, :nn]
        return Tf

    _parents_first(N, A, ch, step1)
    Y = np.zeros((n, n))
    Up = [None] * ns
    for j in range(ns):
        Nj, Aj = N[j], A[j]
        nn = len(Nj)
        Dj = D[np.ix_(Nj, Nj)]
        KNN = Dj @ MNN[j] @ Dj
        KAN = np.linalg.solve(S[np.ix_(Aj, Aj)], MAN[j] @ Dj) if len(Aj) else np.zeros((0, nn))
        Kf = np.block([[KNN, KAN.T], [KAN, np.zeros((len(Aj), len(Aj)))]])
        Gm = np.eye(nn + len(Aj))
        Gm[nn:, :nn] = L[np.ix_(Aj, Nj)]
        F = Gm @ Kf @ Gm.T
        for i in ch[j]:
            p = _pos(N, A, j, i)
            F[np.ix_(p, p)] -= Up[i]
            Up[i] = None
        J = np.concatenate([Nj, Aj])
        Y[np.ix_(Nj, J)] = F[:nn, :]
        Y[np.ix_(Aj, Nj)] = F[nn:, :nn]
        Up[j] = -F[nn:, nn:]
    return Y


def hessian_factor(n, colptr, rowind, L, D, S, y, snode_ptr):
    """Block form of W = R(Y) (Algorithm 5.3, §5.4): K from the block
    Hessian's step 1, then per supernode, with D_NN = C C^T (C lower) and
    V = S_{AA} = Q Q^T (Q upper, the factor §5.4 prescribes):
    W_NN = C^{-1} K_NN C^{-T} (its lower triangle) and W_AN = Q^T K_AN C^{-T}.
    Returns W as a dense lower triangular matrix on V."""
    Y = to_dense(n, colptr, rowind, y)
    N, A, par, ch = _tree(n, colptr, rowind, snode_ptr)
    ns = len(N)
    KNN, KAN = _hessian_step1(Y, L, N, A, ch)
    W = np.zeros((n, n))
    for j in range(ns):
        Nj, Aj = N[j], A[j]
        C = np.linalg.cholesky(D[np.ix_(Nj, Nj)])
        Ci = np.linalg.inv(C)
        W[np.ix_(Nj, Nj)] = np.tril(Ci @ KNN[j] @ Ci.T)
        if len(Aj):
            Q = reverse_cholesky(S[np.ix_(Aj, Aj)])
            W[np.ix_(Aj, Nj)] = Q.T @ KAN[j] @ Ci.T
    return W


def hessian_factor_adj(n, colptr, rowind, L, D, S, w, snode_ptr):
    """Block form of T = R^adj(W) (Algorithm 5.4): per supernode
    M_NN = C^{-T} W_NN C^{-1} (W_NN symmetric from its lower triangle) and
    M_AN = Q W_AN C^{-1}, then the block Hessian's step 3."""
    Wl = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(np.asarray(colptr)))
    Wl[np.asarray(rowind, dtype=np.int64), rows] = w
    N, A, par, ch = _tree(n, colptr, rowind, snode_ptr)
    ns = len(N)
    MNN, MAN = [None] * ns, [None] * ns
    for j in range(ns):
        Nj, Aj = N[j], A[j]
        C = np.linalg.cholesky(D[np.ix_(Nj, Nj)])
        Ci = np.linalg.inv(C)
        Wn = Wl[np.ix_(Nj, Nj)]
        Wn = Wn + np.tril(Wn, -1).T
        MNN[j] = Ci.T @ Wn @ Ci
        if len(Aj):
            Q = reverse_cholesky(S[np.ix_(Aj, Aj)])
            MAN[j] = Q @ Wl[np.ix_(Aj, Nj)] @ Ci
        else:
            MAN[j] = np.zeros((0, len(Nj)))
    T = np.zeros((n, n))

    def step3(j, Vp):
        Nj, Aj = N[j], A[j]
        nn = len(Nj)
        Mf = np.block([[MNN[j], MAN[j].T], [MAN[j], Vp]])
        Bm = np.eye(nn + len(Aj))
        Bm[:nn, nn:] = -L[np.ix_(Aj, Nj)].T
        Tf = Bm @ Mf @ Bm.T
        T[np.ix_(Nj, Nj)] = Tf[:nn, :nn]
        T[np.ix_(Aj, Nj)] = Tf[nn:, :nn]
        T[np.ix_(Nj, Aj)] = Tf[:nn, nn:]
        return Tf

    _parents_first(N, A, ch, step3)
    return T
