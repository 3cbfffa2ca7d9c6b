"""Symbolic structure of a filled (chordal) pattern (test infrastructure only).

Definitions followed here:

* filled pattern of L for a given pattern of X: column k of L holds the rows
  of column k of X below the diagonal together with I_c minus {k} for every
  child c of k, where the parent of a vertex is the first row below its
  diagonal (§2: Eq. (e-filled), the elimination tree definition and
  Eq. (e-etree-ch)).  Equivalently this is the elimination game; the
  brute-force version is ``fill_bruteforce`` and is used to pin this one.
* elimination tree: parent(k) = min I_k (§2).
* monotone degree: |I_k| (§2).
* representative vertices: i is representative iff J_i is not contained in
  J_j for any j < i (§6.1, by definition; the cliques are exactly those J_i).
* supernode partition N_k, ancestor sets A_k and clique tree par(k) following
  the steps of Algorithm 6.1 (§6.4), with an explicit tie-break rule for the
  choice of child in step 1.
* separators of a clique tree: the ancestor sets A_k of the non-root cliques
  of Algorithm 6.1, cross-checked against a maximum-weight spanning tree of
  the clique intersection graph.

Indices are 0-based here; the paper's are 1-based.
"""
from __future__ import annotations

import numpy as np


def columns_from_csc(n, colptr, rowind):
    """List of sorted strictly-lower row index arrays per column."""
    cols = []
    for j in range(n):
        r = np.asarray(rowind[colptr[j]:colptr[j + 1]], dtype=np.int64)
        cols.append(np.unique(r[r > j]))
    return cols


def fill(n, lower_cols):
    """Filled pattern I_k of L from the strictly-lower pattern of X.

    Column k of L = (rows of X below the diagonal in column k) united with
    I_c \\ {k} over the children c of k in the elimination tree; the parent
    of k is min I_k.  Returns (I, parent) with I[k] a sorted int64 array.
    """
    pending = [[] for _ in range(n)]
    I = [None] * n
    parent = np.full(n, -1, dtype=np.int64)
    for k in range(n):
        parts = [np.asarray(lower_cols[k], dtype=np.int64)] + pending[k]
        s = np.unique(np.concatenate(parts)) if parts else np.zeros(0, np.int64)
        s = s[s > k]
        I[k] = s
        if len(s):
            p = int(s[0])
            parent[k] = p
            pending[p].append(s)
        pending[k] = None
    return I, parent


def fill_bruteforce(n, lower_cols):
    """Elimination game: eliminating k makes its higher neighbours a clique."""
    adj = [set() for _ in range(n)]
    for j in range(n):
        for i in lower_cols[j]:
            adj[j].add(int(i))
            adj[int(i)].add(j)
    I = []
    for k in range(n):
        hi = sorted(v for v in adj[k] if v > k)
        for a in range(len(hi)):
            for b in range(a + 1, len(hi)):
                adj[hi[a]].add(hi[b])
                adj[hi[b]].add(hi[a])
        I.append(np.asarray(hi, dtype=np.int64))
    return I


def is_filled(n, I):
    """Eq. (e-filled): i > j > k, (i,k), (j,k) in V  =>  (i,j) in V."""
    sets = [set(map(int, x)) for x in I]
    for k in range(n):
        lst = sorted(sets[k])
        for a in range(len(lst)):
            for b in range(a + 1, len(lst)):
                if lst[b] not in sets[lst[a]]:
                    return False
    return True


def etree(I):
    return np.array([int(x[0]) if len(x) else -1 for x in I], dtype=np.int64)


def children(parent):
    n = len(parent)
    ch = [[] for _ in range(n)]
    for k in range(n):
        if parent[k] >= 0:
            ch[int(parent[k])].append(k)
    return ch


def degrees(I):
    return np.array([len(x) for x in I], dtype=np.int64)


def representatives_bruteforce(I):
    """i is representative iff J_i is not a subset of J_j for some j < i."""
    n = len(I)
    J = [set(map(int, I[k])) | {k} for k in range(n)]
    rep = []
    for i in range(n):
        if not any(J[i] <= J[j] for j in range(i)):
            rep.append(i)
    return rep


def cliques(I):
    """The maximal cliques J_i of the filled graph, one per representative."""
    n = len(I)
    return [np.concatenate([[i], I[i]]).astype(np.int64)
            for i in representatives_bruteforce(I)]


def clique_sets_fast(I, parent):
    """Cliques via Eq. (e-repr-test); used only at sizes brute force cannot do.

    Pinned against ``cliques`` on small patterns.
    """
    n = len(I)
    ch = children(parent)
    d = degrees(I)
    out = []
    for j in range(n):
        if all(d[j] > d[k] - 1 for k in ch[j]):
            out.append(np.concatenate([[j], I[j]]).astype(np.int64))
    return out


def separators_mwst(clq):
    """Separators of a clique tree built as a maximum-weight spanning tree of
    the clique intersection graph (weight |J_s ∩ J_t|; a classical
    characterisation of clique trees of chordal graphs).  Returns the list of
    non-empty separators J_s ∩ J_t over the tree edges.  Small sizes only.
    """
    m = len(clq)
    sets = [set(map(int, c)) for c in clq]
    edges = []
    for s in range(m):
        for t in range(s + 1, m):
            w = len(sets[s] & sets[t])
            if w:
                edges.append((w, s, t))
    edges.sort(key=lambda e: (-e[0], e[1], e[2]))
    root = list(range(m))

    def find(x):
        while root[x] != x:
            root[x] = root[root[x]]
            x = root[x]
        return x

    seps = []
    for w, s, t in edges:
        a, b = find(s), find(t)
        if a != b:
            root[a] = b
            seps.append(np.asarray(sorted(sets[s] & sets[t]), dtype=np.int64))
    return seps


def cliques_and_separators(I, parent, tie="last"):
    """Cliques J_k and separators A_k (non-root k) of the clique tree of
    Algorithm 6.1 (§6.3: A_k ⊂ J_par(k)); the multiset of separators is the
    same for every clique tree of the pattern."""
    N, A, par, _ = clique_tree_alg61(I, parent, tie=tie)
    cl, seps = [], []
    for k in sorted(N):
        cl.append(np.asarray(sorted(set(N[k]) | set(A[k])), dtype=np.int64))
        if par[k] >= 0:
            seps.append(np.asarray(A[k], dtype=np.int64))
    return cl, seps


def clique_tree_alg61(I, parent, tie="last"):
    """Algorithm 6.1 (§6.4): representatives, N_k, first ancestors, par(k).

    For i = 0..n-1: if |I_i| > |I_j| - 1 for every child j of i, i is a
    representative and N_i = {i}; otherwise choose a child j with
    |I_i| = |I_j| - 1 and add i to the supernode containing j.  ``tie``
    picks, among several such children, the one with the largest index
    ("last") or the smallest ("first").  Then every child j of i that lies
    in a supernode l other than i's gets par(l) = that supernode and first
    ancestor min A_l = i.

    Returns (N, A, par, snode_of): dicts keyed by representative vertex,
    with A_k = J_k \\ N_k where J_k = {k} ∪ I_k (§6.2).
    """
    n = len(I)
    ch = children(parent)
    d = degrees(I)
    snode_of = np.full(n, -1, dtype=np.int64)
    N = {}
    par = {}
    first_anc = {}
    for i in range(n):
        cand = [j for j in ch[i] if d[i] == d[j] - 1]
        if all(d[i] > d[j] - 1 for j in ch[i]):
            k = i
            N[k] = [i]
        else:
            j = max(cand) if tie == "last" else min(cand)
            k = int(snode_of[j])
            N[k].append(i)
        snode_of[i] = k
        for j in ch[i]:
            l = int(snode_of[j])
            if l != k:
                par[l] = k
                first_anc[l] = i
    A = {}
    for k, members in N.items():
        Jk = set(map(int, I[k])) | {k}
        A[k] = sorted(Jk - set(members))
    for k in N:
        par.setdefault(k, -1)
    return N, A, par, snode_of


def supernodal_pattern(n, I, snode_ptr):
    """Pattern of a partition of the columns into contiguous supernodes
    (§6.2, §7): every column j of supernode [f, l) holds the rows
    {j, .., l-1} together with the ancestor set A = I_{l-1} of the
    supernode's last column.  With the fundamental partition of a filled
    pattern this is the pattern itself; with a relaxed partition (chains of
    the elimination tree merged into one supernode) it adds the explicit
    zeros that make the merged columns share one structure.

    I: filled strictly-lower rows per column (``fill``); snode_ptr: first
    column of each supernode and n at the end.  Returns (colptr, rowind) of
    the lower CSC, diagonal included, rows increasing.
    """
    colptr = [0]
    rows = []
    for k in range(len(snode_ptr) - 1):
        f, l = int(snode_ptr[k]), int(snode_ptr[k + 1])
        A = np.asarray(I[l - 1], dtype=np.int64)
        for j in range(f, l):
            col = np.concatenate([np.arange(j, l, dtype=np.int64), A])
            rows.append(col)
            colptr.append(colptr[-1] + len(col))
    rowind = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    return np.asarray(colptr, dtype=np.int64), rowind
