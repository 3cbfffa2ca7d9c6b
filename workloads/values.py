"""Random values on a given lower-CSC pattern (input generation only)."""
from __future__ import annotations

import numpy as np


def _pairs(n, colptr, rowind):
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(np.asarray(colptr, np.int64)))
    return np.asarray(rowind, np.int64), cols


def diag_dominant(n, colptr, rowind, rng, lo=-1.0, hi=1.0, shift=1.0):
    """Off-diagonals uniform[lo, hi] on V; diagonal = symmetric row abs-sum + shift."""
    r, c = _pairs(n, colptr, rowind)
    v = rng.uniform(lo, hi, size=len(r))
    off = r != c
    v[~off] = 0.0
    rowsum = np.zeros(n)
    np.add.at(rowsum, r[off], np.abs(v[off]))
    np.add.at(rowsum, c[off], np.abs(v[off]))
    v[~off] = rowsum[r[~off]] + shift
    return v


def uniform_sym(n, colptr, rowind, rng, count=1, lo=-1.0, hi=1.0):
    """``count`` matrices with every lower entry on V uniform[lo, hi]."""
    nnz = len(rowind)
    return rng.uniform(lo, hi, size=(count, nnz))


def projected_gram(n, colptr, rowind, G, c):
    """Entries of G G^T + c I at the lower positions of V."""
    r, cc = _pairs(n, colptr, rowind)
    G = np.asarray(G, dtype=np.float64)
    out = np.einsum("ij,ij->i", G[r], G[cc])
    out[r == cc] += c
    return out


def grid_perturbed(n, colptr, rowind, grid_lower, rng, amp=0.1):
    """Grid Laplacian (4 on the diagonal, -1 on stencil neighbours; 6 and -1 in 3D
    are given by the caller through ``grid_lower``) plus E uniform[-amp, amp] on the
    off-diagonal of V, with the diagonal raised by the symmetric row abs-sum of E.

    ``grid_lower`` is a dict {(row, col): value} of the Laplacian's lower entries
    in the same (permuted) numbering as the pattern.
    """
    r, c = _pairs(n, colptr, rowind)
    e = rng.uniform(-amp, amp, size=len(r))
    off = r != c
    e[~off] = 0.0
    rowsum = np.zeros(n)
    np.add.at(rowsum, r[off], np.abs(e[off]))
    np.add.at(rowsum, c[off], np.abs(e[off]))
    v = e.copy()
    v[~off] = rowsum[r[~off]]
    key = r * n + c
    gk = np.fromiter((a * n + b for (a, b) in grid_lower.keys()), dtype=np.int64,
                     count=len(grid_lower))
    gv = np.fromiter(grid_lower.values(), dtype=np.float64, count=len(grid_lower))
    order = np.argsort(key)
    pos = np.searchsorted(key[order], gk)
    v[order[pos]] += gv
    return v


def planted_factor(n, colptr, rowind, rng, dmin=1e-6, dmax=1.0, lamp=0.1):
    """X = L0 D0 L0^T with L0 unit lower on V (off-diagonal uniform[-lamp, lamp])
    and D0 log-uniform in [dmin, dmax].

    Returns (x, l0, d0): the lower entries of X on V, the entries of L0 on V
    (ones on the diagonal) and the pivots D0.  Uses a sparse product, so it
    works at any size; for a filled pattern the product stays on V.
    """
    import scipy.sparse as sp
    r, c = _pairs(n, colptr, rowind)
    l0 = rng.uniform(-lamp, lamp, size=len(r))
    l0[r == c] = 1.0
    d0 = np.exp(rng.uniform(np.log(dmin), np.log(dmax), size=n))
    L = sp.csc_matrix((l0, (r, c)), shape=(n, n))
    Xs = (L @ sp.diags(d0) @ L.T).tocsc()
    x = np.asarray(Xs[r, c]).ravel()
    return x, l0, d0


def random_dense_lower(n, rng):
    return rng.standard_normal((n, n))
