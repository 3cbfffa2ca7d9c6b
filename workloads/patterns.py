"""Sparsity patterns as lower CSC (colptr int64[n+1], rowind int32), diagonal included.

Rows are sorted ascending within a column and the diagonal is the first
entry of every column.
"""
from __future__ import annotations

import hashlib

import numpy as np


def lower_csc_from_pairs(n, rows, cols):
    """Lower CSC from (row, col) pairs; adds the diagonal, drops duplicates."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    lo = np.maximum(rows, cols)
    hi = np.minimum(rows, cols)
    d = np.arange(n, dtype=np.int64)
    r = np.concatenate([lo, d])
    c = np.concatenate([hi, d])
    key = np.unique(c * n + r)
    c = key // n
    r = key % n
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(colptr, c + 1, 1)
    colptr = np.cumsum(colptr)
    return n, colptr, r.astype(np.int32)


def band(n, w):
    """Band pattern of half-bandwidth w: (i, j) with 0 <= i - j <= w (§4.3.1)."""
    j = np.repeat(np.arange(n), w + 1)
    i = j + np.tile(np.arange(w + 1), n)
    keep = i < n
    return lower_csc_from_pairs(n, i[keep], j[keep])


def arrow(n, w):
    """Block-arrow pattern: diagonal plus dense last w rows/columns (§4.3.1)."""
    tail = np.arange(n - w, n)
    rows, cols = [], []
    for j in range(n):
        if j < n - w:
            rows.append(tail)
            cols.append(np.full(w, j))
        else:
            rr = np.arange(j, n)
            rows.append(rr)
            cols.append(np.full(len(rr), j))
    return lower_csc_from_pairs(n, np.concatenate(rows), np.concatenate(cols))


def erdos_renyi(n, p, rng):
    """Each off-diagonal pair (i > j) present independently with probability p."""
    m = n * (n - 1) // 2
    # geometric skipping over the m pairs in column-major lower order
    k = rng.binomial(m, p)
    idx = np.sort(rng.choice(m, size=k, replace=False))
    # pair index t -> (i, j): columns j hold n-1-j pairs each
    starts = np.concatenate([[0], np.cumsum(np.arange(n - 1, 0, -1))])
    j = np.searchsorted(starts, idx, side="right") - 1
    i = j + 1 + (idx - starts[j])
    return lower_csc_from_pairs(n, i, j)


def grid2d(nx, ny):
    """5-point stencil on an nx-by-ny grid, vertex (x, y) -> x + nx*y."""
    x, y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    v = (x + nx * y).ravel()
    xr, yr = x.ravel(), y.ravel()
    rows, cols = [], []
    m = xr + 1 < nx
    rows.append(v[m] + 1); cols.append(v[m])
    m = yr + 1 < ny
    rows.append(v[m] + nx); cols.append(v[m])
    return lower_csc_from_pairs(nx * ny, np.concatenate(rows), np.concatenate(cols))


def grid3d(nx, ny, nz):
    """7-point stencil on an nx-by-ny-by-nz grid, (x,y,z) -> x + nx*(y + ny*z)."""
    x, y, z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    v = (x + nx * (y + ny * z)).ravel()
    xr, yr, zr = x.ravel(), y.ravel(), z.ravel()
    rows, cols = [], []
    for cond, off in ((xr + 1 < nx, 1), (yr + 1 < ny, nx), (zr + 1 < nz, nx * ny)):
        rows.append(v[cond] + off); cols.append(v[cond])
    return lower_csc_from_pairs(nx * ny * nz, np.concatenate(rows), np.concatenate(cols))


def nested_dissection(dims, leaf=8):
    """Geometric nested-dissection order of a grid with the given dimensions.

    Recursive bisection of the box along its longest side by a one-plane
    separator; the two halves are ordered first (recursively), the separator
    last.  Boxes with at most ``leaf`` vertices are ordered lexicographically.
    Returns perm with perm[new] = old (old = lexicographic grid index,
    x fastest).
    """
    dims = tuple(int(d) for d in dims)
    order = []

    def index(coords):
        idx = 0
        stride = 1
        for c, d in zip(coords, dims):
            idx += c * stride
            stride *= d
        return idx

    def emit_box(lo, hi):
        rng = [range(l, h) for l, h in zip(lo, hi)]
        # x fastest
        import itertools
        for tup in itertools.product(*reversed(rng)):
            order.append(index(tuple(reversed(tup))))

    stack = [(tuple(0 for _ in dims), dims, False)]
    out_stack = []

    def rec(lo, hi):
        size = 1
        for l, h in zip(lo, hi):
            size *= (h - l)
        if size == 0:
            return
        if size <= leaf:
            emit_box(lo, hi)
            return
        ext = [h - l for l, h in zip(lo, hi)]
        ax = int(np.argmax(ext))
        if ext[ax] < 3:
            emit_box(lo, hi)
            return
        mid = lo[ax] + ext[ax] // 2
        lo1, hi1 = list(lo), list(hi)
        hi1[ax] = mid
        lo2, hi2 = list(lo), list(hi)
        lo2[ax] = mid + 1
        rec(tuple(lo1), tuple(hi1))
        rec(tuple(lo2), tuple(hi2))
        slo, shi = list(lo), list(hi)
        slo[ax] = mid
        shi[ax] = mid + 1
        emit_box(tuple(slo), tuple(shi))

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10000))
    try:
        rec(tuple(0 for _ in dims), dims)
    finally:
        sys.setrecursionlimit(old)
    perm = np.asarray(order, dtype=np.int64)
    assert len(perm) == int(np.prod(dims)) and len(np.unique(perm)) == len(perm)
    return perm


def permute(pattern, perm):
    """Pattern of P A P^T with perm[new] = old, as lower CSC."""
    n, colptr, rowind = pattern
    perm = np.asarray(perm, dtype=np.int64)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    cols = np.repeat(np.arange(n), np.diff(colptr))
    return lower_csc_from_pairs(n, inv[np.asarray(rowind, np.int64)], inv[cols])


def pattern_hash(pattern):
    n, colptr, rowind = pattern
    h = hashlib.sha256()
    h.update(np.int64(n).tobytes())
    h.update(np.asarray(colptr, np.int64).tobytes())
    h.update(np.asarray(rowind, np.int32).tobytes())
    return h.hexdigest()[:16]


def nd_options(dims, leaf=8):
    """The analysis options that make the library order a grid of `dims` by
    the same geometric nested dissection as nested_dissection(dims, leaf)."""
    return {"ordering": "nd_geometric", "nd_dims": tuple(int(d) for d in dims), "nd_leaf": int(leaf)}


def grid_dims(kind, n):
    """Grid dimensions of a batch_mix instance of this kind and size (None
    for the families that keep their natural order)."""
    if kind != "grid":
        return None
    side = int(round(np.sqrt(n)))
    return (side, side)


def batch_mix(count, seed, nmin=300, nmax=30000):
    """Independent instances for batched runs: n log-uniform in [nmin, nmax],
    a third each band (half-bandwidth uniform in 4..64), block arrow (arrow
    width 32) and 2D grid (side round(sqrt(n))) with a geometric nested
    dissection order.  Returns a list of (pattern, perm or None, kind)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        kind = ("band", "arrow", "grid")[i % 3]
        if kind == "band":
            out.append((band(n, int(rng.integers(4, 65))), None, kind))
        elif kind == "arrow":
            out.append((arrow(n, 32), None, kind))
        else:
            side = max(2, int(round(np.sqrt(n))))
            out.append((grid2d(side, side), nested_dissection((side, side), leaf=8), kind))
    return out
