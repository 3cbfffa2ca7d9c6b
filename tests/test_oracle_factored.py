"""Pins of the factored completion (Algorithm 4.3, supernodal form of §7.2)
against what the mathematics fixes: its X-hat is the max-det completion
(the closed form of chordal patterns and Newton's method on Eq.
(e-dual-barrier-def) reach it by other routes), and every propagated factor
satisfies R_j R_j^T = S_{A_j A_j} with R_j upper triangular."""
import numpy as np
import pytest

from oracle import dense as OD
from oracle import factored as OF
from oracle import symbolic as OS
import workloads as W


def _filled(pattern):
    n, cp, ri = pattern
    I, parent = OS.fill(n, OS.columns_from_csc(n, cp, ri))
    return n, I, parent


def _chain_partition(n, I, parent):
    """Contiguous supernodes along the chains of Algorithm 6.1."""
    N, _, _, _ = OS.clique_tree_alg61(I, parent, tie="last")
    member = {}
    for k, cols in N.items():
        for c in cols:
            member[c] = k
    sp = [0] + [j for j in range(1, n) if member[j] != member[j - 1] or j - 1 not in N[member[j]]] + [n]
    return sp


def _case(name):
    """(n, colptr, rowind, snode_ptr): a filled pattern and a contiguous
    partition of it (singletons: the scalar Algorithm 4.3; chains:
    fundamental supernodes; merged: supernodes with added zeros)."""
    if name.startswith("band"):
        pat = W.band(30, 4)
    elif name.startswith("grid"):
        pat = W.permute(W.grid2d(7, 7), W.nested_dissection((7, 7), leaf=4))
    elif name.startswith("arrow"):
        pat = W.arrow(24, 4)
    else:
        rng = np.random.default_rng(8)
        pat = W.permute(W.erdos_renyi(36, 0.1, rng), rng.permutation(36))
    n, I, parent = _filled(pat)
    if name.endswith("singletons"):
        sp = list(range(n + 1))
    elif name.endswith("chains"):
        sp = _chain_partition(n, I, parent)
    else:  # merged: blocks of 4 columns on the band (chains of the etree)
        sp = list(range(0, n, 4)) + [n]
    cp, ri = OS.supernodal_pattern(n, I, sp)
    return n, cp, ri, sp


CASES = ["band_singletons", "band_chains", "band_merged", "grid_singletons", "grid_chains",
         "arrow_chains", "random_singletons", "random_chains"]


def _gram(n, cp, ri, seed, c=0.5):
    rng = np.random.default_rng(seed)
    return W.projected_gram(n, cp, ri, rng.standard_normal((n, 4)), c)


@pytest.mark.parametrize("name", CASES)
def test_factored_completion_is_the_maxdet_completion(name):
    n, cp, ri, sp = _case(name)
    s = _gram(n, cp, ri, 1)
    x, Rs, _ = OF.completion_factored(n, cp, ri, s, sp)
    I = [np.asarray(ri[cp[k] + 1:cp[k + 1]], dtype=np.int64) for k in range(n)]
    parent = OS.etree(I)
    cl, seps = OS.cliques_and_separators(I, parent)
    ref = OD.completion_refined(n, cp, ri, s, cl, seps)
    assert OD.rel_err(n, cp, ri, x, ref) < 1e-12
    # P(X-hat^{-1}) = S, the defining equation (Eq. (e-Xhat-eq))
    assert OD.rel_err(n, cp, ri, OD.projected_inverse(n, cp, ri, x), s) < 1e-11


@pytest.mark.parametrize("name", CASES)
def test_propagated_factors_are_factors_of_the_ancestor_blocks(name):
    n, cp, ri, sp = _case(name)
    s = _gram(n, cp, ri, 2)
    S = OD.to_dense(n, cp, ri, s)
    _, Rs, _ = OF.completion_factored(n, cp, ri, s, sp)
    N, A, par = OF.partition(n, cp, ri, sp)
    for j, R in enumerate(Rs):
        assert R.shape == (len(A[j]), len(A[j]))
        assert np.allclose(np.tril(R, -1), 0.0)
        if len(A[j]):
            V = S[np.ix_(A[j], A[j])]
            assert np.linalg.norm(R @ R.T - V) <= 1e-13 * np.linalg.norm(V)


def test_newton_agrees_on_a_tiny_pattern():
    """Another route to X-hat: Newton's method with a dense Hessian solve."""
    n, cp, ri, sp = _case("grid_chains")
    s = _gram(n, cp, ri, 3, c=1.0)
    x, _, _ = OF.completion_factored(n, cp, ri, s, sp)
    assert OD.rel_err(n, cp, ri, x, OD.completion_newton(n, cp, ri, s)) < 1e-12


def test_deleted_rows_of_a_band():
    """Half-bandwidth w, natural order, one column per supernode: A_j =
    {j+1..j+w}, A_{j+1} = {j+2..j+w+1}, so C drops exactly one row of
    R_{j+1} (its last) for every j < n-w-1, and none near the root."""
    n, w = 30, 4
    pat = W.band(n, w)
    _, I, parent = _filled(pat)
    sp = list(range(n + 1))
    cp, ri = OS.supernodal_pattern(n, I, sp)
    s = _gram(n, cp, ri, 4)
    _, _, deleted = OF.completion_factored(n, cp, ri, s, sp)
    assert deleted[:n - w - 1].tolist() == [1] * (n - w - 1)
    assert deleted[n - w - 1:].tolist() == [0] * (w + 1)


def test_chain_without_deletions_keeps_the_parent_factor():
    """When A_i = J_j (a split supernode's pieces), no row is deleted: R is
    R_j itself up to the signs of its columns."""
    n = 12
    pat = W.band(n, n - 1)  # dense
    _, I, parent = _filled(pat)
    sp = [0, 4, 8, 12]
    cp, ri = OS.supernodal_pattern(n, I, sp)
    s = _gram(n, cp, ri, 5)
    _, Rs, deleted = OF.completion_factored(n, cp, ri, s, sp)
    assert deleted.tolist() == [0, 0, 0]
    # piece 0's V = S on {4..11}; its trailing block R is piece 1's R_1
    R0, R1 = Rs[0], Rs[1]
    assert np.allclose(np.abs(R0[4:, 4:]), np.abs(R1), rtol=0, atol=1e-13 * np.abs(R1).max())
