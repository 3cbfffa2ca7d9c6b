"""Pins of the oracle's symbolic routines against the paper's worked example
(Figure 1, Table t-example, Figure f-etree2) and against brute force."""
import json
import os

import numpy as np
import pytest

from oracle import symbolic as OS
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def fig1():
    pairs = np.loadtxt(os.path.join(GOLD, "fig1_pattern.txt"), dtype=np.int64, comments="#")
    return W.lower_csc_from_pairs(17, pairs[:, 0], pairs[:, 1])


def gold():
    with open(os.path.join(GOLD, "fig1_symbolic.json")) as f:
        return json.load(f)


def fig1_structure():
    n, cp, ri = fig1()
    cols = OS.columns_from_csc(n, cp, ri)
    I, parent = OS.fill(n, cols)
    return n, cols, I, parent


def test_fig1_is_filled_and_fill_adds_nothing():
    n, cols, I, parent = fig1_structure()
    assert OS.is_filled(n, cols)
    for k in range(n):
        assert list(I[k]) == list(cols[k])
    # the text's example: (5,3),(15,3) in V implies (15,5) in V (1-based)
    assert 14 in set(I[4])


def test_fig1_etree_matches_figure():
    n, cols, I, parent = fig1_structure()
    g = gold()["etree_edges_child_parent"]["value"]
    want = np.full(n, -1)
    for c, p in g:
        want[c - 1] = p - 1
    assert list(parent) == list(want)
    assert list(OS.etree(I)) == list(want)


def test_fig1_monotone_degrees():
    n, cols, I, parent = fig1_structure()
    assert list(OS.degrees(I)) == gold()["monotone_degrees"]["value"]


def test_fig1_clique_J5_dense():
    n, cols, I, parent = fig1_structure()
    J5 = [4] + list(I[4])
    assert [v + 1 for v in J5] == gold()["dense_clique_example"]["value"]
    s = [set(map(int, x)) for x in I]
    for a in J5:
        for b in J5:
            if a < b:
                assert b in s[a]


def test_fig1_representatives_definition_and_degree_test():
    n, cols, I, parent = fig1_structure()
    rep = [v + 1 for v in OS.representatives_bruteforce(I)]
    assert rep == gold()["representatives"]["value"]
    fast = sorted(int(c[0]) + 1 for c in OS.clique_sets_fast(I, parent))
    assert fast == rep


@pytest.mark.parametrize("tie,key", [("last", "partition_1"), ("first", "partition_2")])
def test_fig1_algorithm61_partitions(tie, key):
    n, cols, I, parent = fig1_structure()
    N, A, par, snode_of = OS.clique_tree_alg61(I, parent, tie=tie)
    g = gold()[key]
    got_N = {str(k + 1): [v + 1 for v in N[k]] for k in N}
    got_A = {str(k + 1): [v + 1 for v in A[k]] for k in A}
    got_par = {str(k + 1): (par[k] + 1 if par[k] >= 0 else 0) for k in par}
    assert got_N == g["N"]
    assert got_A == g["A"]
    assert got_par == g["par"]


def test_fig1_supernode_list_partition_1():
    n, cols, I, parent = fig1_structure()
    N, A, par, _ = OS.clique_tree_alg61(I, parent, tie="last")
    got = sorted([sorted(v + 1 for v in N[k]) for k in N])
    assert got == sorted(gold()["supernodes"]["value"])


def test_clique_tree_properties_fig1():
    # A_j ⊂ J_par(j) and min A_j ∈ N_par(j) (§6.3)
    n, cols, I, parent = fig1_structure()
    for tie in ("last", "first"):
        N, A, par, _ = OS.clique_tree_alg61(I, parent, tie=tie)
        for k in N:
            if par[k] >= 0:
                p = par[k]
                Jp = set(N[p]) | set(A[p])
                assert set(A[k]) <= Jp
                assert A[k][0] in N[p]


def _random_pattern(rng, n, p):
    rows, cols = [], []
    for j in range(n):
        for i in range(j + 1, n):
            if rng.random() < p:
                rows.append(i)
                cols.append(j)
    return W.lower_csc_from_pairs(n, np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64))


@pytest.mark.parametrize("seed", range(12))
def test_fill_matches_elimination_game(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 30))
    n, cp, ri = _random_pattern(rng, n, rng.uniform(0.05, 0.4))
    cols = OS.columns_from_csc(n, cp, ri)
    I, parent = OS.fill(n, cols)
    Ib = OS.fill_bruteforce(n, cols)
    assert all(list(a) == list(b) for a, b in zip(I, Ib))
    assert OS.is_filled(n, I)
    # cliques: definition vs degree test (Eq. (e-repr-test))
    c1 = sorted(tuple(map(int, c)) for c in OS.cliques(I))
    c2 = sorted(tuple(map(int, c)) for c in OS.clique_sets_fast(I, parent))
    assert c1 == c2
    # every filled column set J_k is contained in some clique
    cl = [set(c) for c in c1]
    for k in range(n):
        assert any((set(map(int, I[k])) | {k}) <= c for c in cl)
    # separators: Algorithm 6.1 clique tree (both tie-breaks) vs maximum-weight
    # spanning tree of the clique intersection graph (same multiset)
    mw = sorted(tuple(map(int, s)) for s in OS.separators_mwst(OS.cliques(I)))
    for tie in ("last", "first"):
        cl, seps = OS.cliques_and_separators(I, parent, tie=tie)
        assert sorted(tuple(map(int, c)) for c in cl) == c1
        assert sorted(tuple(map(int, s)) for s in seps if len(s)) == mw


def test_band_and_arrow_degrees():
    # §4.3.1 Figure f-band: vertices 1..n-w have monotone degree w, vertex k > n-w has n-k
    n, w = 30, 4
    p = W.band(n, w)
    I, _ = OS.fill(n, OS.columns_from_csc(*p))
    d = OS.degrees(I)
    assert all(d[k] == w for k in range(n - w))
    assert all(d[k] == n - 1 - k for k in range(n - w, n))
    # arrow: every vertex before the dense tail has degree w
    p = W.arrow(n, w)
    I, _ = OS.fill(n, OS.columns_from_csc(*p))
    d = OS.degrees(I)
    assert all(d[k] == w for k in range(n - w))
