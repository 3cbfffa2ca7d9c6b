"""The library's host symbolic phase (chd_analyze) against the paper's worked
example and the oracle's symbolic routines.  Integer results: bit-exact."""
import json
import os

import numpy as np
import pytest

from oracle import symbolic as OS
import workloads as W
from tests.helpers import lib, product_structure

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def fig1():
    pairs = np.loadtxt(os.path.join(GOLD, "fig1_pattern.txt"), dtype=np.int64, comments="#")
    return W.lower_csc_from_pairs(17, pairs[:, 0], pairs[:, 1])


@pytest.mark.parametrize("tie,key", [(True, "partition_1"), (False, "partition_2")])
def test_fig1_supernodes_and_clique_tree(tie, key):
    B = lib()
    g = json.load(open(os.path.join(GOLD, "fig1_symbolic.json")))[key]
    sym = B.Symbolic(*fig1(), tie_last=tie)
    assert sym.nnz == len(fig1()[2])  # filled already: no fill
    st = product_structure(B, sym)
    # map representative (paper label) -> (N, A)
    got = {}
    for N, A, par in st:
        got[str(min(N) + 1)] = ([v + 1 for v in N], [v + 1 for v in A], par)
    assert {k: v[0] for k, v in got.items()} == g["N"]
    assert {k: v[1] for k, v in got.items()} == g["A"]
    rep_of_index = [str(min(N) + 1) for N, A, par in st]
    par = {rep_of_index[i]: (int(rep_of_index[p]) if p >= 0 else 0) for i, (_, _, p) in enumerate(st)}
    assert par == g["par"]


def _oracle_filled_pairs(pattern, perm):
    n, cp, ri = W.permute(pattern, perm)
    I, _ = OS.fill(n, OS.columns_from_csc(n, cp, ri))
    return {(int(r), k) for k in range(n) for r in I[k]} | {(k, k) for k in range(n)}


def _product_pairs(sym):
    cols = np.repeat(np.arange(sym.n), np.diff(sym.colptr))
    return set(zip(sym.rowind.astype(int).tolist(), cols.tolist()))


CASES = {
    "band": (lambda: W.band(60, 5), "natural", None),
    "arrow": (lambda: W.arrow(50, 6), "natural", None),
    "grid_nd": (lambda: W.grid2d(12, 12), "user", lambda: W.nested_dissection((12, 12), leaf=6)),
    "grid3d_nd": (lambda: W.grid3d(6, 6, 6), "user", lambda: W.nested_dissection((6, 6, 6), leaf=8)),
    "er_mindeg": (lambda: W.erdos_renyi(300, 0.02, np.random.default_rng(3)), "mindeg", None),
    "er_natural": (lambda: W.erdos_renyi(120, 0.03, np.random.default_rng(4)), "natural", None),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fill_and_supernodes_match_oracle(name):
    B = lib()
    mk, ordering, permf = CASES[name]
    pattern = mk()
    perm_in = permf() if permf else None
    sym = B.Symbolic(*pattern, ordering=ordering, perm=perm_in)
    perm = sym.perm
    assert sorted(perm.tolist()) == list(range(sym.n))
    # V in the analysed order equals the oracle's filled pattern for that order
    assert _product_pairs(sym) == _oracle_filled_pairs(pattern, perm)
    # supernodes: contiguous, and identical to Algorithm 6.1 (tie: last child) run
    # by the oracle on the analysed order
    n = sym.n
    p2 = W.permute(pattern, perm)
    I, parent = OS.fill(n, OS.columns_from_csc(*p2))
    N, A, par, snode_of = OS.clique_tree_alg61(I, parent, tie="last")
    sp, spar, rp, rows = sym.supernodes()
    got = []
    for k in range(len(sp) - 1):
        nk = int(sp[k + 1] - sp[k])
        J = rows[rp[k]:rp[k + 1]]
        assert list(J[:nk]) == list(range(sp[k], sp[k + 1]))
        got.append((tuple(int(v) for v in J[:nk]), tuple(int(v) for v in J[nk:])))
    want = sorted((tuple(N[k]), tuple(A[k])) for k in N)
    assert sorted(got) == want
    # clique tree parents: the supernode containing min A_k
    owner = np.empty(n, dtype=np.int64)
    for k in range(len(sp) - 1):
        owner[sp[k]:sp[k + 1]] = k
    for k in range(len(sp) - 1):
        nk = int(sp[k + 1] - sp[k])
        J = rows[rp[k]:rp[k + 1]]
        assert spar[k] == (owner[J[nk]] if len(J) > nk else -1)
        if spar[k] >= 0:
            assert spar[k] > k  # postorder numbering: parents after children


@pytest.mark.parametrize("relax", [4, 16, 64])
def test_relaxed_supernodes_only_add_entries(relax):
    B = lib()
    pattern = W.erdos_renyi(400, 0.01, np.random.default_rng(9))
    s0 = B.Symbolic(*pattern, ordering="mindeg", relax=0)
    s1 = B.Symbolic(*pattern, ordering="mindeg", relax=relax)
    assert (s0.perm == s1.perm).all()
    p0, p1 = _product_pairs(s0), _product_pairs(s1)
    assert p0 <= p1
    assert s1.nsuper <= s0.nsuper
    # the enlarged pattern is still filled (Eq. (e-filled))
    n = s1.n
    I = [np.array(sorted(r for (r, c) in p1 if c == k and r > k)) for k in range(n)]
    assert OS.is_filled(n, I)


def test_flop_counts_band_scaling():
    # §4.3.1: Cholesky and projected inverse cost O(n w^2) on band patterns
    B = lib()
    f1 = B.Symbolic(*W.band(2000, 10)).flops()
    f2 = B.Symbolic(*W.band(4000, 10)).flops()
    f3 = B.Symbolic(*W.band(2000, 20)).flops()
    for op in ("factor", "gradient", "hessian"):
        assert abs(f2[op] / f1[op] - 2.0) < 0.02
        assert 3.4 < f3[op] / f1[op] < 4.6


@pytest.mark.parametrize("split", [4, 16])
def test_supernode_splitting_keeps_the_pattern(split):
    """Splitting a wide supernode into a chain (V unchanged, each piece's
    ancestor set = later columns of the original supernode + its A)."""
    B = lib()
    pattern = W.arrow(120, 40)  # dense tail of 40 columns: one wide supernode
    s0 = B.Symbolic(*pattern, split_cols=-1)
    s1 = B.Symbolic(*pattern, split_cols=split)
    assert (s0.perm == s1.perm).all()
    assert _product_pairs(s0) == _product_pairs(s1)
    assert s1.nsuper > s0.nsuper
    sp, par, rp, rows = s1.supernodes()
    widths = np.diff(sp)
    assert widths.max() <= split + split // 2
    # every supernode's structure is a clique's tail: J_k = N_k followed by A_k,
    # and the parent holds min A_k among its columns
    for k in range(len(sp) - 1):
        nk = int(sp[k + 1] - sp[k])
        J = rows[rp[k]:rp[k + 1]]
        if len(J) > nk:
            p = par[k]
            assert sp[p] <= J[nk] < sp[p + 1]


def test_batch_analysis_equals_single_analyses():
    """chd_analyze_batch: each instance keeps its own ordering, fill and
    supernodes, in a contiguous block of the union (bit-exact)."""
    B = lib()
    rng = np.random.default_rng(31)
    pats = [W.band(50, 3), W.arrow(40, 5), W.permute(W.grid2d(8, 8), W.nested_dissection((8, 8), leaf=4)),
            W.erdos_renyi(60, 0.05, rng), W.band(7, 6)]
    ords = ["natural", "natural", "natural", "mindeg", "natural"]
    sb = B.SymbolicBatch(pats, orderings=ords)
    assert sb.count == len(pats)
    assert sb.nsuper == sum(B.Symbolic(*p, ordering=o).nsuper for p, o in zip(pats, ords))
    for i, (p, o) in enumerate(zip(pats, ords)):
        (ni, cp, ri), perm = sb.instance_pattern(i)
        s1 = B.Symbolic(*p, ordering=o)
        assert ni == s1.n
        assert (perm == s1.perm).all()
        assert (cp == s1.colptr).all() and (ri == s1.rowind).all()


# ---------------------------------------------------------------------------
# launch schedule: tasks and levels
# ---------------------------------------------------------------------------

SCHEDULE_CASES = {
    "band200_w8": lambda B, cr: B.Symbolic(*W.band(200, 8), chain_runs=cr),
    "band300_w40": lambda B, cr: B.Symbolic(*W.band(300, 40), chain_runs=cr),
    "band500_w70": lambda B, cr: B.Symbolic(*W.band(500, 70), chain_runs=cr),
    "arrow150_w48": lambda B, cr: B.Symbolic(*W.arrow(150, 48), chain_runs=cr),
    "grid20_nd": lambda B, cr: B.Symbolic(*W.permute(W.grid2d(20, 20), W.nested_dissection((20, 20), leaf=6)),
                                          chain_runs=cr),
    "er400_mindeg": lambda B, cr: B.Symbolic(*W.erdos_renyi(400, 0.02, np.random.default_rng(3)),
                                             ordering="mindeg", chain_runs=cr),
    "dense_tier_er": lambda B, cr: B.Symbolic(*W.erdos_renyi(300, 0.02, np.random.default_rng(5)),
                                              ordering="mindeg", relax=16, big_rows=40, big_cols=20,
                                              chain_runs=cr),
    "batch": lambda B, cr: B.SymbolicBatch([W.band(120, 6), W.grid2d(8, 8), W.band(90, 30)],
                                           chain_runs=cr),
}


@pytest.mark.parametrize("chain", [False, True])
@pytest.mark.parametrize("name", list(SCHEDULE_CASES))
def test_schedule_invariants(name, chain):
    """Every front in exactly one task (a leaf group through its first
    member); children before parents inside a task; a task only depends on
    tasks of lower levels; chain runs (only with the option) are runs of
    one-column fronts with contiguous rows, one a, 1 <= a <= 64, each the
    only child of the next, starting at a leaf."""
    B = lib()
    sym = SCHEDULE_CASES[name](B, chain)
    sp, par, rp, rows = sym.supernodes()
    nsn = len(sp) - 1
    d = sym.schedule()
    lp, lc, tp, tf = d["lvl_ptr"], d["lvl_counts"], d["task_ptr"], d["task_fronts"]
    assert len(set(tf.tolist())) == len(tf)
    task_of = np.full(nsn, -1, np.int64)
    for q in range(len(tp) - 1):
        task_of[tf[tp[q]:tp[q + 1]]] = q
    # fronts outside the lists: members of a leaf group, after their first
    # member (one-column leaves of one parent with the same A)
    A_of = lambda k: rows[rp[k] + (sp[k + 1] - sp[k]):rp[k + 1]].tolist()
    for k in range(nsn):
        if task_of[k] < 0:
            g0 = k - 1
            while task_of[g0] < 0:
                g0 -= 1
            for g in range(g0, k + 1):
                assert sp[g + 1] - sp[g] == 1 and par[g] == par[k] and A_of(g) == A_of(k)
            task_of[k] = task_of[g0]
    level_of = np.empty(len(tp) - 1, np.int64)
    for l in range(len(lp) - 1):
        level_of[lp[l]:lp[l + 1]] = l
    pos = np.full(nsn, -1, np.int64)
    pos[tf] = np.arange(len(tf))
    nkids = np.zeros(nsn, np.int64)
    for k in range(nsn):
        if par[k] >= 0:
            nkids[par[k]] += 1
            if task_of[par[k]] == task_of[k]:
                assert pos[k] < pos[par[k]] or pos[k] < 0
            else:
                assert level_of[task_of[k]] < level_of[task_of[par[k]]]
    nrun = 0
    for l in range(len(lp) - 1):
        r32, r64, warp, w64, big = lc[l]
        assert r32 + r64 + warp + w64 + big <= lp[l + 1] - lp[l]
        if not chain:
            assert r32 == 0 and r64 == 0
        for i in range(r32 + r64):
            q = lp[l] + i
            fr = tf[tp[q]:tp[q + 1]]
            nrun += 1
            assert len(fr) >= 8 and np.array_equal(fr, np.arange(fr[0], fr[0] + len(fr)))
            a = int(rp[fr[0] + 1] - rp[fr[0]]) - 1
            assert 1 <= a <= 64 and ((a + 1 <= 32) == (i < r32))
            assert nkids[fr[0]] == 0
            for j, k in enumerate(fr):
                assert sp[k + 1] - sp[k] == 1
                J = rows[rp[k]:rp[k + 1]]
                assert np.array_equal(J, np.arange(sp[k], sp[k] + a + 1))
                if j + 1 < len(fr):
                    assert par[k] == k + 1
                if j > 0:
                    assert nkids[k] == 1
    if chain and name in ("band200_w8", "band300_w40"):
        assert nrun >= 1  # the band chains are found (a <= 64)
    if name == "band500_w70":
        assert nrun == 0  # a = 70 > 64: no chain tier


def _pairs_of(colptr, rowind):
    cols = np.repeat(np.arange(len(colptr) - 1), np.diff(colptr))
    return set(zip(np.asarray(rowind).astype(int).tolist(), cols.tolist()))


@pytest.mark.parametrize("name", list(CASES))
def test_supernodal_pattern_of_fundamental_partition(name):
    """The oracle's supernodal pattern of Algorithm 6.1's partition of a
    filled pattern is that pattern (§6.2: the columns of a supernode share
    the ancestor set of its last column)."""
    mk, ordering, permf = CASES[name]
    pattern = mk()
    n = pattern[0]
    perm = permf() if permf else np.arange(n)
    p2 = W.permute(pattern, perm)
    I, parent = OS.fill(n, OS.columns_from_csc(*p2))
    N, A, par, _ = OS.clique_tree_alg61(I, parent, tie="last")
    # Algorithm 6.1's supernodes are contiguous only after a postorder; take
    # the chain-contiguous ones of this order (columns k, k+1, .. each the
    # only chain child of the next) by splitting at every break
    sp = [0]
    for j in range(1, n):
        same = any(j in set(Nk) and (j - 1) in set(Nk) for Nk in N.values())
        if not same:
            sp.append(j)
    sp.append(n)
    cp, ri = OS.supernodal_pattern(n, I, sp)
    want = {(int(r), k) for k in range(n) for r in I[k]} | {(k, k) for k in range(n)}
    assert _pairs_of(cp, ri) == want


def test_supernodal_pattern_of_merged_partition():
    """Merging a chain of the elimination tree into one supernode: every
    merged column gets the rows below it inside the supernode and the
    ancestor set of the last column; the result contains V and is filled
    (Eq. (e-filled)); the added entries are exactly the explicit zeros."""
    # arrow with a band: columns 0..5 form chains with different structures
    n, cp0, ri0 = W.band(12, 2)
    I, parent = OS.fill(n, OS.columns_from_csc(n, cp0, ri0))
    sp = [0, 4, 8, 12]  # supernodes {0..3}, {4..7}, {8..11}
    cp, ri = OS.supernodal_pattern(n, I, sp)
    got = _pairs_of(cp, ri)
    # by hand: column j of [f, l) holds rows j..l-1 and I_{l-1} = {l, l+1} (l < 12)
    want = set()
    for f, l in ((0, 4), (4, 8), (8, 12)):
        for j in range(f, l):
            want |= {(r, j) for r in range(j, l)} | {(r, j) for r in (l, l + 1) if r < n}
    assert got == want
    assert _pairs_of(cp0, ri0) <= got
    cols = [np.asarray(ri[cp[k] + 1:cp[k + 1]], dtype=np.int64) for k in range(n)]
    assert OS.is_filled(n, cols)
    # the band of half-bandwidth 2 with these blocks has no added entry in the
    # first two columns of each block and one per block in column f+2 .. :
    extra = got - _pairs_of(cp0, ri0)
    assert extra == {(3, 0), (7, 4), (11, 8)} | {(r, j) for (f, l) in ((0, 4), (4, 8)) for j in range(f, l)
                                                  for r in (l, l + 1) if r - j > 2}


def test_stored_er5000_analysis():
    """The stored analysis of the Erdos-Renyi workload (used by the CPU
    oracle's timing arm, which does not load the library) is what the
    library's minimum-degree ordering and relaxed supernodes give, and the
    oracle's fill and supernodal pattern of it equal the library's V."""
    from workloads import analysed
    B = lib()
    pattern, perm, sp = analysed.load_er5000()
    sym = B.Symbolic(*pattern, ordering="mindeg", relax=16, split_cols=-1)
    assert np.array_equal(np.asarray(sym.perm, dtype=np.int64), perm)
    assert np.array_equal(np.asarray(sym.supernodes()[0], dtype=np.int64), sp)
    n, cp, ri = W.permute(pattern, perm)
    I, _ = OS.fill(n, OS.columns_from_csc(n, cp, ri))
    vcp, vri = OS.supernodal_pattern(n, I, sp)
    assert np.array_equal(vcp, sym.colptr) and np.array_equal(vri, sym.rowind)
    # the split partition the benchmark may choose has the same pattern
    sym2 = B.Symbolic(*pattern, ordering="mindeg", relax=16, split_cols=512)
    assert np.array_equal(sym2.colptr, sym.colptr) and np.array_equal(sym2.rowind, sym.rowind)


def test_tier_table_assigns_tiers_by_front_shape():
    """chd_opts.tier_table: all -1 reproduces the threshold rule; 1 in every
    bucket sends every front to the dense tier, 0 none; a single bucket
    moves exactly the fronts of that (n_k, a_k) bucket."""
    B = lib()
    pat = W.erdos_renyi(600, 0.01, np.random.default_rng(65))
    kw = dict(ordering="mindeg", relax=8, big_rows=64, big_cols=32)
    dense = lambda sym: int(sym.schedule()["lvl_counts"][:, 4].sum())
    base = B.Symbolic(*pat, **kw)
    nb = B.TIER_BUCKETS
    assert dense(B.Symbolic(*pat, **kw, tier_table=-np.ones((nb, nb), np.int32))) == dense(base)
    assert dense(B.Symbolic(*pat, **kw, tier_table=np.ones((nb, nb), np.int32))) == base.nsuper
    assert dense(B.Symbolic(*pat, **kw, tier_table=np.zeros((nb, nb), np.int32))) == 0
    sp, par, rp, rows = base.supernodes()
    n = np.diff(sp)
    a = np.diff(rp) - n
    J = n + a
    is_dense = (J >= 64) | (n >= 32)
    keys = [(B.tier_bucket(x), B.tier_bucket(y)) for x, y in zip(n, a)]
    k = next(key for key, d in zip(keys, is_dense) if d)  # a bucket holding a dense front
    t = -np.ones((nb, nb), np.int32)
    t[k] = 0
    moved = sum(1 for key, d in zip(keys, is_dense) if d and key == k)
    assert dense(B.Symbolic(*pat, **kw, tier_table=t)) == dense(base) - moved


# ---------------------------------------------------------------------------
# geometric nested dissection inside the analysis
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,leaf", [((9, 9), 8), ((14, 14), 6), ((7, 3, 4), 8), ((5, 5, 5), 8),
                                       ((1, 30), 4), ((150, 150), 8)])
def test_nested_dissection_ordering_in_analysis(dims, leaf):
    """ordering="nd_geometric" gives the same analysis (perm, filled pattern,
    supernodes) as the input generator's nested-dissection permutation
    handed over as a user ordering: two independent codings of one rule."""
    B = lib()
    pat = W.grid2d(*dims) if len(dims) == 2 else W.grid3d(*dims)
    s1 = B.Symbolic(*pat, ordering="nd_geometric", nd_dims=dims, nd_leaf=leaf)
    s2 = B.Symbolic(*pat, perm=W.nested_dissection(dims, leaf=leaf))
    assert (s1.perm == s2.perm).all()
    assert (s1.colptr == s2.colptr).all() and (s1.rowind == s2.rowind).all()
    for x, y in zip(s1.supernodes(), s2.supernodes()):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_nested_dissection_separators_and_fill():
    """On a k x k grid the top separator (the middle column, k vertices) is
    eliminated last and lies in the root clique (Algorithm 6.1 joins one
    half's separator to it: their columns have |I| one apart), and the fill
    stays O(n log n): far below the natural order's band fill of about n k."""
    B = lib()
    k = 63
    pat = W.grid2d(k, k)
    s = B.Symbolic(*pat, ordering="nd_geometric", nd_dims=(k, k))
    assert sorted((np.asarray(s.perm[-k:]) % k).tolist()) == [k // 2] * k
    sp, par, rp, rows = s.supernodes()
    root = int(np.flatnonzero(np.asarray(par) < 0)[0])
    assert sp[root + 1] == k * k and sp[root + 1] - sp[root] == k + k // 2  # + a half's separator row
    assert rp[root + 1] - rp[root] == sp[root + 1] - sp[root]
    nat = B.Symbolic(*pat)
    assert s.nnz < 0.4 * nat.nnz
    assert s.nnz < 2 * k * k * np.log2(k * k)


def test_nested_dissection_rejects_wrong_dimensions():
    B = lib()
    with pytest.raises(B.ChdError):
        B.Symbolic(*W.grid2d(6, 6), ordering="nd_geometric", nd_dims=(6, 5))
    with pytest.raises(B.ChdError):
        B.Symbolic(*W.grid2d(6, 6), ordering="nd_geometric", nd_dims=(36, 0, 1))


def test_batch_with_nested_dissection_orderings():
    """Per-instance ordering options in a batch analysis."""
    B = lib()
    pats = [W.grid2d(12, 12), W.band(40, 3), W.grid3d(4, 5, 3)]
    ords = [{"ordering": "nd_geometric", "nd_dims": (12, 12), "nd_leaf": 6}, "natural",
            {"ordering": "nd_geometric", "nd_dims": (4, 5, 3)}]
    sb = B.SymbolicBatch(pats, orderings=ords)
    perms = [W.nested_dissection((12, 12), leaf=6), None, W.nested_dissection((4, 5, 3), leaf=8)]
    for i, (p, q) in enumerate(zip(pats, perms)):
        (ni, cp, ri), perm = sb.instance_pattern(i)
        s1 = B.Symbolic(*p, perm=q)
        assert (perm == s1.perm).all() and (cp == s1.colptr).all() and (ri == s1.rowind).all()


def test_factored_completion_plan_flops():
    """The factored completion's propagation work (Algorithm 4.3: one
    reflection per kept row whose columns were mixed, then the rows of A_k in
    N_parent) against the independent Cholesky of every V_k (a^3 / 3).  On a
    band each front drops one row of its parent's factor: the reflections
    cost O(a^2) per front, less than a^3 / 3 once a is large (w = 40), more
    for a narrow band (w = 8, where the per-row constant dominates).  Split
    supernodes delete no rows: only the N_parent block remains."""
    B = lib()
    f40 = B.Symbolic(*W.band(300, 40), completion="factored").completion_flops()
    assert 0 < f40["factored"] < 0.5 * f40["independent"]
    # independent: 259 one-column fronts with a = 40 below the root (its 41 columns, a = 0)
    assert f40["independent"] == pytest.approx(259 * 40 ** 3 / 3)
    f8 = B.Symbolic(*W.band(300, 8), completion="factored").completion_flops()
    assert f8["factored"] > f8["independent"]
    # a band propagates along one chain: one level per front below the root
    assert f40["levels"] == 259
    fs = B.Symbolic(*W.band(150, 149), big_rows=64, big_cols=64, split_cols=24,
                    completion="factored").completion_flops()
    assert fs["factored"] < fs["independent"]


# ---------------------------------------------------------------------------
# the factored completion's plan: what its kernels index, checked on the host
# ---------------------------------------------------------------------------

PLAN_CASES = {
    "er5000": lambda B: B.Symbolic(*_er5000_pattern(), big_rows=192, big_cols=96, split_cols=512),
    "grid150": lambda B: B.Symbolic(*W.grid2d(150, 150), **W.nd_options((150, 150))),
    "grid3d_12": lambda B: B.Symbolic(*W.grid3d(12, 12, 12), **W.nd_options((12, 12, 12)), big_rows=64, big_cols=32),
    "arrow_groups": lambda B: B.Symbolic(*W.arrow(300, 40)),
    "split_dense": lambda B: B.Symbolic(*W.band(700, 699), split_cols=256),
    "band": lambda B: B.Symbolic(*W.band(400, 20)),
    "batch": lambda B: B.SymbolicBatch([W.band(120, 6), W.grid2d(14, 14), W.arrow(90, 30)]),
}


def _er5000_pattern():
    from workloads import analysed
    pattern, perm, sp = analysed.load_er5000()
    n, cp, ri = pattern
    return n, cp, ri


@pytest.mark.parametrize("name", list(PLAN_CASES))
def test_factored_completion_plan_layout(name):
    """Every front with ancestors (a leaf group through its first member) is
    planned once, after its parent's level; q_k (rows of A_k in A_parent)
    and the gather width w_k recomputed from the clique tree give each
    front's scratch need, and the ranges of one level neither overlap nor
    pass the level scratch (fc_total); the kernels' parent rows
    rho = J_p - 1 - pos stay inside the parent's a_p x a_p factor."""
    B = lib()
    sym = PLAN_CASES[name](B)
    sp, par, rp, rows = [np.asarray(v) for v in sym.supernodes()]
    nsn = len(sp) - 1
    plan = sym.completion_plan()
    tf = sym.schedule()["task_fronts"]
    member = np.ones(nsn, dtype=bool)
    member[tf] = False  # fronts outside the task lists: leaf-group members after the first
    level = np.full(nsn, -1)
    big = np.zeros(nsn, dtype=bool)
    lv, fr, blv, bg = plan["fc_lvl"], plan["fc_fronts"], plan["fc_big_lvl"], plan["fc_big"]
    for l in range(len(lv) - 1):
        for k in fr[lv[l]:lv[l + 1]]:
            assert level[k] < 0
            level[k] = l
        for k in bg[blv[l]:blv[l + 1]]:
            assert level[k] < 0
            level[k], big[k] = l, True
    used = {}
    for k in range(nsn):
        n_k = sp[k + 1] - sp[k]
        a = rp[k + 1] - rp[k] - n_k
        if a == 0 or member[k]:
            assert level[k] < 0
            continue
        assert level[k] >= 0, k
        p = par[k]
        a_p = rp[p + 1] - rp[p] - (sp[p + 1] - sp[p])
        if a_p > 0 and not member[p]:
            assert level[p] < level[k]
        Jk, Jp = rows[rp[k]:rp[k + 1]], rows[rp[p]:rp[p + 1]]
        pos = np.searchsorted(Jp, Jk[n_k:])
        assert np.array_equal(Jp[pos], Jk[n_k:])  # A_k inside J_p
        n_p = sp[p + 1] - sp[p]
        q = int((pos >= n_p).sum())
        w = len(Jp) - pos[a - q] if q else 0
        if q:
            rho = len(Jp) - 1 - pos[a - 1 - np.arange(q)]
            assert rho.min() >= 0 and rho.max() < a_p and w == rho.max() + 1
            assert np.all(np.diff(rho) > 0)
        need = (q * w + 3) // 4 * 4 + (32 * (2 * w + q + 32) if big[k] and q else 0)
        if a > 256:
            assert big[k]
        used.setdefault(level[k], []).append((int(plan["fc_off"][k]), need))
    for l, ranges in used.items():
        ranges.sort()
        for (o1, n1), (o2, _) in zip(ranges, ranges[1:]):
            assert o1 + n1 <= o2
        o, n_ = ranges[-1]
        assert o + n_ <= plan["fc_total"]


@pytest.mark.parametrize("name", list(PLAN_CASES))
def test_front_regions_hold_what_the_kernels_index(name):
    """Front k's workspace region holds its J x J front and two J x n
    temporaries, its D_NN block n x n and its V_k block a x a (a leaf
    group's members share the first member's, and the group's scratch --
    V and an a x L block of the members -- fits in the members' regions)."""
    B = lib()
    sym = PLAN_CASES[name](B)
    sp, par, rp, rows = [np.asarray(v) for v in sym.supernodes()]
    nsn = len(sp) - 1
    f_off, d_off, v_off = sym.offsets()
    n = np.diff(sp)
    J = np.diff(rp)
    a = J - n
    assert np.all(np.diff(f_off) >= J * J + 2 * J * n)
    assert np.all(np.diff(d_off) >= n * n)
    tf = sym.schedule()["task_fronts"]
    member = np.ones(nsn, dtype=bool)
    member[tf] = False
    dv = np.diff(v_off)
    assert np.all(dv[~member] >= (a * a)[~member])
    k = 0
    while k < nsn:
        if k + 1 < nsn and member[k + 1]:
            c0, L = k, 1
            while k + L < nsn and member[k + L]:
                L += 1
            assert np.all(n[c0:c0 + L] == 1) and np.all(a[c0:c0 + L] == a[c0])
            assert np.all(v_off[c0 + 1:c0 + L + 1] == v_off[c0 + 1])  # one shared V slot
            aa = int(a[c0])
            assert aa * aa + aa * L <= f_off[c0 + L] - f_off[c0 + 1]
            k += L
        else:
            k += 1
