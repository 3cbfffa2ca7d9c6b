"""GPU parity: every operation of the library against the FP64 oracle.

Inputs are seeded and synthetic; the pattern V is produced by chd_analyze
and validated against the oracle's own fill before any value is drawn on it.
Tolerance (relative Frobenius error in the symmetric norm, off-diagonals
counted twice): 1e-10 on well-conditioned inputs, 1e-8 at condition ~1e6.
"""
import numpy as np
import pytest

from oracle import dense as OD
from oracle import symbolic as OS
import workloads as W
from tests.helpers import lib

pytestmark = pytest.mark.gpu

TOL = 1e-10


def torch():
    import torch as t
    return t


class Case:
    def __init__(self, pattern, ordering="natural", perm=None, relax=0, seed=0, x=None, big=None, split=0, tc=0,
                 **extra):
        self.B = lib()
        kw = dict(extra) if big is None else dict(extra, big_rows=big[0], big_cols=big[1])
        kw["split_cols"] = split
        kw["tc_products"] = tc
        self.sym = self.B.Symbolic(*pattern, ordering=ordering, perm=perm, relax=relax, **kw)
        s = self.sym
        self.n, self.cp, self.ri = s.n, s.colptr, s.rowind
        # V must be filled (Eq. (e-filled)) and contain the permuted input pattern
        I = [s.rowind[s.colptr[k] + 1:s.colptr[k + 1]] for k in range(s.n)]
        assert OS.is_filled(s.n, I)
        rng = np.random.default_rng(seed)
        self.x = W.diag_dominant(s.n, s.colptr, s.rowind, rng) if x is None else x(s, rng)
        self.rng = rng

    def dev(self, a):
        t = torch()
        return t.as_tensor(np.ascontiguousarray(a), dtype=t.float64, device="cuda")

    def host(self, t_):
        torch().cuda.synchronize()
        return t_.cpu().numpy()

    def err(self, a, ref):
        return OD.rel_err(self.n, self.cp, self.ri, a, ref)


def small_cases(**extra):
    """The parity cases; `extra` analysis options go to every one."""
    return {
        "band200_w8": lambda: Case(W.band(200, 8), seed=0, **extra),
        "band40_w1": lambda: Case(W.band(40, 1), seed=1, **extra),
        "arrow60_w7": lambda: Case(W.arrow(60, 7), seed=2, **extra),
        "grid14_nd": lambda: Case(W.grid2d(14, 14), ordering="user",
                                  perm=W.nested_dissection((14, 14), leaf=6), seed=3, **extra),
        "grid3d_5": lambda: Case(W.grid3d(5, 5, 5), ordering="user",
                                 perm=W.nested_dissection((5, 5, 5), leaf=8), seed=4, **extra),
        "er300_mindeg_relax16": lambda: Case(W.erdos_renyi(300, 0.02, np.random.default_rng(5)),
                                             ordering="mindeg", relax=16, seed=5, **extra),
        "dense70": lambda: Case(W.band(70, 69), seed=6, **extra),
        "diag30": lambda: Case(W.band(30, 0), seed=7, **extra),
        "wide_front": lambda: Case(W.arrow(200, 120), seed=8, **extra),
        # the same kinds of pattern with low thresholds, so that many fronts run
        # through the multi-CTA dense tier and hand over to and from the per-task tier
        "dense_tier_grid": lambda: Case(W.grid2d(16, 16), ordering="user",
                                        perm=W.nested_dissection((16, 16), leaf=6), seed=9, **extra, big=(20, 8)),
        "dense_tier_er": lambda: Case(W.erdos_renyi(300, 0.02, np.random.default_rng(5)),
                                      ordering="mindeg", relax=16, seed=10, **extra, big=(40, 20)),
        "dense_tier_full": lambda: Case(W.band(150, 149), seed=11, **extra, big=(64, 64)),
        "dense_tier_arrow": lambda: Case(W.arrow(260, 100), seed=12, **extra, big=(90, 70)),
        # wide supernodes split into chains (dense, CTA and warp pieces)
        "split_dense": lambda: Case(W.band(150, 149), seed=13, **extra, big=(64, 64), split=24),
        "split_arrow": lambda: Case(W.arrow(200, 90), seed=14, **extra, split=8),
        # wide warp tier (|N| <= 8, 32 < |J| <= 64, chains only): two chains
        # handing over to the CTA tier at the root, and thin leaves of one parent
        # (CTA tier)
        "band300_w40": lambda: Case(W.band(300, 40), seed=15, **extra),
        "arrow150_w48": lambda: Case(W.arrow(150, 48), seed=16, **extra),
        "band120_w63": lambda: Case(W.band(120, 63), seed=17, **extra),
        # every dense-tier product with at least 64 x 16 outputs on the tensor
        # cores (FP64-accurate digit products), on the dense-tier cases above
        "tc_dense_grid": lambda: Case(W.grid2d(16, 16), ordering="user",
                                      perm=W.nested_dissection((16, 16), leaf=6), seed=9, **extra, big=(20, 8), tc=1),
        "tc_dense_er": lambda: Case(W.erdos_renyi(300, 0.02, np.random.default_rng(5)),
                                    ordering="mindeg", relax=16, seed=10, **extra, big=(40, 20), tc=1),
        "tc_dense_full": lambda: Case(W.band(150, 149), seed=11, **extra, big=(64, 64), tc=1),
        "tc_dense_arrow": lambda: Case(W.arrow(260, 100), seed=12, **extra, big=(90, 70), tc=1),
        "tc_split_dense": lambda: Case(W.band(150, 149), seed=13, **extra, big=(64, 64), split=24, tc=1),
        "tc_wide_arrow": lambda: Case(W.arrow(400, 330), seed=18, **extra, tc=1),
    }


CASES = small_cases()


@pytest.mark.parametrize("name", list(CASES))
def test_factor_logdet(name):
    c = CASES[name]()
    f = c.sym.factor(c.dev(c.x))
    ld = f.logdet()
    assert f.status() == 0
    l, d = f.export()
    lv, dv, _ = OD.factor(c.n, c.cp, c.ri, c.x)
    want_ld = OD.logdet(c.n, c.cp, c.ri, c.x)
    assert abs(ld - want_ld) <= TOL * max(1.0, abs(want_ld))
    np.testing.assert_allclose(c.host(d), dv, rtol=1e-11)
    assert c.err(c.host(l), lv) < TOL


@pytest.mark.parametrize("name", list(CASES))
def test_gradient(name):
    c = CASES[name]()
    f = c.sym.factor(c.dev(c.x))
    g = c.host(f.gradient())
    assert c.err(g, OD.gradient(c.n, c.cp, c.ri, c.x)) < TOL


@pytest.mark.parametrize("name", list(CASES))
def test_hessian(name):
    c = CASES[name]()
    f = c.sym.factor(c.dev(c.x))
    ys = W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=3)
    t = c.host(f.hessian(c.dev(ys)))
    want = OD.hessian(c.n, c.cp, c.ri, c.x, list(ys))
    for i in range(3):
        assert c.err(t[i], want[i]) < TOL


@pytest.mark.parametrize("name", list(CASES))
def test_inverse_hessian(name):
    c = CASES[name]()
    f = c.sym.factor(c.dev(c.x))
    ts = W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=2)
    y = c.host(f.inv_hessian(c.dev(ts)))
    Z = OD.inverse(c.n, c.cp, c.ri, c.x)
    for i in range(2):
        if len(c.ri) <= 2500:
            want = OD.inv_hessian_dense(c.n, c.cp, c.ri, c.x, [ts[i]], Z=Z)[0]
        else:
            I, parent = OS.fill(c.n, OS.columns_from_csc(c.n, c.cp, c.ri))
            cl, seps = OS.cliques_and_separators(I, parent)
            want = OD.inv_hessian_cliquesum(c.n, c.cp, c.ri, c.x, ts[i], cl, seps, S=Z)
        assert c.err(y[i], want) < TOL


@pytest.mark.parametrize("name", list(CASES))
def test_completion(name):
    c = CASES[name]()
    G = c.rng.standard_normal((c.n, 10))
    s = W.projected_gram(c.n, c.cp, c.ri, G, 0.5)
    fx, fstar = c.sym.complete(c.dev(s))
    assert fx.status() == 0
    I, parent = OS.fill(c.n, OS.columns_from_csc(c.n, c.cp, c.ri))
    cl, seps = OS.cliques_and_separators(I, parent)
    xh = OD.completion_refined(c.n, c.cp, c.ri, s, cl, seps)
    lv, dv, _ = OD.factor(c.n, c.cp, c.ri, xh)
    l, d = fx.export()
    np.testing.assert_allclose(c.host(d), dv, rtol=1e-10)
    assert c.err(c.host(l), lv) < TOL
    want_fs = OD.dual_barrier(c.n, c.cp, c.ri, xh)
    assert abs(fstar - want_fs) <= TOL * max(1.0, abs(want_fs))
    # the completion factor serves the dual barrier's Hessian (Eq. (e-legendre-rels)):
    # grad^2 f_*(S)[T] = H_{Xhat}^{-1}(T)
    t = W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=1)
    yh = c.host(fx.inv_hessian(c.dev(t)))[0]
    Sd = OD.to_dense(c.n, c.cp, c.ri, s)
    want = OD.inv_hessian_cliquesum(c.n, c.cp, c.ri, xh, t[0], cl, seps, S=Sd)
    assert c.err(yh, want) < 1e-9


@pytest.mark.parametrize("name", list(CASES))
def test_cholesky_product(name):
    """Algorithm 3.2: L D L^T on V from a factor object is X; from a completion
    object it is X-hat, whose negative is the dual gradient (§1.2)."""
    c = CASES[name]()
    f = c.sym.factor(c.dev(c.x))
    assert c.err(c.host(f.product()), c.x) < 1e-12
    G = c.rng.standard_normal((c.n, 10))
    s = W.projected_gram(c.n, c.cp, c.ri, G, 0.5)
    fx, _ = c.sym.complete(c.dev(s))
    I, parent = OS.fill(c.n, OS.columns_from_csc(c.n, c.cp, c.ri))
    cl, seps = OS.cliques_and_separators(I, parent)
    xh = OD.completion_cliquesum(c.n, c.cp, c.ri, s, cl, seps)
    assert c.err(c.host(fx.product()), xh) < TOL


@pytest.mark.parametrize("name", list(CASES))
def test_hessian_factor(name):
    """W = R(Y) (Algorithm 5.3, R_j upper) and T = R^adj(W) (Algorithm 5.4)
    against the oracle's per-column definitions; R^adj(R(Y)) = H(Y)."""
    c = CASES[name]()
    f = c.sym.factor(c.dev(c.x))
    ys = W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=3)
    ws = W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=2)
    parts = OD.hessian_factor_parts(c.n, c.cp, c.ri, c.x)
    w = f.hessian_factor(c.dev(ys))
    want_w = OD.hessian_factor(c.n, c.cp, c.ri, c.x, list(ys), parts=parts)
    wh = c.host(w)
    for i in range(3):
        assert c.err(wh[i], want_w[i]) < TOL
    # R^adj o R = H, computed in place
    t = c.host(f.hessian_factor_adj(w, out=w))
    want_t = OD.hessian(c.n, c.cp, c.ri, c.x, list(ys))
    for i in range(3):
        assert c.err(t[i], want_t[i]) < TOL
    # R^adj of unrelated W, out of place
    ta = c.host(f.hessian_factor_adj(c.dev(ws)))
    want_a = OD.hessian_factor_adj(c.n, c.cp, c.ri, c.x, list(ws), parts=parts)
    for i in range(2):
        assert c.err(ta[i], want_a[i]) < TOL


def _figure_case(case, big):
    """Figure 1's pattern in the library's order (a postorder of the same
    elimination tree: the factors, the ordered sets I_j and so R(Y) only get
    permuted), Y with the figure's nonzero, and the map of W's nonzeros back
    to the figure's numbering."""
    from tests.test_oracle_dense import fig_spy_w
    pattern, cases = fig_spy_w()
    c = Case(pattern, seed=97, big=big)
    perm = np.asarray(c.sym.perm)  # perm[new] = old
    rr, cc = OD.pattern_pairs(c.n, c.cp, c.ri)
    orr, occ = np.maximum(perm[rr], perm[cc]), np.minimum(perm[rr], perm[cc])
    y = np.where((orr == cases[case]["y"][0]) & (occ == cases[case]["y"][1]), 1.0, 0.0)
    assert y.sum() == 1.0

    def spy_orig(w):
        big_ = np.abs(w) > 1e-12 * np.abs(w).max()
        return {(int(a), int(b)) for a, b, t in zip(orr, occ, big_) if t}
    return c, y, spy_orig, cases[case]["w"]


@pytest.mark.parametrize("case", ["a", "b"])
@pytest.mark.parametrize("big", [None, (4, 2)])
def test_hessian_factor_sparsity_of_figure(case, big):
    """Figure fig-spy-W (§5.5): the nonzeros of R(Y) on Figure 1's pattern for
    a Y with one nonzero, through the per-task tiers and through the dense
    tier (low thresholds)."""
    c, y, spy_orig, want = _figure_case(case, big)
    f = c.sym.factor(c.dev(c.x))
    w = c.host(f.hessian_factor(c.dev(y)))
    assert spy_orig(w) == want
    assert c.err(w, OD.hessian_factor(c.n, c.cp, c.ri, c.x, [y])[0]) < TOL


def sparse_args(c, count, k, rng):
    """`count` matrices on V with `k` nonzero lower entries each at random
    positions (the sparse arguments of §5.5), values uniform[-1, 1]."""
    nnz = len(c.ri)
    out = np.zeros((count, nnz))
    for i in range(count):
        pos = rng.choice(nnz, size=min(k, nnz), replace=False)
        out[i, pos] = rng.uniform(-1.0, 1.0, size=len(pos))
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_hessian_factor_sparse_arguments(name):
    """R(Y) with the clique tree pruned per Y (§5.5) equals the oracle's R(Y)
    for Y with two nonzeros (the paper's experiment), a dense Y and Y = 0,
    in one batch."""
    c = CASES[name]()
    f = c.sym.factor(c.dev(c.x))
    ys = np.concatenate([sparse_args(c, 4, 2, c.rng), W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=1),
                         np.zeros((1, len(c.ri)))])
    wp = c.host(f.hessian_factor(c.dev(ys), sparse=True))
    want = OD.hessian_factor(c.n, c.cp, c.ri, c.x, list(ys[:5]))
    for i in range(5):
        assert c.err(wp[i], want[i]) < TOL
    assert not np.any(wp[5])  # Y = 0: every front pruned, W = 0 exactly
    # the pruned and the full computation agree on the same batch
    wf = c.host(f.hessian_factor(c.dev(ys)))
    for i in range(6):
        assert c.err(wp[i], wf[i]) < 1e-13 or not np.any(wf[i])


@pytest.mark.parametrize("case", ["a", "b"])
def test_hessian_factor_sparse_figure(case):
    """Figure fig-spy-W through the pruned path."""
    c, y, spy_orig, want = _figure_case(case, None)
    f = c.sym.factor(c.dev(c.x))
    w = c.host(f.hessian_factor(c.dev(y), sparse=True))
    assert spy_orig(w) == want
    assert c.err(w, OD.hessian_factor(c.n, c.cp, c.ri, c.x, [y])[0]) < TOL


@pytest.mark.parametrize("name", ["grid14_nd", "dense_tier_er", "arrow150_w48", "wide_front"])
def test_schur_by_hessian_factor(name):
    """H_ij = R(A_i) . R(A_j) (§5.4) equals A_i . H(A_j)."""
    c = CASES[name]()
    m = 6
    A = W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=m)
    f = c.sym.factor(c.dev(c.x))
    R = c.host(f.hessian_factor(c.dev(A)))
    got = np.array([[OD.sym_dot(c.n, c.cp, c.ri, R[i], R[j]) for j in range(m)] for i in range(m)])
    Th = OD.hessian(c.n, c.cp, c.ri, c.x, list(A))
    want = np.array([[OD.sym_dot(c.n, c.cp, c.ri, A[i], Th[j]) for j in range(m)] for i in range(m)])
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("name", ["grid14_nd", "er300_mindeg_relax16", "dense_tier_er", "arrow150_w48"])
def test_schur_complement(name):
    """H_ij = A_i . H(A_j) (§5.5) against the oracle's Hessian and inner product."""
    c = CASES[name]()
    m = 5
    A = W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=m)
    f = c.sym.factor(c.dev(c.x))
    H, T = f.schur(c.dev(A))
    H = c.host(H)
    Th = OD.hessian(c.n, c.cp, c.ri, c.x, list(A))
    want = np.array([[OD.sym_dot(c.n, c.cp, c.ri, A[i], Th[j]) for j in range(m)] for i in range(m)])
    assert np.abs(H - want).max() <= 1e-10 * np.abs(want).max()
    assert np.abs(H - H.T).max() <= 1e-10 * np.abs(want).max()
    assert np.linalg.eigvalsh(0.5 * (H + H.T)).min() > 0  # H is positive definite


CHAIN_CASES = {
    "band200_w8": lambda: W.band(200, 8),      # |J| = 9: one run of 191 fronts
    "band300_w40": lambda: W.band(300, 40),    # |J| = 41
    "band120_w63": lambda: W.band(120, 63),    # |J| = 64, the largest window
    "band90_w1": lambda: W.band(90, 1),        # a = 1
}


@pytest.mark.parametrize("name", list(CHAIN_CASES))
def test_chain_runs(name):
    """The chain tier (sliding windows along runs of one-column band fronts)
    against the oracle, and against the same pattern without the option:
    factor, log det, gradient, Hessian, inverse Hessian, product, Hessian
    factor (plain and pruned) and its adjoint."""
    B = lib()
    pattern = CHAIN_CASES[name]()
    rng = np.random.default_rng(41)
    on = B.Symbolic(*pattern, chain_runs=True)
    off = B.Symbolic(*pattern, chain_runs=False)
    assert np.array_equal(on.colptr, off.colptr) and np.array_equal(on.rowind, off.rowind)
    n, cp, ri = on.n, on.colptr, on.rowind
    x = W.diag_dominant(n, cp, ri, rng)
    ys = W.uniform_sym(n, cp, ri, rng, count=3)
    y2 = np.zeros_like(ys)
    for i in range(3):
        y2[i, rng.choice(len(ri), size=2, replace=False)] = rng.uniform(-1.0, 1.0, size=2)
    c = Case(pattern, seed=41)
    dev = c.dev
    res = {}
    for key, sym in (("on", on), ("off", off)):
        f = sym.factor(dev(x))
        l, d = f.export()
        res[key] = dict(logdet=f.logdet(), l=c.host(l), d=c.host(d), g=c.host(f.gradient()),
                        t=c.host(f.hessian(dev(ys))), yi=c.host(f.inv_hessian(dev(ys))), xp=c.host(f.product()),
                        w=c.host(f.hessian_factor(dev(ys))), w2=c.host(f.hessian_factor(dev(y2), sparse=True)),
                        ta=c.host(f.hessian_factor_adj(dev(ys))))
    err = lambda a, b: OD.rel_err(n, cp, ri, a, b)
    for key in ("g", "l", "xp"):
        assert err(res["on"][key], res["off"][key]) < 1e-12, key
    assert abs(res["on"]["logdet"] - res["off"]["logdet"]) <= 1e-12 * max(1.0, abs(res["off"]["logdet"]))
    for key in ("t", "yi", "w", "w2", "ta"):
        for i in range(3):
            assert err(res["on"][key][i], res["off"][key][i]) < 1e-11, key
    # and the oracle
    assert abs(res["on"]["logdet"] - OD.logdet(n, cp, ri, x)) <= 1e-10 * max(1.0, abs(OD.logdet(n, cp, ri, x)))
    assert err(res["on"]["g"], OD.gradient(n, cp, ri, x)) < TOL
    want = OD.hessian(n, cp, ri, x, list(ys))
    wantw = OD.hessian_factor(n, cp, ri, x, list(ys))
    for i in range(3):
        assert err(res["on"]["t"][i], want[i]) < TOL
        assert err(res["on"]["w"][i], wantw[i]) < TOL


@pytest.mark.parametrize("name", list(CHAIN_CASES))
def test_chain_runs_inverse_hessian(name):
    """The inverse Hessian's passes in the chain tier, against the oracle's
    dense solve and against the path without chain runs."""
    B = lib()
    pattern = CHAIN_CASES[name]()
    rng = np.random.default_rng(43)
    on = B.Symbolic(*pattern, chain_runs=True)
    off = B.Symbolic(*pattern, chain_runs=False)
    n, cp, ri = on.n, on.colptr, on.rowind
    x = W.diag_dominant(n, cp, ri, rng)
    ts = W.uniform_sym(n, cp, ri, rng, count=3)
    c = Case(pattern, seed=43)
    yi = {k: c.host(sym.factor(c.dev(x)).inv_hessian(c.dev(ts))) for k, sym in (("on", on), ("off", off))}
    want = OD.inv_hessian_dense(n, cp, ri, x, list(ts))
    for i in range(3):
        assert OD.rel_err(n, cp, ri, yi["on"][i], yi["off"][i]) < 1e-11
        assert OD.rel_err(n, cp, ri, yi["on"][i], want[i]) < TOL


def test_planted_condition_1e6():
    def planted(s, rng):
        x, _, _ = W.planted_factor(s.n, s.colptr, s.rowind, rng, dmin=1e-6, dmax=1.0)
        return x
    c = Case(W.band(150, 6), x=planted, seed=11)
    X = OD.to_dense(c.n, c.cp, c.ri, c.x)
    kappa = np.linalg.cond(X)
    assert kappa > 1e5
    f = c.sym.factor(c.dev(c.x))
    l, d = f.export()
    lv, dv, _ = OD.factor(c.n, c.cp, c.ri, c.x)
    assert c.err(c.host(l), lv) < 1e-8
    g = c.host(f.gradient())
    assert c.err(g, OD.gradient(c.n, c.cp, c.ri, c.x)) < 1e-8
    ys = W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=2)
    t = c.host(f.hessian(c.dev(ys)))
    want = OD.hessian(c.n, c.cp, c.ri, c.x, list(ys))
    for i in range(2):
        assert c.err(t[i], want[i]) < 1e-8


def test_not_positive_definite_is_reported():
    B = lib()
    c = Case(W.band(50, 3), seed=12)
    x = c.x.copy()
    x[c.cp[20]] = -5.0  # a negative diagonal entry: X is indefinite
    f = c.sym.factor(c.dev(x))
    assert f.status() == B.CHD_ERR_NOT_PD
    rc, snode, col = f.error_detail()
    assert rc == B.CHD_ERR_NOT_PD and 0 <= col <= 20


def test_not_completable_is_reported():
    B = lib()
    c = Case(W.band(40, 2), seed=13)
    s = -np.abs(W.diag_dominant(c.n, c.cp, c.ri, c.rng))  # negative diagonal: no PSD completion
    try:
        c.sym.complete(c.dev(s))
        raise AssertionError("expected CHD_ERR_NOT_COMPLETABLE")
    except B.ChdError as e:
        assert e.code == B.CHD_ERR_NOT_COMPLETABLE


def test_batched_rhs_strides_and_refactor():
    c = CASES["grid14_nd"]()
    f = c.sym.factor(c.dev(c.x))
    t_ = torch()
    m = 5
    ld = c.sym.nnz + 7
    ybuf = t_.zeros((m, ld), dtype=t_.float64, device="cuda")
    ys = W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=m)
    ybuf[:, :c.sym.nnz] = c.dev(ys)
    tbuf = t_.full((m, ld), 7.0, dtype=t_.float64, device="cuda")
    c.B.chd_hessian(f.handle, ybuf, tbuf, c.sym.nnz)
    out = c.host(tbuf)
    want = OD.hessian(c.n, c.cp, c.ri, c.x, list(ys))
    for i in range(m):
        assert c.err(out[i, :c.sym.nnz], want[i]) < TOL
        assert np.all(out[i, c.sym.nnz:] == 7.0)  # padding untouched
    # refactor with new values invalidates cached blocks
    x2 = W.diag_dominant(c.n, c.cp, c.ri, np.random.default_rng(99))
    f.refactor(c.dev(x2))
    g = c.host(f.gradient())
    assert c.err(g, OD.gradient(c.n, c.cp, c.ri, x2)) < TOL


def test_hessian_more_right_hand_sides_than_one_launch_indexes():
    """chd_hessian runs m > 65535 right-hand sides (more than one grid
    dimension indexes) in chunks: the same products as two separate calls."""
    c = Case(W.band(4, 1), seed=31)
    t_ = torch()
    f = c.sym.factor(c.dev(c.x))
    m = 65537
    ys = c.rng.uniform(-1.0, 1.0, size=(m, c.sym.nnz))
    Y = c.dev(ys)
    T = t_.empty_like(Y)
    c.B.chd_hessian(f.handle, Y, T, c.sym.nnz)
    T1 = t_.empty_like(Y[:65535])
    T2 = t_.empty_like(Y[65535:])
    c.B.chd_hessian(f.handle, Y[:65535].contiguous(), T1, c.sym.nnz)
    c.B.chd_hessian(f.handle, Y[65535:].contiguous(), T2, c.sym.nnz)
    both = c.host(t_.cat([T1, T2]))
    got = c.host(T)
    assert np.array_equal(got, both)
    want = OD.hessian(c.n, c.cp, c.ri, c.x, [ys[0], ys[-1]])
    assert c.err(got[0], want[0]) < TOL and c.err(got[-1], want[1]) < TOL
