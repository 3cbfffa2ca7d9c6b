"""The scalar multifrontal algorithms of the paper (Algorithms 3.1, 3.2,
4.1, 4.2, 5.1, 5.2, restated in ``oracle.multifrontal``) against the dense
definitions of ``oracle.dense``: two independent routes to the same
objects, so a mistake in either fails here.  The library's supernodal block
forms reduce to these algorithms for one-column supernodes."""
import numpy as np
import pytest

from oracle import dense as OD
from oracle import multifrontal as OM
from oracle import symbolic as OS
import workloads as W
from tests.test_oracle_dense import filled, random_chordal

PATTERNS = {
    "band": lambda: W.band(24, 3),
    "arrow": lambda: W.arrow(20, 4),
    "grid": lambda: filled(W.permute(W.grid2d(5, 5), W.nested_dissection((5, 5), leaf=4))),
    "random": lambda: random_chordal(7, n=22, p=0.15),
    "dense": lambda: W.band(8, 7),
    "diagonal": lambda: W.band(6, 0),
}


def _case(name, seed):
    n, cp, ri = PATTERNS[name]()
    rng = np.random.default_rng(seed)
    x = W.diag_dominant(n, cp, ri, rng)
    return n, cp, ri, x, rng


def _close(n, cp, ri, A, ref_vals, tol):
    return OD.rel_err(n, cp, ri, OD.project(n, cp, ri, A), ref_vals) < tol


@pytest.mark.parametrize("name", list(PATTERNS))
def test_cholesky_and_product(name):
    n, cp, ri, x, _ = _case(name, 1)
    L, D = OM.cholesky(n, cp, ri, x)
    lv, dv, _ = OD.factor(n, cp, ri, x)
    np.testing.assert_allclose(D, dv, rtol=1e-13)
    assert _close(n, cp, ri, L, lv, 1e-13)
    # the factor of a filled pattern has no fill outside V (Eq. (e-filled))
    Ld = L - np.eye(n)
    mask = OD.to_dense(n, cp, ri, np.ones(len(ri))) != 0
    assert np.all(Ld[~np.tril(mask)] == 0.0)
    X = OM.cholesky_product(n, cp, ri, L, D)
    assert _close(n, cp, ri, X, x, 1e-13)


@pytest.mark.parametrize("name", list(PATTERNS))
def test_projected_inverse(name):
    n, cp, ri, x, _ = _case(name, 2)
    L, D = OM.cholesky(n, cp, ri, x)
    S = OM.projected_inverse(n, cp, ri, L, D)
    assert _close(n, cp, ri, S, OD.projected_inverse(n, cp, ri, x), 1e-12)


@pytest.mark.parametrize("name", list(PATTERNS))
def test_completion(name):
    n, cp, ri, x, rng = _case(name, 3)
    s = W.projected_gram(n, cp, ri, rng.standard_normal((n, 4)), 0.5)
    L, D = OM.completion(n, cp, ri, s)
    Xh = L @ np.diag(D) @ L.T
    # P(X-hat^{-1}) = S (Eq. (e-Xhat-eq)), and X-hat is the refined closed form
    assert OD.rel_err(n, cp, ri, OD.project(n, cp, ri, np.linalg.inv(Xh)), s) < 1e-12
    I, parent = OS.fill(n, OS.columns_from_csc(n, cp, ri))
    cl, seps = OS.cliques_and_separators(I, parent)
    assert _close(n, cp, ri, Xh, OD.completion_refined(n, cp, ri, s, cl, seps), 1e-12)


@pytest.mark.parametrize("name", list(PATTERNS))
def test_hessian_and_inverse(name):
    n, cp, ri, x, rng = _case(name, 4)
    L, D = OM.cholesky(n, cp, ri, x)
    S = OM.projected_inverse(n, cp, ri, L, D)
    ys = W.uniform_sym(n, cp, ri, rng, count=2)
    want = OD.hessian(n, cp, ri, x, list(ys))
    for k in range(2):
        T = OM.hessian(n, cp, ri, L, D, S, ys[k])
        assert _close(n, cp, ri, T, want[k], 1e-12)
        Y = OM.inv_hessian(n, cp, ri, L, D, S, OD.project(n, cp, ri, T))
        assert _close(n, cp, ri, Y, ys[k], 1e-11)
    # against the dense |V| x |V| solve on a T not produced by H
    t = W.uniform_sym(n, cp, ri, rng, count=1)[0]
    Y = OM.inv_hessian(n, cp, ri, L, D, S, t)
    assert _close(n, cp, ri, Y, OD.inv_hessian_dense(n, cp, ri, x, [t])[0], 1e-11)
