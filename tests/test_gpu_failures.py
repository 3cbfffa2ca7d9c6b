"""Failure reporting in every tier: a matrix that is not positive definite
(Algorithm 7.1 meets a non-positive pivot) and a matrix S without a
positive definite completion (Algorithm 7.3, §4.2: a pivot of chol(S_AA)
or of S_NN - S_AN^T S_AA^{-1} S_AN is not positive) are reported through the
factor's status, never by a fault; the first failing supernode and column
are recorded, and the same factor object computes correct results after a
refactor with a valid matrix.

The failing pivot is planted in a front of a chosen tier: the per-task
CTA tier (the 121-column root of an arrow), a leaf group (the one-column
leaves of the same arrow, processed together), the multi-CTA dense tier
(a dense 150 x 150 pattern, and dense-tier one-column leaves of an arrow
with low thresholds), and the warp tier (a band).
"""
import numpy as np
import pytest

from oracle import dense as OD
import workloads as W
from tests.helpers import lib

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def dev(a):
    t = _torch()
    return t.as_tensor(np.ascontiguousarray(a), dtype=t.float64, device="cuda")


def host(t_):
    _torch().cuda.synchronize()
    return t_.cpu().numpy()


# pattern, analysis options, the column whose diagonal entry is made negative
CASES = {
    "cta_root": (lambda: W.arrow(200, 120), dict(), 150),
    "leaf_group": (lambda: W.arrow(200, 120), dict(), 10),
    "dense_front": (lambda: W.band(150, 149), dict(big_rows=64, big_cols=64), 100),
    "dense_leaf": (lambda: W.arrow(260, 100), dict(big_rows=90, big_cols=70), 10),
    "dense_split_piece": (lambda: W.band(600, 599), dict(split_cols=256), 300),
    "warp_band": (lambda: W.band(50, 3), dict(), 20),
}


@pytest.mark.parametrize("name", list(CASES))
def test_not_positive_definite_reported(name):
    B = lib()
    mk, opts, col = CASES[name]
    sym = B.Symbolic(*mk(), **opts)
    n, cp, ri = sym.n, sym.colptr, sym.rowind
    assert np.array_equal(sym.perm, np.arange(n))  # natural order kept: col is the planted column
    rng = np.random.default_rng(5)
    x_ok = W.diag_dominant(n, cp, ri, rng)
    x = x_ok.copy()
    x[cp[col]] = -5.0
    f = sym.factor(dev(x))
    assert f.status() == B.CHD_ERR_NOT_PD
    rc, snode, c = f.error_detail()
    assert rc == B.CHD_ERR_NOT_PD
    sp = sym.supernodes()[0]
    assert 0 <= snode < len(sp) - 1 and sp[snode] <= c < sp[snode + 1]
    # the columns before the planted one are unchanged and positive
    # definite, and every later column depends on it: the first failing
    # pivot is the planted column's
    assert c == col
    # recovery: the same factor object with a valid matrix
    f.refactor(dev(x_ok))
    assert f.status() == 0
    g = host(f.gradient())
    assert OD.rel_err(n, cp, ri, g, OD.gradient(n, cp, ri, x_ok)) < 1e-10


@pytest.mark.parametrize("completion", ["independent", "factored"])
@pytest.mark.parametrize("name", list(CASES))
def test_not_completable_reported(name, completion):
    """Both completion forms: the factored one (Algorithm 4.3) meets the
    failing pivot while propagating R_k or in the front's own Cholesky."""
    B = lib()
    mk, opts, col = CASES[name]
    sym = B.Symbolic(*mk(), completion=completion, **opts)
    n, cp, ri = sym.n, sym.colptr, sym.rowind
    rng = np.random.default_rng(6)
    s_ok = W.projected_gram(n, cp, ri, rng.standard_normal((n, 10)), 0.5)
    s = s_ok.copy()
    s[cp[col]] = -1.0  # a negative diagonal entry: no positive semidefinite completion
    try:
        sym.complete(dev(s))
        raise AssertionError("expected CHD_ERR_NOT_COMPLETABLE")
    except B.ChdError as e:
        assert e.code == B.CHD_ERR_NOT_COMPLETABLE
    # a valid S on the same symbolic object completes, and X-hat is right
    fx, fstar = sym.complete(dev(s_ok))
    assert fx.status() == 0
    X = OD.to_dense(n, cp, ri, host(fx.product()))
    # P(X-hat^{-1}) = S (Eq. (e-Xhat-eq))
    assert OD.rel_err(n, cp, ri, OD.project(n, cp, ri, np.linalg.inv(X)), s_ok) < 1e-10
