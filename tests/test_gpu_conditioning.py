"""Accuracy at condition number 1e6 for every operation, in every tier.

X = L0 D0 L0^T is planted on the analysed pattern with L0 unit lower
(off-diagonals uniform[-0.1, 0.1]) and D0 log-uniform in [1e-6, 1], so
that cond(X) is about 1e6 (measured densely and asserted).  The factor,
log det, gradient and Hessian are compared with the dense oracle at
relative error 1e-8.  The inverse Hessian is compared with the oracle's
clique-sum H^{-1}(T), also at 1e-8, although the Hessian's condition number
is about cond(X)^2 (1.0e12 measured on the band case's |V| x |V| matrix):
forward errors stay far below that bound (the two sides agree to 6e-10 or
better on these cases).  The completion of S = P(X^{-1}) has the planted X
itself as its solution (Eq. (e-Xhat-eq)), so its factor is compared with
the planted L0, D0 and with the oracle's refined completion.
"""
import numpy as np
import pytest

from oracle import dense as OD
from oracle import symbolic as OS
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


CASES = {
    "warp_band": (lambda: W.band(150, 6), dict()),
    "cta_arrow": (lambda: W.arrow(200, 120), dict()),
    "cta_grid": (lambda: W.grid2d(24, 24), dict(perm=W.nested_dissection((24, 24), leaf=6))),
    "dense_full": (lambda: W.band(150, 149), dict(big_rows=64, big_cols=64)),
    "dense_arrow": (lambda: W.arrow(260, 100), dict(big_rows=90, big_cols=70)),
    # the same dense-tier fronts with every product on the tensor cores
    "tc_dense_full": (lambda: W.band(150, 149), dict(big_rows=64, big_cols=64, tc_products=1)),
    "tc_dense_arrow": (lambda: W.arrow(260, 100), dict(big_rows=90, big_cols=70, tc_products=1)),
    "tc_dense600": (lambda: W.band(600, 599), dict(split_cols=256, tc_products=1)),
}

TOL = 1e-8        # factor, log det, gradient, Hessian (spec bound at condition 1e6)
TOL_INV = 1e-8    # inverse Hessian and completion, see the module docstring


@pytest.mark.parametrize("name", list(CASES))
def test_condition_1e6_factored_completion(name):
    """The completion with factored update matrices (Algorithm 4.3) at
    condition 1e6: S = P(X^{-1}) of the planted X, whose completion is X."""
    B = lib()
    mk, opts = CASES[name]
    sym = B.Symbolic(*mk(), completion="factored", **opts)
    n, cp, ri = sym.n, sym.colptr, sym.rowind
    rng = np.random.default_rng(11)
    x, l0, d0 = W.planted_factor(n, cp, ri, rng, dmin=1e-6, dmax=1.0)
    err = lambda a, b: OD.rel_err(n, cp, ri, a, b)
    s = OD.projected_inverse(n, cp, ri, x)
    fx, _ = sym.complete(dev(s))
    assert fx.status() == 0
    lh, dh = fx.export()
    assert err(host(lh), l0) < TOL_INV
    np.testing.assert_allclose(host(dh), d0, rtol=TOL_INV)


@pytest.mark.parametrize("name", list(CASES))
def test_condition_1e6_all_operations(name):
    B = lib()
    mk, opts = CASES[name]
    sym = B.Symbolic(*mk(), **opts)
    n, cp, ri = sym.n, sym.colptr, sym.rowind
    rng = np.random.default_rng(11)
    x, l0, d0 = W.planted_factor(n, cp, ri, rng, dmin=1e-6, dmax=1.0)
    X = OD.to_dense(n, cp, ri, x)
    kappa = np.linalg.cond(X)
    assert kappa > 1e5
    err = lambda a, b: OD.rel_err(n, cp, ri, a, b)

    f = sym.factor(dev(x))
    assert f.status() == 0
    l, d = f.export()
    lv, dv, _ = OD.factor(n, cp, ri, x)
    assert err(host(l), lv) < TOL
    np.testing.assert_allclose(host(d), dv, rtol=TOL)
    ld = f.logdet()
    want_ld = OD.logdet(n, cp, ri, x)
    assert abs(ld - want_ld) <= TOL * max(1.0, abs(want_ld))

    Z = OD.inverse(n, cp, ri, x)
    assert err(host(f.gradient()), -OD.project(n, cp, ri, Z)) < TOL
    ys = W.uniform_sym(n, cp, ri, rng, count=2)
    t = host(f.hessian(dev(ys)))
    want = OD.hessian(n, cp, ri, x, list(ys), Z=Z)
    for i in range(2):
        assert err(t[i], want[i]) < TOL

    I = [np.asarray(ri[cp[k] + 1:cp[k + 1]], dtype=np.int64) for k in range(n)]
    cl, seps = OS.cliques_and_separators(I, OS.etree(I))
    ts = W.uniform_sym(n, cp, ri, rng, count=2)
    yi = host(f.inv_hessian(dev(ts)))
    for i in range(2):
        wy = OD.inv_hessian_cliquesum(n, cp, ri, x, ts[i], cl, seps, S=Z)
        assert err(yi[i], wy) < TOL_INV

    s = OD.project(n, cp, ri, Z)  # S = P(X^{-1}): its completion is X (Eq. (e-Xhat-eq))
    fx, fstar = sym.complete(dev(s))
    assert fx.status() == 0
    lh, dh = fx.export()
    lh, dh = host(lh), host(dh)
    assert err(lh, l0) < TOL_INV
    np.testing.assert_allclose(dh, d0, rtol=TOL_INV)
    xh = OD.completion_refined(n, cp, ri, s, cl, seps)
    lv2, dv2, _ = OD.factor(n, cp, ri, xh)
    assert err(lh, lv2) < TOL_INV
    np.testing.assert_allclose(dh, dv2, rtol=TOL_INV)
    want_fs = OD.dual_barrier(n, cp, ri, xh)
    assert abs(fstar - want_fs) <= TOL_INV * max(1.0, abs(want_fs))
