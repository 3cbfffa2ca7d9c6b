"""The completion with factored update matrices (chd_opts.completion = 1;
Algorithm 4.3 and its supernodal form at the end of §7.2) on the GPU: the
parity cases of every tier (warp, wide warp, CTA, leaf groups, the dense
tier with and without tensor-core products, split supernodes whose pieces
delete no rows) against the oracle's max-det completion, against the
independent form on the same pattern, and through the propagated factors
G_k = P R_k P that the Hessian factor of the completion object reuses."""
import numpy as np
import pytest

from oracle import dense as OD
from oracle import symbolic as OS
import workloads as W
from tests.test_gpu_parity import small_cases

pytestmark = pytest.mark.gpu

TOL = 1e-10
FCASES = small_cases(completion="factored")
ICASES = small_cases()


def _s(c):
    G = c.rng.standard_normal((c.n, 10))
    return W.projected_gram(c.n, c.cp, c.ri, G, 0.5)


@pytest.mark.parametrize("name", list(FCASES))
def test_factored_completion(name):
    c = FCASES[name]()
    s = _s(c)
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
    # the same factor as the independent form, up to rounding
    ci = ICASES[name]()
    assert np.array_equal(ci.cp, c.cp) and np.array_equal(ci.ri, c.ri)
    fi, fstar_i = ci.sym.complete(ci.dev(s))
    li, di = fi.export()
    assert c.err(c.host(l), c.host(li)) < 1e-12
    np.testing.assert_allclose(c.host(d), c.host(di), rtol=1e-12)
    # the dual Hessian on the completion object: H_{X-hat}^{-1}
    t = W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=1)
    yh = c.host(fx.inv_hessian(c.dev(t)))[0]
    Sd = OD.to_dense(c.n, c.cp, c.ri, s)
    want = OD.inv_hessian_cliquesum(c.n, c.cp, c.ri, xh, t[0], cl, seps, S=Sd)
    assert c.err(yh, want) < 1e-9


@pytest.mark.parametrize("name", ["band200_w8", "grid14_nd", "arrow60_w7", "dense_tier_grid", "dense_tier_er",
                                  "split_dense", "tc_dense_arrow", "wide_front"])
def test_propagated_factors_serve_the_hessian_factor(name):
    """The factored form leaves G_k = P R_k P = chol(P V_k P) in place of the
    Hessian factor's own Cholesky factorisations of V_k (§5.4): R(Y) on the
    completion object equals R(Y) on an independent completion object."""
    c = FCASES[name]()
    ci = ICASES[name]()
    s = _s(c)
    fx, _ = c.sym.complete(c.dev(s))
    fi, _ = ci.sym.complete(ci.dev(s))
    y = W.uniform_sym(c.n, c.cp, c.ri, c.rng, count=3)
    w = c.host(fx.hessian_factor(c.dev(y)))
    wi = c.host(fi.hessian_factor(ci.dev(y)))
    for j in range(3):
        assert np.linalg.norm(w[j] - wi[j]) <= 1e-12 * np.linalg.norm(wi[j])
