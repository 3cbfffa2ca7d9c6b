"""The supernodal block algorithms (Algorithms 7.1-7.3 and the block forms
of Algorithms 5.1 and 5.2 derived by linearising the block factorisation,
``oracle.supernodal``) against the dense definitions, on one-column,
fundamental and merged partitions of the same patterns: the block reading
of the Hessian and inverse Hessian checked on the CPU, independently of the
GPU."""
import numpy as np
import pytest

from oracle import dense as OD
from oracle import supernodal as OSN
from oracle import symbolic as OS
import workloads as W
from tests.test_oracle_factored import CASES, _case


def _vals(n, cp, ri, A):
    return OD.project(n, cp, ri, A)


@pytest.mark.parametrize("name", CASES)
def test_block_factor_projected_inverse_and_completion(name):
    n, cp, ri, sp = _case(name)
    rng = np.random.default_rng(11)
    x = W.diag_dominant(n, cp, ri, rng)
    L, D = OSN.factor(n, cp, ri, x, sp)
    err = lambda a, b: OD.rel_err(n, cp, ri, a, b)
    assert err(_vals(n, cp, ri, L @ D @ L.T), x) < 1e-13
    # L_AN blocks only on V (Eq. (e-filled)): no fill outside the pattern
    mask = np.tril(OD.to_dense(n, cp, ri, np.ones(len(ri))) != 0)
    assert np.all((L - np.eye(n))[~mask] == 0.0)
    S = OSN.projected_inverse(n, cp, ri, L, D, sp)
    assert err(_vals(n, cp, ri, S), OD.projected_inverse(n, cp, ri, x)) < 1e-12
    s = W.projected_gram(n, cp, ri, rng.standard_normal((n, 4)), 0.5)
    Lc, Dc = OSN.completion(n, cp, ri, s, sp)
    Xh = Lc @ Dc @ Lc.T
    I = [np.asarray(ri[cp[k] + 1:cp[k + 1]], dtype=np.int64) for k in range(n)]
    cl, seps = OS.cliques_and_separators(I, OS.etree(I))
    assert err(_vals(n, cp, ri, Xh), OD.completion_refined(n, cp, ri, s, cl, seps)) < 1e-12


@pytest.mark.parametrize("name", CASES)
def test_block_hessian_and_inverse(name):
    n, cp, ri, sp = _case(name)
    rng = np.random.default_rng(12)
    x = W.diag_dominant(n, cp, ri, rng)
    L, D = OSN.factor(n, cp, ri, x, sp)
    S = OD.to_dense(n, cp, ri, OD.projected_inverse(n, cp, ri, x))
    err = lambda a, b: OD.rel_err(n, cp, ri, a, b)
    ys = W.uniform_sym(n, cp, ri, rng, count=2)
    want = OD.hessian(n, cp, ri, x, list(ys))
    for k in range(2):
        T = OSN.hessian(n, cp, ri, L, D, S, ys[k], sp)
        assert err(_vals(n, cp, ri, T), want[k]) < 1e-12
        Y = OSN.inv_hessian(n, cp, ri, L, D, S, _vals(n, cp, ri, T), sp)
        assert err(_vals(n, cp, ri, Y), ys[k]) < 1e-11


@pytest.mark.parametrize("name", CASES)
def test_block_hessian_factor_equals_the_per_column_one(name):
    """Reading of §5.4 in block form: W_NN = C^{-1} K_NN C^{-T} (lower) and
    W_AN = Q^T K_AN C^{-T} give the per-column W of Algorithm 5.3 on every
    partition, and R^adj(R(Y)) = H(Y)."""
    n, cp, ri, sp = _case(name)
    rng = np.random.default_rng(13)
    x = W.diag_dominant(n, cp, ri, rng)
    L, D = OSN.factor(n, cp, ri, x, sp)
    S = OD.to_dense(n, cp, ri, OD.projected_inverse(n, cp, ri, x))
    err = lambda a, b: OD.rel_err(n, cp, ri, a, b)
    ys = W.uniform_sym(n, cp, ri, rng, count=2)
    want_w = OD.hessian_factor(n, cp, ri, x, list(ys))
    want_t = OD.hessian(n, cp, ri, x, list(ys))
    for k in range(2):
        Wb = OSN.hessian_factor(n, cp, ri, L, D, S, ys[k], sp)
        wv = _vals(n, cp, ri, Wb)  # lower entries on V
        assert err(wv, want_w[k]) < 1e-12
        T = OSN.hessian_factor_adj(n, cp, ri, L, D, S, wv, sp)
        assert err(_vals(n, cp, ri, T), want_t[k]) < 1e-12
