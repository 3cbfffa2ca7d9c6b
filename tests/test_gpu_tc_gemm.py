"""The tensor-core FP64 product (digit splitting, tcgen05 bf16 MMAs) against
FP64 products computed on the host with numpy.

Bound: every entry within 2^-48 K max_l |a_il| max_l |b_lj| of the FP64
product (the splitting keeps 56 bits of each row's and column's scale and
drops digit pairs below 2^-52 of K max|a| max|b|; FP64 itself carries
2^-53 K of the same scale), and relative Frobenius error below 1e-13 on
well-scaled inputs.  Sizes cover single elements, ragged tiles, K longer
than one tensor-core pass, and rows spanning six decades.
"""
import numpy as np
import pytest

from tests.helpers import lib

pytestmark = pytest.mark.gpu


def _cm(t, x):
    """Column-major CUDA copy of the host matrix x."""
    return t.as_tensor(np.ascontiguousarray(x.T), dtype=t.float64, device="cuda").T


def _check(a, b, c0, alpha, beta, got):
    want = beta * c0 + alpha * (a @ b)
    K = a.shape[1]
    scale = K * np.abs(a).max(axis=1)[:, None] * np.abs(b).max(axis=0)[None, :] * abs(alpha)
    scale = scale + abs(beta) * np.abs(c0)
    assert np.all(np.abs(got - want) <= 2.0 ** -48 * scale + 1e-300)
    return np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)


SHAPES = [(1, 1, 1), (5, 3, 7), (100, 37, 300), (128, 32, 32), (257, 33, 1025), (640, 640, 512), (300, 900, 64)]


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_dgemm_tc_random(m, n, k):
    import torch
    B = lib()
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    a = rng.standard_normal((m, k))
    b = rng.uniform(-1.0, 1.0, (k, n))
    c = B.chd_dgemm_tc(_cm(torch, a), _cm(torch, b))
    torch.cuda.synchronize()
    rel = _check(a, b, np.zeros((m, n)), 1.0, 0.0, c.cpu().numpy())
    assert rel < 1e-13


def test_dgemm_tc_alpha_beta_and_scales():
    """beta C + alpha A B with rows of A spanning six decades and columns of
    B spanning three: the error stays within the row/column-scaled bound."""
    import torch
    B = lib()
    rng = np.random.default_rng(5)
    m, n, k = 300, 200, 700
    a = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-6, 0, (m, 1)) * 10.0 ** rng.uniform(-3, 0, (m, k))
    b = rng.standard_normal((k, n)) * 10.0 ** rng.uniform(-3, 0, (1, n))
    c0 = rng.standard_normal((m, n))
    c = _cm(torch, c0)
    B.chd_dgemm_tc(_cm(torch, a), _cm(torch, b), c, alpha=-0.5, beta=2.0)
    torch.cuda.synchronize()
    _check(a, b, c0, -0.5, 2.0, c.cpu().numpy())


def test_dgemm_tc_exact_integers():
    """Small integers are digits of themselves: the product is exact."""
    import torch
    B = lib()
    rng = np.random.default_rng(6)
    a = rng.integers(-1000, 1000, (130, 260)).astype(np.float64)
    b = rng.integers(-1000, 1000, (260, 70)).astype(np.float64)
    c = B.chd_dgemm_tc(_cm(torch, a), _cm(torch, b))
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy(), a @ b)


def test_tc_bf16_probe():
    """The raw bf16 MMA throughput probe runs and reports a positive rate."""
    B = lib()
    assert B.chd_probe_tc_bf16_peak() > 0.0
