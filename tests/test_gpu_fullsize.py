"""GPU parity on the paths and at the sizes the benchmark runs.

* Dense-tier fronts whose products are split along their inner dimension
  (partial products summed in a fixed order by a second launch): a dense
  600 x 600 pattern split into 256-column supernodes, an arrow whose
  one-column fronts have |A| = 330, and a dense 1000 x 1000 pattern split
  into 512-column supernodes.  The library's split-product counter shows
  that the split path ran.
* The Erdos-Renyi workload of the benchmark (n = 5000, p = 0.001, minimum
  degree, relaxed supernodes, 8 right-hand sides) built exactly as
  ``bench.py`` builds it, under every tier setting the autotuner can choose:
  factor, log det, gradient, Hessian, inverse Hessian, completion and f_*
  against the dense oracle (all entries; the completion's reference is the
  clique-sum closed form refined by Newton steps until P(X^{-1}) = S holds
  to rounding, see ``oracle.dense.completion_refined``).
* The 150 x 150 grid (n = 22500, 64 right-hand sides in one call), on
  entries sampled from the outputs, which the oracle computes one by one.

Tolerance: relative Frobenius error 1e-10 in the symmetric norm
(off-diagonals counted twice); entry samples: max |error| <= 1e-10 times
the largest |entry| of the sample.
"""
import numpy as np
import pytest

from oracle import dense as OD
from oracle import symbolic as OS
import workloads as W
from tests.helpers import lib

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _torch():
    import torch
    return torch


def dev(a):
    t = _torch()
    return t.as_tensor(np.ascontiguousarray(a), dtype=t.float64, device="cuda")


def host(t_):
    _torch().cuda.synchronize()
    return t_.cpu().numpy()


def _cliques(n, cp, ri):
    I = [np.asarray(ri[cp[k] + 1:cp[k + 1]], dtype=np.int64) for k in range(n)]
    return OS.cliques_and_separators(I, OS.etree(I))


# ---------------------------------------------------------------------------
# split products in the dense tier
# ---------------------------------------------------------------------------

SPLIT_CASES = {
    # 600-column clique in 256-column pieces: the first piece's gradient
    # product (256 x 256 output, inner dimension |A| = 344) is split
    "dense600_split256": (lambda: W.band(600, 599), dict(split_cols=256), True),
    # one-column fronts with |A| = 330 (dense tier): V K_AN has 3 x 1 tiles
    # per right-hand side and inner dimension 330
    "arrow400_w330": (lambda: W.arrow(400, 330), dict(), True),
    # the benchmark's widest split setting on a wide clique
    "dense1000_split512": (lambda: W.band(1000, 999), dict(split_cols=512), False),
}


@pytest.mark.parametrize("name", list(SPLIT_CASES))
def test_dense_tier_split_products(name):
    B = lib()
    mk, opts, must_split = SPLIT_CASES[name]
    sym = B.Symbolic(*mk(), **opts)
    n, cp, ri = sym.n, sym.colptr, sym.rowind
    rng = np.random.default_rng(len(ri))
    x = W.diag_dominant(n, cp, ri, rng)
    k0 = B.chd_split_k_launches()
    f = sym.factor(dev(x))
    ld = f.logdet()
    assert f.status() == 0
    l, d = f.export()
    g = host(f.gradient())
    ys = W.uniform_sym(n, cp, ri, rng, count=3)
    t1 = host(f.hessian(dev(ys[:1])))
    t3 = host(f.hessian(dev(ys)))
    ts = W.uniform_sym(n, cp, ri, rng, count=2)
    y1 = host(f.inv_hessian(dev(ts[:1])))
    y2 = host(f.inv_hessian(dev(ts)))
    s = W.projected_gram(n, cp, ri, rng.standard_normal((n, 20)), 0.5)
    fx, fstar = sym.complete(dev(s))
    assert fx.status() == 0
    lh, dh = fx.export()
    xp = host(f.product())
    if must_split:
        assert B.chd_split_k_launches() > k0, "the split-product path did not run"

    err = lambda a, b: OD.rel_err(n, cp, ri, a, b)
    Z = OD.inverse(n, cp, ri, x)
    lv, dv, _ = OD.factor(n, cp, ri, x)
    assert abs(ld - OD.logdet(n, cp, ri, x)) <= TOL * max(1.0, abs(ld))
    np.testing.assert_allclose(host(d), dv, rtol=1e-11)
    assert err(host(l), lv) < TOL
    assert err(g, -OD.project(n, cp, ri, Z)) < TOL
    want = OD.hessian(n, cp, ri, x, list(ys), Z=Z)
    assert err(t1[0], want[0]) < TOL
    for i in range(3):
        assert err(t3[i], want[i]) < TOL
    cl, seps = _cliques(n, cp, ri)
    for i in range(2):
        wy = OD.inv_hessian_cliquesum(n, cp, ri, x, ts[i], cl, seps, S=Z)
        assert err(y2[i], wy) < TOL
        if i == 0:
            assert err(y1[0], wy) < TOL
    xh = OD.completion_refined(n, cp, ri, s, cl, seps)
    lv2, dv2, _ = OD.factor(n, cp, ri, xh)
    np.testing.assert_allclose(host(dh), dv2, rtol=1e-10)
    assert err(host(lh), lv2) < TOL
    want_fs = OD.dual_barrier(n, cp, ri, xh)
    assert abs(fstar - want_fs) <= TOL * max(1.0, abs(want_fs))
    assert err(xp, x) < 1e-12


# ---------------------------------------------------------------------------
# the Erdos-Renyi workload of the benchmark, all entries
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def er5000():
    import bench
    B = lib()
    wl = bench.make_workload("er5000")
    sym = bench.make_symbolic(B, wl)
    n, cp, ri = sym.n, sym.colptr, sym.rowind
    x, ys, s = bench.workload_values(wl, n, cp, ri)
    ts = W.uniform_sym(n, cp, ri, np.random.default_rng(77), count=wl["m"])
    Z = OD.inverse(n, cp, ri, x)
    lv, dv, _ = OD.factor(n, cp, ri, x)
    cl, seps = _cliques(n, cp, ri)
    xh = OD.completion_refined(n, cp, ri, s, cl, seps)
    lh, dh, _ = OD.factor(n, cp, ri, xh)
    want = dict(
        logdet=OD.logdet(n, cp, ri, x), l=lv, d=dv, g=-OD.project(n, cp, ri, Z),
        t=OD.hessian(n, cp, ri, x, list(ys), Z=Z),
        yi=[OD.inv_hessian_cliquesum(n, cp, ri, x, ts[i], cl, seps, S=Z) for i in range(2)],
        xh=xh, lh=lh, dh=dh, fstar=OD.dual_barrier(n, cp, ri, xh))
    return dict(wl=wl, n=n, cp=cp, ri=ri, x=x, ys=ys, ts=ts, s=s, want=want)


def _candidates():
    from paper_1203_2742_gb300 import autotune
    return [dict(c) for c in autotune.DEFAULT_CANDIDATES]


@pytest.mark.parametrize("cfg", _candidates(), ids=lambda c: "r{big_rows}-c{big_cols}-s{split_cols}".format(**c))
def test_er5000_full_size(er5000, cfg):
    """Every operation of the benchmark step on its Erdos-Renyi workload,
    with each tier setting the autotuner may pick, against the oracle."""
    import bench
    B = lib()
    E = er5000
    n, cp, ri, w = E["n"], E["cp"], E["ri"], E["want"]
    sym = bench.make_symbolic(B, E["wl"], **cfg)
    assert np.array_equal(sym.colptr, cp) and np.array_equal(sym.rowind, ri)  # splitting keeps V
    m = E["wl"]["m"]
    f = sym.factor(dev(E["x"]))
    ld = f.logdet()
    assert f.status() == 0
    l, d = f.export()
    g = host(f.gradient())
    T = f.hessian(dev(E["ys"]))
    t = host(T)
    yr = host(f.inv_hessian(T))           # the benchmark's round trip H^{-1}(H(Y))
    yi = host(f.inv_hessian(dev(E["ts"])))
    fx, fstar = sym.complete(dev(E["s"]))
    assert fx.status() == 0
    lh, dh = fx.export()
    xh = host(fx.product())

    err = lambda a, b: OD.rel_err(n, cp, ri, a, b)
    assert abs(ld - w["logdet"]) <= TOL * max(1.0, abs(w["logdet"]))
    np.testing.assert_allclose(host(d), w["d"], rtol=1e-11)
    assert err(host(l), w["l"]) < TOL
    assert err(g, w["g"]) < TOL
    for i in range(m):
        assert err(t[i], w["t"][i]) < TOL, i
        assert err(yr[i], E["ys"][i]) < TOL, i
    for i in range(2):
        assert err(yi[i], w["yi"][i]) < TOL, i
    np.testing.assert_allclose(host(dh), w["dh"], rtol=1e-10)
    assert err(host(lh), w["lh"]) < TOL
    assert err(xh, w["xh"]) < TOL
    assert abs(fstar - w["fstar"]) <= TOL * max(1.0, abs(w["fstar"]))


def test_er5000_factored_completion(er5000):
    """The completion with factored update matrices (Algorithm 4.3) on the
    benchmark's Erdos-Renyi workload with its tier setting, all entries."""
    import bench
    B = lib()
    E = er5000
    n, cp, ri, w = E["n"], E["cp"], E["ri"], E["want"]
    sym = bench.make_symbolic(B, E["wl"], big_rows=192, big_cols=96, split_cols=512, completion="factored")
    fx, fstar = sym.complete(dev(E["s"]))
    assert fx.status() == 0
    lh, dh = fx.export()
    err = lambda a, b: OD.rel_err(n, cp, ri, a, b)
    np.testing.assert_allclose(host(dh), w["dh"], rtol=1e-10)
    assert err(host(lh), w["lh"]) < TOL
    assert err(host(fx.product()), w["xh"]) < TOL
    assert abs(fstar - w["fstar"]) <= TOL * max(1.0, abs(w["fstar"]))


def test_er5000_reaches_split_products():
    """The Erdos-Renyi workload of the benchmark runs split products (its
    dense-tier fronts with few columns and long ancestor sets) under every
    tier setting the autotuner may pick, so the comparisons above cover the
    split path."""
    import bench
    B = lib()
    wl = bench.make_workload("er5000")
    for cfg in _candidates():
        sym = bench.make_symbolic(B, wl, **cfg)
        n, cp, ri = sym.n, sym.colptr, sym.rowind
        x, ys, s = bench.workload_values(wl, n, cp, ri)
        k0 = B.chd_split_k_launches()
        f = sym.factor(dev(x))
        f.gradient()
        f.inv_hessian(f.hessian(dev(ys)))
        sym.complete(dev(s))
        _torch().cuda.synchronize()
        assert B.chd_split_k_launches() > k0, cfg


# ---------------------------------------------------------------------------
# the 150 x 150 grid with 64 right-hand sides, sampled entries
# ---------------------------------------------------------------------------

def _max_err(got, want):
    return float(np.max(np.abs(got - want))) / max(float(np.max(np.abs(want))), 1e-300)


def test_grid150_full_size_sampled():
    """The grid workload of the benchmark at full size: one Hessian call and
    one inverse-Hessian call with 64 right-hand sides.  The oracle computes
    sampled entries of the gradient and of the Hessian of two right-hand
    sides one by one from the dense X^{-1}; the inverse Hessian is checked
    through the round trip H^{-1}(H(Y)) = Y on every right-hand side, and
    log det against the dense Cholesky factor."""
    import bench
    B = lib()
    wl = bench.make_workload("grid150")
    sym = bench.make_symbolic(B, wl)
    n, cp, ri = sym.n, sym.colptr, sym.rowind
    x, ys, _ = bench.workload_values(wl, n, cp, ri)
    f = sym.factor(dev(x))
    ld = f.logdet()
    g = host(f.gradient())
    T = f.hessian(dev(ys))
    t = host(T)
    yr = host(f.inv_hessian(T))
    m = ys.shape[0]
    assert m == 64
    rng = np.random.default_rng(150)
    r, c = OD.pattern_pairs(n, cp, ri)
    sel = np.concatenate([rng.choice(len(r), size=400, replace=False), np.flatnonzero(r == c)[:50]])
    Z = OD.inverse(n, cp, ri, x)
    assert abs(ld - OD.logdet(n, cp, ri, x)) <= TOL * max(1.0, abs(ld))
    assert _max_err(g[sel], -Z[r[sel], c[sel]]) < TOL
    for i in (0, m - 1):
        want = OD.hessian_entries(n, cp, ri, Z, ys[i], r[sel], c[sel])
        assert _max_err(t[i][sel], want) < TOL, i
    for i in range(m):
        assert OD.rel_err(n, cp, ri, yr[i], ys[i]) < TOL, i
