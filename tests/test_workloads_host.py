"""The synthetic input recipe (patterns and values) and the autotuner's table
logic, on the host: the shapes, sizes and value distributions the measured
configurations are stated with."""
import json

import numpy as np
import pytest

import workloads as W
from oracle import dense as OD


def check_lower_csc(n, cp, ri):
    assert cp[0] == 0 and len(cp) == n + 1 and cp[-1] == len(ri)
    for j in range(n):
        col = ri[cp[j]:cp[j + 1]]
        assert col[0] == j  # diagonal first
        assert np.all(np.diff(col) > 0) and col[-1] < n  # sorted, in range


def test_band_and_arrow():
    n, cp, ri = W.band(50, 7)
    check_lower_csc(n, cp, ri)
    assert np.array_equal(np.diff(cp), np.minimum(8, 50 - np.arange(50)))
    assert all(ri[cp[j + 1] - 1] == min(j + 7, 49) for j in range(50))
    n, cp, ri = W.arrow(40, 6)
    check_lower_csc(n, cp, ri)
    for j in range(34):
        assert ri[cp[j]:cp[j + 1]].tolist() == [j] + list(range(34, 40))


def test_grids_and_nested_dissection():
    n, cp, ri = W.grid2d(7, 5)
    check_lower_csc(n, cp, ri)
    assert len(ri) - n == 7 * 4 + 5 * 6  # 5-point stencil edges
    n, cp, ri = W.grid3d(4, 3, 5)
    check_lower_csc(n, cp, ri)
    assert len(ri) - n == 3 * 3 * 5 + 4 * 2 * 5 + 4 * 3 * 4  # 7-point stencil edges
    perm = W.nested_dissection((9, 9), leaf=8)
    assert sorted(perm.tolist()) == list(range(81))
    # the top separator (the middle column of the 9 x 9 box) is ordered last
    assert sorted((perm[-9:] % 9).tolist()) == [4] * 9
    # a permuted pattern has the same entries, relabelled
    p2 = W.permute(W.grid2d(9, 9), perm)
    check_lower_csc(*p2)
    assert len(p2[2]) == len(W.grid2d(9, 9)[2])
    ident = W.permute(W.band(20, 3), np.arange(20))
    assert np.array_equal(ident[1], W.band(20, 3)[1]) and np.array_equal(ident[2], W.band(20, 3)[2])


def test_erdos_renyi_density():
    n, p = 2000, 0.001
    n_, cp, ri = W.erdos_renyi(n, p, np.random.default_rng(1))
    check_lower_csc(n, cp, ri)
    m = n * (n - 1) / 2
    k = len(ri) - n
    assert abs(k - p * m) < 5 * np.sqrt(p * m)


def test_values():
    n, cp, ri = W.band(60, 5)
    rng = np.random.default_rng(4)
    x = W.diag_dominant(n, cp, ri, rng)
    X = OD.to_dense(n, cp, ri, x)
    off = X - np.diag(np.diag(X))
    assert np.all(np.abs(off) <= 1.0)
    np.testing.assert_allclose(np.diag(X), np.abs(off).sum(axis=1) + 1.0, rtol=1e-15)
    assert np.linalg.eigvalsh(X).min() >= 1.0 - 1e-12  # Gershgorin: diagonal dominance by 1
    ys = W.uniform_sym(n, cp, ri, rng, count=3)
    assert ys.shape == (3, len(ri)) and np.all(np.abs(ys) <= 1.0)
    G = rng.standard_normal((n, 4))
    s = W.projected_gram(n, cp, ri, G, 0.5)
    np.testing.assert_allclose(s, OD.project(n, cp, ri, G @ G.T + 0.5 * np.eye(n)), rtol=1e-14, atol=1e-14)


def test_batch_mix_recipe():
    inst = W.batch_mix(30, 3)
    assert len(inst) == 30
    for i, (pat, perm, kind) in enumerate(inst):
        assert kind == ("band", "arrow", "grid")[i % 3]
        n = pat[0]
        assert 280 <= n <= 30100  # log-uniform in [300, 30000]; grids round to a square
        if kind == "grid":
            assert perm is not None and sorted(perm.tolist()) == list(range(n))


def test_autotune_signature_and_table(tmp_path):
    from paper_1203_2742_gb300 import autotune

    class Fake:
        n, nnz = 5000, 1114524

        def supernodes(self):
            return np.array([0, 1]), np.array([-1]), np.array([0, 1390]), np.arange(1390)
    assert autotune.signature(Fake(), 8) == "n12-z20-J10-m3"
    path = str(tmp_path / "table.json")
    t = autotune.Table(path)
    assert t.lookup("n12-z20-J10-m3") is None
    cfg = dict(big_rows=128, big_cols=64, split_cols=256)
    t.store("n12-z20-J10-m3", cfg, {"a": 1.0})
    assert autotune.Table(path).lookup("n12-z20-J10-m3") == cfg
    assert json.load(open(path))["n12-z20-J10-m3"]["timings_ms"] == {"a": 1.0}
