"""Autotuner: the tier cutovers change how fronts map onto the GPU, never the
results (beyond rounding); tuning picks one of the candidates and the table
persists it."""
import json

import numpy as np
import pytest

from oracle import dense as OD
import workloads as W
from tests.helpers import lib

pytestmark = pytest.mark.gpu

def _checker_table():
    """A tier table that alternates the tier by bucket (dense where the
    bucket indices have an odd sum, per-front tiers elsewhere)."""
    t = np.fromfunction(lambda i, j: (i + j) % 2, (13, 13)).astype(np.int32)
    return t


CONFIGS = [dict(), dict(big_rows=16, big_cols=8), dict(big_rows=4096, big_cols=4096),
           dict(split_cols=8), dict(big_rows=40, big_cols=12, split_cols=16),
           dict(tier_table=_checker_table()), dict(tc_products=1, big_rows=16, big_cols=8)]


@pytest.mark.parametrize("case", ["grid", "er"])
def test_results_invariant_under_tier_settings(case):
    import torch
    B = lib()
    if case == "grid":
        pat, kw = W.permute(W.grid2d(24, 24), W.nested_dissection((24, 24), leaf=6)), {}
    else:
        pat, kw = W.erdos_renyi(260, 0.03, np.random.default_rng(61)), dict(ordering="mindeg", relax=8)
    ref = None
    for cfg in CONFIGS:
        sym = B.Symbolic(*pat, **kw, **cfg)
        rng = np.random.default_rng(62)
        x = W.diag_dominant(sym.n, sym.colptr, sym.rowind, rng)
        ys = W.uniform_sym(sym.n, sym.colptr, sym.rowind, rng, count=3)
        s = W.projected_gram(sym.n, sym.colptr, sym.rowind, rng.standard_normal((sym.n, 6)), 0.5)
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        f = sym.factor(dev(x))
        out = dict(ld=f.logdet(), g=f.gradient().cpu().numpy(), t=f.hessian(dev(ys)).cpu().numpy(),
                   y=f.inv_hessian(dev(ys)).cpu().numpy())
        fx, fstar = sym.complete(dev(s))
        out["fstar"] = fstar
        out["xl"] = fx.export()[0].cpu().numpy()
        if ref is None:
            ref, rsym = out, sym
            want = OD.hessian(sym.n, sym.colptr, sym.rowind, x, list(ys))
            for j in range(3):
                assert OD.rel_err(sym.n, sym.colptr, sym.rowind, out["t"][j], want[j]) < 1e-10
            continue
        # same analysed pattern whatever the tier settings (splitting keeps V)
        assert (sym.colptr == rsym.colptr).all() and (sym.rowind == rsym.rowind).all()
        err = lambda a, b: OD.rel_err(sym.n, sym.colptr, sym.rowind, a, b)
        assert abs(out["ld"] - ref["ld"]) < 1e-12 * abs(ref["ld"])
        assert abs(out["fstar"] - ref["fstar"]) < 1e-12 * abs(ref["fstar"])
        assert err(out["g"], ref["g"]) < 1e-12
        assert err(out["xl"], ref["xl"]) < 1e-12
        for j in range(3):
            assert err(out["t"][j], ref["t"][j]) < 1e-12
            assert err(out["y"][j], ref["y"][j]) < 1e-12


def test_tune_and_table(tmp_path):
    B = lib()
    from paper_1203_2742_gb300 import autotune
    pat = W.permute(W.grid2d(30, 30), W.nested_dissection((30, 30), leaf=6))
    make = lambda **cfg: B.Symbolic(*pat, **cfg)
    cands = (dict(big_rows=64, big_cols=32), dict(big_rows=4096, big_cols=4096))
    path = str(tmp_path / "tune.json")
    table = autotune.Table(path)
    sym, cfg, sig = autotune.analyze_tuned(make, 4, table, candidates=cands)
    assert cfg in [dict(c) for c in cands]
    assert table.lookup(sig) == cfg
    again = autotune.Table(path)  # persisted
    assert again.lookup(sig) == cfg
    with open(path) as f:
        data = json.load(f)
    assert len(data[sig]["timings_ms"]) == len(cands)
    # a tier table round-trips through the file
    table.store("with-table", dict(cfg, tier_table=_checker_table()), {})
    got = autotune.Table(path).lookup("with-table")
    assert np.array_equal(got["tier_table"], _checker_table())


def test_refine_tiers_returns_a_table_and_keeps_results():
    """The per-front-shape refinement runs on a pattern with fronts on both
    sides of the cutover, returns a valid table, and the table's analysis
    gives the same Hessian as the default one."""
    import torch
    B = lib()
    from paper_1203_2742_gb300 import autotune
    pat = W.erdos_renyi(600, 0.01, np.random.default_rng(63))
    make = lambda **cfg: B.Symbolic(*pat, ordering="mindeg", relax=8, **cfg)
    cfg = dict(big_rows=64, big_cols=32)
    best, timings = autotune.tune(make, 2, candidates=(cfg,), op="step", reps=1)
    base = timings[json.dumps(cfg, sort_keys=True)]
    table, trials, ms = autotune.refine_tiers(make, cfg, 2, base, trials=3, reps=1)
    assert table.shape == (13, 13) and set(np.unique(table)) <= {-1, 0, 1}
    assert len(trials) <= 3 and ms <= base
    s0, s1 = make(**cfg), make(**cfg, tier_table=table)
    rng = np.random.default_rng(64)
    x = W.diag_dominant(s0.n, s0.colptr, s0.rowind, rng)
    ys = W.uniform_sym(s0.n, s0.colptr, s0.rowind, rng, count=2)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    t0 = s0.factor(dev(x)).hessian(dev(ys)).cpu().numpy()
    t1 = s1.factor(dev(x)).hessian(dev(ys)).cpu().numpy()
    for j in range(2):
        assert OD.rel_err(s0.n, s0.colptr, s0.rowind, t1[j], t0[j]) < 1e-12


def test_refine_tc_chooses_a_setting_and_keeps_results():
    """The tensor-core trial: the returned setting is the given one or the
    same with FP64 units only, and both give the same Hessian."""
    import torch
    B = lib()
    from paper_1203_2742_gb300 import autotune
    pat = W.band(500, 499)
    make = lambda **cfg: B.Symbolic(*pat, **cfg)
    cfg = dict(big_rows=64, big_cols=32, split_cols=128)
    best, timings = autotune.tune(make, 4, candidates=(cfg,), op="step", reps=1)
    chosen, ms = autotune.refine_tc(make, cfg, 4, timings[json.dumps(cfg, sort_keys=True)], reps=1)
    assert ms > 0 and chosen in (cfg, dict(cfg, tc_products=-1))
    s0, s1 = make(**cfg), make(**cfg, tc_products=-1)
    rng = np.random.default_rng(65)
    x = W.diag_dominant(s0.n, s0.colptr, s0.rowind, rng)
    ys = W.uniform_sym(s0.n, s0.colptr, s0.rowind, rng, count=4)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    t0 = s0.factor(dev(x)).hessian(dev(ys)).cpu().numpy()
    t1 = s1.factor(dev(x)).hessian(dev(ys)).cpu().numpy()
    for j in range(4):
        assert OD.rel_err(s0.n, s0.colptr, s0.rowind, t1[j], t0[j]) < 1e-12
