"""Autotuner for the tier cutovers of the front kernels and the per-front
tier table.

Which tier processes a front -- one warp (small fronts), one CTA (medium),
or the multi-CTA dense tier (fronts with |J| >= big_rows or |N| >= big_cols)
-- and how wide supernodes are split (split_cols) decide how the work of a
pattern maps onto the GPU; the numbers do not change the results beyond
rounding.  ``tune`` times a set of candidate settings on the pattern itself
(the chosen operation with m right-hand sides, CUDA events after a warm-up
call) and keeps the fastest.  ``Table`` persists the choices in a JSON file,
keyed by a coarse signature of the pattern (order, filled nonzeros, largest
front and m, each bucketed by powers of two), so that later patterns of the
same shape reuse a choice without tuning again.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import binding as B

DEFAULT_CANDIDATES = (
    dict(big_rows=320, big_cols=160, split_cols=256),
    dict(big_rows=96, big_cols=48, split_cols=256),
    dict(big_rows=128, big_cols=64, split_cols=256),
    dict(big_rows=192, big_cols=96, split_cols=256),
    dict(big_rows=512, big_cols=256, split_cols=256),
    dict(big_rows=320, big_cols=160, split_cols=128),
    dict(big_rows=320, big_cols=160, split_cols=512),
    dict(big_rows=128, big_cols=64, split_cols=512),
    dict(big_rows=192, big_cols=96, split_cols=512),
)


def _bucket(v):
    return int(math.floor(math.log2(max(1, v))))


def signature(sym, m):
    """Coarse shape of an analysed pattern: log2 buckets of n, nnz, the
    largest front and m."""
    sp, par, rp, rows = sym.supernodes()
    maxJ = int(np.max(np.diff(rp))) if len(rp) > 1 else 1
    return f"n{_bucket(sym.n)}-z{_bucket(sym.nnz)}-J{_bucket(maxJ)}-m{_bucket(m)}"


def _time_config(make_symbolic, config, x_of, y_of, s_of, m, op, reps):
    import torch
    sym = make_symbolic(**config)
    x = x_of(sym)
    ys = y_of(sym)
    fac = sym.factor(x)
    fac.gradient()
    out = torch.empty_like(ys)
    out2 = torch.empty_like(ys)
    comp = None
    if op == "step":
        s = s_of(sym)
        comp, _ = sym.complete(s)

    def step():
        # one pass of every operation: refactor, gradient, Hessian, inverse
        # Hessian (with its per-factor V^{-1}) and completion
        fac.refactor(x)
        fac.gradient()
        fac.hessian(ys, out=out)
        fac.inv_hessian(out, out=out2)
        comp.recomplete(s, want_fstar=False)
    call = {"hessian": lambda: fac.hessian(ys, out=out),
            "inv_hessian": lambda: fac.inv_hessian(ys, out=out),
            "factor": lambda: fac.refactor(x),
            "gradient": lambda: fac.gradient(),
            "step": step}[op]
    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    fac.free()
    if comp is not None:
        comp.free()
    return ms


def _inputs(m, seed):
    import torch
    import workloads as W

    def x_of(sym):
        rng = np.random.default_rng(seed)
        return torch.as_tensor(W.diag_dominant(sym.n, sym.colptr, sym.rowind, rng), device="cuda")

    def y_of(sym):
        rng = np.random.default_rng(seed + 1)
        return torch.as_tensor(W.uniform_sym(sym.n, sym.colptr, sym.rowind, rng, count=m), device="cuda")

    def s_of(sym):
        rng = np.random.default_rng(seed + 2)
        G = rng.standard_normal((sym.n, 10))
        return torch.as_tensor(W.projected_gram(sym.n, sym.colptr, sym.rowind, G, 0.5), device="cuda")
    return x_of, y_of, s_of


def tune(make_symbolic, m, candidates=DEFAULT_CANDIDATES, op="hessian", reps=2, seed=0):
    """Time every candidate setting; returns (best_config, {config_key: ms}).

    make_symbolic(**config) must return an analysed ``Symbolic`` for the
    pattern with the given tier settings.  Values: X diagonally dominant, m
    right-hand sides uniform in [-1, 1] and S = P(G G^T + 0.5 I) (G n x 10)
    on the analysed pattern (seeded).  op: "hessian", "inv_hessian",
    "factor", "gradient", or "step" (every operation once, the inverse
    Hessian on the Hessian's output after a refactor, as a benchmark step
    runs them).
    """
    x_of, y_of, s_of = _inputs(m, seed)
    timings = {}
    best, best_ms = None, float("inf")
    for cfg in candidates:
        ms = _time_config(make_symbolic, cfg, x_of, y_of, s_of, m, op, reps)
        timings[json.dumps(cfg, sort_keys=True)] = ms
        if ms < best_ms:
            best, best_ms = dict(cfg), ms
    return best, timings


def refine_tc(make_symbolic, config, m, base_ms, op="step", reps=2, gain=0.02, seed=0):
    """The tensor-core choice on top of the chosen tiers: the library's cost
    model judges each dense-tier product alone; where many fronts share the
    GPU the FP64 units can be faster.  Times `config` with tc_products = -1
    (FP64 units only) and returns (config, ms of the trial): the trial's
    setting when it is more than `gain` faster than base_ms."""
    x_of, y_of, s_of = _inputs(m, seed)
    trial = dict(config, tc_products=-1)
    ms = _time_config(make_symbolic, trial, x_of, y_of, s_of, m, op, reps)
    return (trial if ms < (1.0 - gain) * base_ms else dict(config)), ms


def front_buckets(sym):
    """Per front: its (n_k, a_k) buckets of the tier table and its Hessian
    flops per right-hand side (6 a^2 n + 8 a n^2 + 2 n^3)."""
    sp, par, rp, rows = sym.supernodes()
    n = np.diff(np.asarray(sp, dtype=np.int64))
    a = np.diff(np.asarray(rp, dtype=np.int64)) - n
    bn = np.array([B.tier_bucket(v) for v in n], dtype=np.int64)
    ba = np.array([B.tier_bucket(v) for v in a], dtype=np.int64)
    work = 6.0 * a * a * n + 8.0 * a * n * n + 2.0 * n ** 3
    return n, a, bn, ba, work


def refine_tiers(make_symbolic, config, m, base_ms, op="step", trials=6, reps=2, gain=0.02, seed=0):
    """Per-front-shape refinement of the tier choice (a tier table, see
    chd_opts.tier_table): starting from the global cutovers of `config`,
    the `trials` buckets (n_k, a_k) that carry the most work among those
    adjacent to the cutover (a bucket whose fronts sit within a factor of
    two of big_rows or big_cols) are moved to the other tier one at a time,
    and a move is kept when the timed operation gets faster by more than
    `gain`.  Returns (table as a TIER_BUCKETS x TIER_BUCKETS int array,
    {bucket: ms} of the trials, best ms)."""
    x_of, y_of, s_of = _inputs(m, seed)
    sym = make_symbolic(**config)
    n, a, bn, ba, work = front_buckets(sym)
    br = config.get("big_rows") or 320
    bc = config.get("big_cols") or 160
    J = n + a
    dense = (J >= br) | (n >= bc)
    near = ((J >= br // 2) & (J < 2 * br)) | ((n >= bc // 2) & (n < 2 * bc))
    stats = {}
    for i in np.flatnonzero(near):
        key = (int(bn[i]), int(ba[i]))
        w, d, c = stats.get(key, (0.0, 0, 0))
        stats[key] = (w + work[i], d + int(dense[i]), c + 1)
    order = sorted(stats, key=lambda k: -stats[k][0])[:trials]
    table = -np.ones((B.TIER_BUCKETS, B.TIER_BUCKETS), dtype=np.int32)
    best_ms, timings = base_ms, {}
    for key in order:
        w, d, c = stats[key]
        trial = table.copy()
        trial[key] = 0 if 2 * d >= c else 1
        ms = _time_config(make_symbolic, dict(config, tier_table=trial), x_of, y_of, s_of, m, op, reps)
        timings[f"n{key[0]}-a{key[1]}->{int(trial[key])}"] = ms
        if ms < best_ms * (1.0 - gain):
            table, best_ms = trial, ms
    return table, timings, best_ms


class Table:
    """Persistent choices: signature -> tier settings (JSON file).  A tier
    table (per front shape) is stored as a nested list."""

    def __init__(self, path):
        self.path = path
        self.entries = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def lookup(self, sig):
        e = self.entries.get(sig)
        if not e:
            return None
        cfg = dict(e["config"])
        if "tier_table" in cfg:
            cfg["tier_table"] = np.asarray(cfg["tier_table"], dtype=np.int32)
        return cfg

    def store(self, sig, config, timings):
        cfg = dict(config)
        if "tier_table" in cfg:
            cfg["tier_table"] = np.asarray(cfg["tier_table"]).tolist()
        self.entries[sig] = {"config": cfg, "timings_ms": timings}
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def analyze_tuned(make_symbolic, m, table, op="hessian", candidates=DEFAULT_CANDIDATES, refine=False):
    """Symbolic object with the table's settings for this pattern shape,
    tuning (and recording) them first if the shape is new; with `refine`,
    the per-front-shape tier table is refined and recorded too."""
    probe = make_symbolic()
    sig = signature(probe, m)
    cfg = table.lookup(sig)
    if cfg is None:
        cfg, timings = tune(make_symbolic, m, candidates=candidates, op=op)
        if refine:
            t, trials, _ = refine_tiers(make_symbolic, cfg, m, timings[json.dumps(cfg, sort_keys=True)], op=op)
            timings = dict(timings, tier_table_trials=trials)
            if (t >= 0).any():
                cfg = dict(cfg, tier_table=t)
        table.store(sig, cfg, timings)
    return make_symbolic(**cfg), cfg, sig
