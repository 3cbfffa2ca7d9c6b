"""Autotuner for the tier cutovers of the front kernels.

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

    timings = {}
    best, best_ms = None, float("inf")
    for cfg in candidates:
        ms = _time_config(make_symbolic, cfg, x_of, y_of, s_of, m, op, reps)
        timings[json.dumps(cfg, sort_keys=True)] = ms
        if ms < best_ms:
            best, best_ms = dict(cfg), ms
    return best, timings


class Table:
    """Persistent choices: signature -> tier settings (JSON file)."""

    def __init__(self, path):
        self.path = path
        self.entries = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def lookup(self, sig):
        e = self.entries.get(sig)
        return dict(e["config"]) if e else None

    def store(self, sig, config, timings):
        self.entries[sig] = {"config": config, "timings_ms": timings}
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def analyze_tuned(make_symbolic, m, table, op="hessian", candidates=DEFAULT_CANDIDATES):
    """Symbolic object with the table's settings for this pattern shape,
    tuning (and recording) them first if the shape is new."""
    probe = make_symbolic()
    sig = signature(probe, m)
    cfg = table.lookup(sig)
    if cfg is None:
        cfg, timings = tune(make_symbolic, m, candidates=candidates, op=op)
        table.store(sig, cfg, timings)
    return make_symbolic(**cfg), cfg, sig
