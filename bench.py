#!/usr/bin/env python
"""Benchmark of the hot path: factor, log det, gradient, Hessian products,
inverse-Hessian products and completion on one synthetic chordal workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload er5000|band200|grid150]

One step = one pass of every operation over one batch of inputs resident in
HBM: refactor(X), log det, gradient, Hessian of m right-hand sides, inverse
Hessian of m right-hand sides, completion of S with f_*.  The metric is
Hessian evaluations per second (m per step) over the whole job; FP64 frontal
TFLOP/s of the dominant operation (the Hessian) is reported against the
measured FP64 FMA throughput of the device.  Multi-GPU runs are independent
replicas (the path has no exchange step); rank 0 prints one JSON line.

``--impl reference`` times the CPU oracle (dense definitions, numpy/LAPACK on
all host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
os.environ.setdefault("OPENBLAS_NUM_THREADS", os.environ["OMP_NUM_THREADS"])

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "Hessian evals/s"
UNIT = "evals/s"
# parity bound of every reported GPU number: relative Frobenius error in the
# symmetric norm against the FP64 oracle (log det and f_*: |error| / max(1, |value|))
TOL_PARITY = 1e-10
# FP64 roofline of the front arithmetic: 152 SMs x 2.07 GHz x 2 FMA per clock per SM
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12
def measured_peaks():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def bf16_peak_tflops():
    """Dense bf16 tensor rate for a call timed alone: the measured burst
    figure of MEASURED_PEAKS.json, else the fallback of an earlier GB300
    measurement."""
    v = measured_peaks().get("bf16_tflops")
    return (float(v), "measured (cuBLAS bf16 GEMM, burst)") if v else (1900.0, "fallback")


# measured HBM copy bandwidth of the GB300s (generated file), else
# the fallback figure of an earlier measurement
def hbm_peak_gbs():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# DRAM bytes (read + write) of one Hessian call, summed over the call's
# launches in one ncu capture of the current kernels (dram__bytes_read.sum +
# dram__bytes_write.sum); absent where there is none.
TRAFFIC_PER_HESSIAN_CALL = {"er5000": 9.716e9}


def make_workload(name):
    """Pattern, analysis options, right-hand-side count and value recipe."""
    if name == "er5000":
        pattern = W.erdos_renyi(5000, 0.001, np.random.default_rng(1))
        return dict(name=name, pattern=pattern, opts=dict(ordering="mindeg", relax=16), m=8, seed=1,
                    gram=(50, 0.1),
                    desc="Erdos-Renyi n=5000 p=0.001, minimum-degree order, relaxed supernodes "
                         "(<=16 zeros per merge), X diag-dominant, 8 Y uniform[-1,1], "
                         "S=P(GG^T+0.1I) G 5000x50")
    if name == "band200":
        return dict(name=name, pattern=W.band(200, 8), opts=dict(), m=1, seed=0, gram=(20, 1.0),
                    desc="band n=200 half-bandwidth 8, natural order, X diag-dominant, 1 Y, "
                         "S=P(GG^T+I) G 200x20")
    if name == "batch256":
        inst = W.batch_mix(256, 3)
        return dict(name=name, batch=inst, m=4, seed=3, gram=(20, 0.5),
                    desc="256 independent instances in one batched symbolic object: n log-uniform in "
                         "[300, 30000], a third each band (half-bandwidth 4..64), block arrow (width 32), "
                         "2D grid with nested dissection; X diag-dominant, 4 Y per instance, "
                         "S=P(GG^T+0.5I) G nx20")
    if name == "serve":
        rng = np.random.default_rng(4)
        pool = []
        for i in range(31):
            n = int(round(np.exp(rng.uniform(np.log(1000), np.log(60000)))))
            kind = ("band", "arrow", "grid")[i % 3]
            if kind == "band":
                pool.append((W.band(n, int(rng.integers(4, 65))), None))
            elif kind == "arrow":
                pool.append((W.arrow(n, 32), None))
            else:
                side = max(2, int(round(np.sqrt(n))))
                pool.append((W.grid2d(side, side), (side, side)))
        pool.append((W.grid3d(40, 40, 40), (40, 40, 40)))
        return dict(name=name, pool=pool, m=16, seed=4, gram=(20, 0.5), rate=2000.0,
                    mix={"factor": 0.1, "gradient": 0.2, "hessian": 0.5, "inv_hessian": 0.1, "completion": 0.1},
                    desc="serving: Poisson 2000 req/s over 32 resident patterns (n log-uniform 1k..60k: band, "
                         "arrow, 2D ND grid; plus the 40x40x40 7-point grid under ND), mix 10% factor, 20% "
                         "gradient, 50% Hessian (m ~ U{1..16}), 10% inverse Hessian, 10% completion")
    if name == "grid150":
        return dict(name=name, pattern=W.grid2d(150, 150),
                    opts=W.nd_options((150, 150)), ref_perm=W.nested_dissection((150, 150), leaf=8), m=64, seed=2,
                    gram=(20, 0.5), small=(W.grid2d(60, 60), W.nested_dissection((60, 60), leaf=8)),
                    desc="5-point grid 150x150 (n=22500), geometric nested dissection, "
                         "X diag-dominant, 64 Y, S=P(GG^T+0.5I) G 22500x20")
    raise SystemExit(f"unknown workload {name}")


def workload_values(wl, n, cp, ri):
    rng = np.random.default_rng(wl["seed"])
    x = W.diag_dominant(n, cp, ri, rng)
    ys = W.uniform_sym(n, cp, ri, rng, count=wl["m"])
    k, c = wl["gram"]
    s = W.projected_gram(n, cp, ri, rng.standard_normal((n, k)), c)
    return x, ys, s


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_hessian_sample(wl, n, cp, ri, x, ys, count, keep=None):
    """Dense oracle: Z = X^{-1} once, then T = P(Z Y Z) for `count` of the Y's.
    Returns (t_inverse, t_per_eval); with a dict `keep`, also stores Z and
    the T's in it (for the accuracy record)."""
    from oracle import dense as OD
    t0 = time.perf_counter()
    Z = OD.inverse(n, cp, ri, x)
    t1 = time.perf_counter()
    T = OD.hessian(n, cp, ri, x, list(ys[:count]), Z=Z)
    t2 = time.perf_counter()
    if keep is not None:
        keep["Z"], keep["T"] = Z, T
    return t1 - t0, (t2 - t1) / count


def oracle_hessian_repeated(wl, n, cp, ri, x, ys, count, budget_s=10.0, keep=None):
    """``oracle_hessian_sample`` repeated until `budget_s` seconds of CPU work
    are spent (at least once); medians of (t_inverse, t_per_eval) and the
    number of repetitions.  A small pattern takes milliseconds per sample,
    where one timing is mostly noise."""
    tz, te, spent = [], [], 0.0
    while spent < budget_s or not tz:
        a, b = oracle_hessian_sample(wl, n, cp, ri, x, ys, count, keep=keep)
        tz.append(a)
        te.append(b)
        spent += a + count * b
    return float(np.median(tz)), float(np.median(te)), len(tz)


def batch_cpu_baseline(sym, x, ys, m, cores, budget_s=15.0):
    """Dense oracle on the smallest instances of a batch (within a time budget),
    extrapolated to every instance by the oracle's n^3 cost."""
    from oracle import dense as OD
    order = np.argsort(np.diff(sym.n_off))
    spent, done, coef = 0.0, 0, []
    for i in order:
        (ni, cpi, rii), _ = sym.instance_pattern(int(i))
        z0, z1 = int(sym.nnz_off[i]), int(sym.nnz_off[i + 1])
        t0 = time.perf_counter()
        Z = OD.inverse(ni, cpi, rii, x[z0:z1])
        OD.hessian(ni, cpi, rii, x[z0:z1], list(ys[:, z0:z1]), Z=Z)
        dt = time.perf_counter() - t0
        spent += dt
        done += 1
        coef.append(dt / float(ni) ** 3)
        if spent > budget_s:
            break
    c = float(np.median(coef))
    total = sum(c * float(v) ** 3 for v in np.diff(sym.n_off))
    return {"value": sym.count * m / total, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"dense oracle (X^-1, then P(X^-1 Y X^-1) for the {m} Y) on the {done} smallest of "
                      f"{sym.count} instances ({spent:.1f} s); extrapolated to all instances by n^3"}


def oracle_pattern(pattern, perm=None, snode_ptr=None):
    """The analysed pattern V computed by the oracle alone (no library): the
    pattern permuted by perm (perm[new] = old), filled by the oracle's
    elimination fill, and -- for a stored relaxed partition -- its
    supernodal pattern.  For the Erdos-Renyi workload the stored analysis
    reproduces the library's V exactly (host test); for the others this is
    the same filled graph in the oracle's own numbering (the library also
    postorders it), which draws the same value recipe on the same shape."""
    from oracle import symbolic as OS
    n = int(pattern[0])
    p = W.permute(pattern, perm) if perm is not None else pattern
    I, _ = OS.fill(n, OS.columns_from_csc(*p))
    sp = np.arange(n + 1) if snode_ptr is None else snode_ptr
    cp, ri = OS.supernodal_pattern(n, I, sp)
    return n, cp, ri


def reference_pattern(wl):
    if wl["name"] == "er5000":
        from workloads import analysed
        pattern, perm, sp = analysed.load_er5000()
        return oracle_pattern(pattern, perm, sp)
    return oracle_pattern(wl["pattern"], wl.get("ref_perm"))


class OracleBatch:
    """Block-diagonal union of independently analysed instances, in the
    oracle's numbering (the reference arm's stand-in for the library's
    batched symbolic object: the same attributes the CPU baseline reads)."""

    def __init__(self, instances):
        self.parts = [oracle_pattern(p, q) for p, q, _ in instances]
        self.count = len(self.parts)
        ns = [p[0] for p in self.parts]
        zs = [len(p[2]) for p in self.parts]
        self.n_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
        self.nnz_off = np.concatenate([[0], np.cumsum(zs)]).astype(np.int64)
        self.n = int(self.n_off[-1])
        self.colptr = np.concatenate([[0]] + [p[1][1:] + self.nnz_off[i] for i, p in enumerate(self.parts)])
        self.rowind = np.concatenate([p[2] + self.n_off[i] for i, p in enumerate(self.parts)]).astype(np.int32)
        self.nnz = int(self.nnz_off[-1])

    def instance_pattern(self, i):
        return self.parts[i], None


def run_reference(args, wl):
    """The CPU oracle on the host cores, on the same workload; loads no part
    of the library (the analysed pattern comes from the oracle, see
    ``oracle_pattern``)."""
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    if "batch" in wl:
        sym = OracleBatch(wl["batch"])
        x, ys, _ = workload_values(wl, sym.n, sym.colptr, sym.rowind)
        times, cpu = [], None
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            cpu = batch_cpu_baseline(sym, x, ys, wl["m"], cores, budget_s=5.0)
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
        line = {"metric": METRIC, "value": cpu["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": float(np.mean(times)) * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": wl["desc"], "global_batch": sym.count * wl["m"], "parallelism": "host cores"},
                "cpu_baseline": cpu,
                "e2e": {"value": cpu["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if wl["name"] == "serve":
        # the serving trace's Hessian requests, timed on the oracle: the same
        # pool, rate, mix and seed as the GPU arm (request values are not
        # drawn here, so the request list is a draw of the same process, not
        # the identical list)
        from types import SimpleNamespace
        from paper_1203_2742_gb300 import serve  # host logic only (no library)
        pool = []
        for (pat, dims) in wl["pool"]:
            n, cp, ri = oracle_pattern(pat, None if dims is None else W.nested_dissection(dims, leaf=8))
            sym = SimpleNamespace(n=n, colptr=cp, rowind=ri, nnz=len(ri))
            x, _, s_ = workload_values(dict(wl, m=1), n, cp, ri)
            pool.append((sym, x, s_))
        trace = serve.poisson_trace(len(pool), wl["rate"], args.serve_seconds, wl["mix"],
                                    np.random.default_rng(wl["seed"]), lambda i: 0, max_m=wl["m"])
        times, cpu = [], None
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            cpu = serve_cpu_baseline(pool, trace, cores, budget_s=5.0)
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
        line = {"metric": METRIC, "value": cpu["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": float(np.mean(times)) * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": wl["desc"], "trace_seconds": args.serve_seconds, "requests": len(trace),
                           "patterns": len(pool), "parallelism": "host cores"},
                "cpu_baseline": cpu,
                "e2e": {"value": cpu["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    n, cp, ri = reference_pattern(wl)
    x, ys, _ = workload_values(wl, n, cp, ri)
    m = wl["m"]
    sample_evals = min(2, m)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        tz, te = oracle_hessian_sample(wl, n, cp, ri, x, ys, sample_evals)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append((dt, tz, te))
    step = float(np.mean([t[0] for t in times]))
    tz = float(np.mean([t[1] for t in times]))
    te = float(np.mean([t[2] for t in times]))
    value = m / (tz + m * te)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": wl["desc"], "n": n, "nnz_filled": int(len(ri)), "rhs_per_step": m,
                   "global_batch": m, "parallelism": "host cores", "l2": "host run"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"dense oracle: X^-1 then P(X^-1 Y X^-1) for {sample_evals} of the "
                                   f"{m} Y per step; value = {m}/(t_inverse + {m}*t_eval)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def scaled_cpu_baseline(wl, n, cores, budget_s=10.0):
    """Dense oracle timed on a smaller instance of the same recipe (the
    workload's "small" pattern, analysed by the oracle alone), extrapolated
    to the full pattern by the dense oracle's n^3 cost: for patterns whose
    dense X^{-1} does not fit a bounded sample."""
    pat, perm = wl["small"]
    ns, cps, ris = oracle_pattern(pat, perm)
    xs_, ys_, _ = workload_values(dict(wl, m=2), ns, cps, ris)
    tz, te, reps = oracle_hessian_repeated(wl, ns, cps, ris, xs_, ys_, 2, budget_s=budget_s)
    f = (float(n) / ns) ** 3
    m = wl["m"]
    return {"value": m / (f * (tz + m * te)), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"dense oracle X^-1 ({tz:.3g} s) and P(X^-1 Y X^-1) ({te:.3g} s per Y) on the same recipe at "
                      f"n = {ns} ({reps} repetitions), extrapolated by (n/{ns})^3 = {f:.0f} to n = {n}; "
                      f"value = {m}/(t_inverse + {m}*t_eval)"}


def make_symbolic(B, wl, **cfg):
    if "batch" in wl:
        inst = wl["batch"] if "subset" not in cfg else [wl["batch"][i] for i in cfg.pop("subset")]
        pats = [p for p, _, _ in inst]
        ords = []
        for p, _, kind in inst:
            dims = W.grid_dims(kind, p[0])
            ords.append(W.nd_options(dims) if dims else "natural")
        return B.SymbolicBatch(pats, orderings=ords, **cfg)
    return B.Symbolic(*wl["pattern"], **wl["opts"], **cfg)


def tuned_config(B, wl):
    """Tier cutovers chosen by the autotuner on the benchmark step itself
    (every operation with the workload's m): on every 8th instance of a
    batch, else on the pattern itself; then, for a single pattern, the
    per-front-shape tier table refined from them."""
    from paper_1203_2742_gb300 import autotune
    if "batch" in wl:
        subset = list(range(0, len(wl["batch"]), 8))
        mk = lambda **c: make_symbolic(B, wl, subset=subset, **c)
        cfg, timings = autotune.tune(mk, wl["m"], op="step", reps=1)
        cfg, tc_ms = autotune.refine_tc(mk, cfg, wl["m"], timings[json.dumps(cfg, sort_keys=True)], reps=1)
        return cfg, dict(timings, fp64_units_only_trial=tc_ms)
    mk = lambda **c: make_symbolic(B, wl, **c)
    cfg, timings = autotune.tune(mk, wl["m"], op="step", reps=2)
    base = timings[json.dumps(cfg, sort_keys=True)]
    table, trials, best = autotune.refine_tiers(mk, cfg, wl["m"], base)
    timings = dict(timings, tier_table_trials=trials)
    if (table >= 0).any():
        cfg = dict(cfg, tier_table=table)
        base = best
    cfg, tc_ms = autotune.refine_tc(mk, cfg, wl["m"], base)
    return cfg, dict(timings, fp64_units_only_trial=tc_ms)


# ---------------------------------------------------------------------------
# replicas: every rank runs the whole step on its own GPU (the path has no
# exchange step); the job's time is the slowest rank's
# ---------------------------------------------------------------------------

def hbm_line(bytes_per_call, ms):
    peak, src = hbm_peak_gbs()
    gbs = bytes_per_call / (ms * 1e-3) / 1e9
    return {"algorithmic_bytes_per_call": bytes_per_call, "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak, "peak_source": src}


def replica_max_ms(dev_ms, device):
    """Max over the ranks of the timed region's device milliseconds."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return dev_ms
    t = torch.tensor([dev_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_value(world, evals_per_step, steps, max_ms):
    """Whole-job throughput: every replica's evaluations over the slowest time."""
    return world * evals_per_step * steps / (max_ms * 1e-3)


def accuracy_record(n, cp, ri, keep, ys, s, g, t, yi, logdet, fstar, xhat, x):
    """Errors of the GPU outputs of the last end-to-end step against the FP64
    oracle, on the CPU-baseline sample: the Hessian of the sampled Y's and
    the gradient against the dense X^{-1} of the timed sample; log det
    against the dense Cholesky factor; the inverse Hessian of the sampled
    T = H(Y) against the oracle's clique-sum H^{-1}, and the round trip
    H^{-1}(H(Y)) = Y for every Y; the completion X-hat against the oracle's
    (the clique-sum closed form refined by Newton steps until Eq.
    (e-Xhat-eq) holds to rounding), and f_* against log det X-hat - n.
    Relative Frobenius errors in the symmetric norm.  The residual of
    P(X-hat^{-1}) = S is reported too but not gated: it amplifies the error
    of X-hat by about cond(X-hat)."""
    from oracle import dense as OD
    from oracle import symbolic as OS
    err = lambda a, b: float(OD.rel_err(n, cp, ri, a, b))
    Z, T = keep["Z"], keep["T"]
    k = len(T)
    I = [np.asarray(ri[cp[j] + 1:cp[j + 1]], dtype=np.int64) for j in range(n)]
    cl, seps = OS.cliques_and_separators(I, OS.etree(I))
    want_ld = OD.logdet(n, cp, ri, x)
    Xh = OD.to_dense(n, cp, ri, xhat)
    ld_xh = float(2.0 * np.sum(np.log(np.diag(np.linalg.cholesky(Xh)))))
    rec = {
        "tolerance": TOL_PARITY,
        "logdet": abs(logdet - want_ld) / max(1.0, abs(want_ld)),
        "gradient": err(g, -OD.project(n, cp, ri, Z)),
        "hessian": max(err(t[i], T[i]) for i in range(k)),
        "inv_hessian": max(err(yi[i], OD.inv_hessian_cliquesum(n, cp, ri, x, t[i], cl, seps, S=Z))
                           for i in range(k)),
        "inv_hessian_roundtrip": max(err(yi[i], ys[i]) for i in range(len(ys))),
        "completion": err(xhat, OD.completion_refined(n, cp, ri, s, cl, seps)),
        "fstar": abs(fstar - (ld_xh - n)) / max(1.0, abs(fstar)),
        "sample": f"Hessian and inverse Hessian of {k} of the {len(ys)} right-hand sides; round trip of all",
    }
    rec["pass"] = all(v <= TOL_PARITY for key, v in rec.items() if key not in ("tolerance", "sample"))
    rec["completion_residual"] = err(OD.project(n, cp, ri, np.linalg.inv(Xh)), s)
    return rec


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, wl, rank, world, local_rank):
    import torch
    from paper_1203_2742_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        build.build()
    from paper_1203_2742_gb300 import binding as B

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()

    tune = None
    cfg = {}
    if args.tiers:
        cfg = dict(big_rows=args.tiers[0], big_cols=args.tiers[1], split_cols=args.tiers[2])
        tune = {"chosen": cfg, "timings_ms": None, "on": "given on the command line"}
    elif not args.no_tune:
        cfg, timings = tuned_config(B, wl)
        chosen = {k: v for k, v in cfg.items() if k != "tier_table"}
        if "tier_table" in cfg:
            t_ = cfg["tier_table"]
            chosen["tier_table"] = {f"n{i}-a{j}": int(t_[i, j]) for i, j in zip(*np.nonzero(t_ >= 0))}
        tune = {"chosen": chosen, "timings_ms": timings,
                "on": ("every 8th instance" if "batch" in wl else "the pattern") + ", the whole step with the same m"}
    t0 = time.perf_counter()
    sym = make_symbolic(B, wl, **cfg)
    analyze_ms = (time.perf_counter() - t0) * 1e3
    count = getattr(sym, "count", 1)
    n, cp, ri, nnz = sym.n, sym.colptr, sym.rowind, sym.nnz
    m = wl["m"]
    x, ys, s = workload_values(wl, n, cp, ri)
    # the method's flops are counted on the relaxed Algorithm 6.1 partition;
    # splitting wide supernodes (a scheduling choice) executes more
    fl_exec = sym.flops()
    fl = make_symbolic(B, wl, **dict({k: v for k, v in cfg.items() if k != "tier_table"}, split_cols=-1)).flops()

    # inputs resident in HBM
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    X, Y, S = d(x), d(ys), d(s)
    G = torch.empty(nnz, dtype=torch.float64, device=dev)
    T = torch.empty((m, nnz), dtype=torch.float64, device=dev)
    YI = torch.empty((m, nnz), dtype=torch.float64, device=dev)
    fac = sym.factor(X)
    fx, _ = sym.complete(S)
    # every step repeats its calls on the same buffers: capture even long
    # launch sequences (the batch's calls hold 11-26 thousand launches)
    fac.set_graph_limit(1 << 20)
    fx.set_graph_limit(1 << 20)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dev)  # > L2

    results = {}
    # the dual side of the step (the completion of S and f*) does not depend
    # on the primal chain (factor, gradient, Hessian, inverse Hessian of X):
    # it runs on a second stream, forked at the step's start and joined
    # before its end, and fills the SMs the primal chain leaves idle
    side = torch.cuda.Stream(device=dev)
    fork, join = torch.cuda.Event(), torch.cuda.Event()

    def step():
        fork.record(stream)
        side.wait_event(fork)
        fx.recomplete(S, want_fstar=False, stream=side)
        fac.refactor(X)
        results["logdet"] = float(np.sum(fac.logdet_batch())) if count > 1 else fac.logdet()
        fac.gradient(out=G)
        fac.hessian(Y, out=T)
        fac.inv_hessian(T, out=YI)
        results["fstar"] = fx.logdet() - n
        join.record(side)
        stream.wait_event(join)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps ----
    sampler = ClockSampler(local_rank)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = B.chd_kernel_launches()
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler capture the timed steps only
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - wall0
    launches = B.chd_kernel_launches() - launches0
    clocks = sampler.stop()
    dev_ms = replica_max_ms(sum(a.elapsed_time(b) for a, b in evs), dev)
    ms_per_step = dev_ms / args.steps
    evals_per_step = count * m  # one Hessian evaluation = one Y of one instance
    value = job_value(world, evals_per_step, args.steps, dev_ms)

    # ---- per-operation breakdown and the dominant kernel's roofline ----
    def time_op(fn, reps):
        es = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        tot = 0.0
        for a, b in es:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in es) / reps

    reps = max(1, min(args.steps, 3))
    ops_ms = {
        "factor": time_op(lambda: fac.refactor(X), reps),
        "gradient": time_op(lambda: fac.gradient(out=G), reps),
        "hessian": time_op(lambda: fac.hessian(Y, out=T), reps),
        "inv_hessian": time_op(lambda: fac.inv_hessian(T, out=YI), reps),
        "completion": time_op(lambda: fx.recomplete(S, want_fstar=False), reps),
    }
    # ---- the two completion forms (chd_opts.completion): independent fronts
    # (the step above) and factored update matrices (Algorithm 4.3) ----
    sym_f = make_symbolic(B, wl, **dict(cfg, completion="factored"))
    fxf, _ = sym_f.complete(S)
    for _ in range(2):
        fxf.recomplete(S, want_fstar=False)
    fact_ms = time_op(lambda: fxf.recomplete(S, want_fstar=False), reps)
    xf, xi = fxf.product(), fx.product()
    cflops = sym_f.completion_flops()
    completion_forms = {
        "independent_ms": ops_ms["completion"], "factored_ms": fact_ms,
        "flops_chol_v": cflops["independent"], "flops_factored_propagation": cflops["factored"],
        "propagation_levels": cflops["levels"],
        "xhat_rel_diff": float(torch.linalg.vector_norm(xf - xi) / torch.linalg.vector_norm(xi)),
        "note": "flops: the part the forms do differently (Cholesky of every V_k against the propagation of "
                "V_k = R_k R_k^T from the parent); the rest of the completion is common",
    }
    del fxf, sym_f, xf, xi
    fp64_peak = B.chd_probe_fp64_peak() / 1e3  # TFLOP/s
    hess_flops = fl["hessian"] * m
    achieved = hess_flops / (ops_ms["hessian"] * 1e-3) / 1e12
    executed = fl_exec["hessian"] * m
    # bf16 tensor-core flops of one Hessian call, counted on a direct run (the
    # library counts the MMAs of the products it issues; graph replays are not
    # counted), and the tensor side of the roofline
    fac.set_graphs(False)
    tc0 = B.chd_tc_flops()
    fac.hessian(Y, out=T)
    torch.cuda.synchronize()
    tc_per_call = B.chd_tc_flops() - tc0
    fac.set_graphs(True)
    bf16_peak, bf16_src = bf16_peak_tflops()
    tc_achieved = tc_per_call / (ops_ms["hessian"] * 1e-3) / 1e12
    step_flops = fl["factor"] + fl["gradient"] + m * (fl["hessian"] + fl["inv_hessian"]) + fl["completion"]

    # ---- batched vs one instance at a time (the plain GPU path) ----
    sequential = None
    if count > 1:
        singles = []
        for i in range(count):
            (ni, cpi, rii), permi = sym.instance_pattern(i)
            si = B.Symbolic(ni, cpi, rii)  # already analysed: natural order keeps it
            z0, z1 = int(sym.nnz_off[i]), int(sym.nnz_off[i + 1])
            fi = si.factor(X[z0:z1].contiguous())
            fi.gradient()
            singles.append((si, fi, Y[:, z0:z1].contiguous(), torch.empty((m, z1 - z0), dtype=torch.float64, device=dev)))
        torch.cuda.synchronize()

        def seq_hessians():
            for si, fi, yi, ti in singles:
                fi.hessian(yi, out=ti)
        seq_hessians()
        torch.cuda.synchronize()
        seq_ms = time_op(seq_hessians, 1)
        sequential = {"hessian_ms_one_at_a_time": seq_ms, "hessian_ms_batched": ops_ms["hessian"],
                      "evals_per_s_one_at_a_time": evals_per_step / (seq_ms * 1e-3),
                      "evals_per_s_batched_hessian_only": evals_per_step / (ops_ms["hessian"] * 1e-3)}
        del singles

    # ---- end to end through the C ABI with host buffers ----
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).pin_memory()
    hX, hY, hS = pin(x), pin(ys), pin(s)
    hG = torch.empty(nnz, dtype=torch.float64).pin_memory()
    hT = torch.empty((m, nnz), dtype=torch.float64).pin_memory()
    hYI = torch.empty((m, nnz), dtype=torch.float64).pin_memory()

    def e2e_step():
        X.copy_(hX, non_blocking=True)
        Y.copy_(hY, non_blocking=True)
        S.copy_(hS, non_blocking=True)
        step()
        hG.copy_(G, non_blocking=True)
        hT.copy_(T, non_blocking=True)
        hYI.copy_(YI, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    eev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in eev:
        flush.zero_()
        a.record(stream)
        e2e_step()
        b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(b) for a, b in eev)
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    e2e_value = world * evals_per_step * args.steps / (e2e_ms * 1e-3)
    h2d = 8 * (x.size + ys.size + s.size)
    d2h = 8 * (nnz + 2 * m * nnz)

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only) ----
    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        if count > 1:
            cpu = batch_cpu_baseline(sym, x, ys, m, cores)
        elif "small" in wl:
            cpu = scaled_cpu_baseline(wl, n, cores)
        else:
            sample = min(2, m)
            keep = {}
            tz, te, reps = oracle_hessian_repeated(wl, n, cp, ri, x, ys, sample, keep=keep)
            cpu = {"value": m / (tz + m * te), "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"dense oracle X^-1 ({tz:.3g} s) then P(X^-1 Y X^-1) for {sample} of the {m} Y "
                             f"({te:.3g} s each), medians of {reps} repetitions (>= 10 s of CPU work or one); "
                             f"value = {m}/(t_inverse + {m}*t_eval)"}
            xhat = fx.product().cpu().numpy()
            accuracy = accuracy_record(n, cp, ri, keep, ys, s, hG.numpy(), hT.numpy(), hYI.numpy(),
                                       results["logdet"], results["fstar"], xhat, x)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "n": n, "nnz_filled": nnz,
                       "rhs_per_step": m, "global_batch": world * evals_per_step,
                       "streams": "primal chain on the caller's stream, completion + f* on a second stream",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "flushed between timed steps (256 MB write)"},
            "supernodes": sym.nsuper,
            "roofline": {"bound": "tensor",
                         "kernel": "one Hessian call (all its launches; its large products run on the tensor cores "
                                   "as FP64-accurate bf16 digit products)",
                         "achieved": tc_achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                         "frac": tc_achieved / bf16_peak, "traffic": TRAFFIC_PER_HESSIAN_CALL.get(wl["name"]),
                         "peak_source": bf16_src,
                         "tc_flops_per_call": tc_per_call,
                         "tc_flops_source": "bf16 MMA flops the call's tensor-core products execute "
                                            "(36 digit pairs per output tile), counted by the library",
                         "fp64_equivalent": {
                             "achieved": achieved, "unit": "TFLOP/s", "flops_per_call": hess_flops,
                             "flops_source": "sum over the fronts of the relaxed Algorithm 6.1 partition (unsplit) "
                                             "of 6a^2n + 8an^2 + 2n^3 per right-hand side, times m",
                             "executed_flops_per_call": executed,
                             "fp64_peak": FP64_PEAK_TFLOPS, "frac_of_fp64_peak": achieved / FP64_PEAK_TFLOPS,
                             "fp64_peak_source": "FP64 FMA rate from unit counts and clock: 152 SMs x 2070 MHz x "
                                                 "4 flop/clk",
                             "fp64_probe": fp64_peak, "frac_of_fp64_probe": achieved / fp64_peak}},
            "cpu_baseline": cpu,
            "accuracy": accuracy,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "ops_ms": {k: round(v, 4) for k, v in ops_ms.items()},
            # every operation in evals/s (Hessian-type calls: m evaluations per call)
            "ops_evals_per_s": {k: (count * m if k in ("hessian", "inv_hessian") else count) / (v * 1e-3)
                                for k, v in ops_ms.items()},
            # the memory side of the roofline: algorithmic bytes of one Hessian call (Y read and
            # T written, m matrices on V, plus one read of the factor's L and S) over its time
            "hbm": hbm_line(8.0 * (2 * m * nnz + 2 * nnz), ops_ms["hessian"]),
            "instances": count,
            "completion_forms": completion_forms,
            "autotune": tune,
            "batched_vs_one_at_a_time": sequential,
            "step_tflops_fp64_equivalent": step_flops / (ms_per_step * 1e-3) / 1e12,
            "analyze_ms": analyze_ms,
            "wall_s": wall,
            "logdet": results.get("logdet"), "fstar": results.get("fstar"),
        }
        return line
    return None


def serve_cpu_baseline(pool, trace, cores, budget_s=15.0):
    """Dense oracle Hessian evaluations on the smallest patterns of the pool
    (X^{-1} cached per pattern, as a server would), extrapolated by n^3 to the
    trace's Hessian requests."""
    from oracle import dense as OD
    order = sorted(range(len(pool)), key=lambda i: pool[i][0].n)
    coef, spent, done = [], 0.0, 0
    for i in order:
        sym, x, _ = pool[i]
        y = np.random.default_rng(i).uniform(-1.0, 1.0, size=sym.nnz)
        Z = OD.inverse(sym.n, sym.colptr, sym.rowind, x)
        t0 = time.perf_counter()
        OD.hessian(sym.n, sym.colptr, sym.rowind, x, [y], Z=Z)
        dt = time.perf_counter() - t0
        spent += dt
        done += 1
        coef.append(dt / float(sym.n) ** 3)
        if spent > budget_s or done >= 4:
            break
    c = float(np.median(coef))
    evals = sum(r.m for r in trace if r.op == "hessian")
    secs = sum(r.m * c * float(pool[r.pattern][0].n) ** 3 for r in trace if r.op == "hessian")
    return {"value": evals / secs if secs > 0 else None, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"dense oracle P(X^-1 Y X^-1) on the {done} smallest of {len(pool)} patterns "
                      f"(X^-1 cached per pattern), extrapolated by n^3 to the trace's {evals} Hessian evaluations"}


def run_serve(args, wl):
    """Serving benchmark: the same bounded Poisson trace served with continuous
    batching on 8 streams and replayed one request at a time."""
    import torch
    from paper_1203_2742_gb300 import build
    build.build()
    from paper_1203_2742_gb300 import binding as B
    from paper_1203_2742_gb300 import serve
    t0 = time.perf_counter()
    pool = []
    for (pat, dims) in wl["pool"]:
        sym = B.Symbolic(*pat, **W.nd_options(dims)) if dims is not None else B.Symbolic(*pat)
        x, _, s = workload_values(dict(wl, m=1), sym.n, sym.colptr, sym.rowind)
        pool.append((sym, x, s))
    analyze_s = time.perf_counter() - t0
    rng = np.random.default_rng(wl["seed"])
    duration = args.serve_seconds
    trace = serve.poisson_trace(len(pool), wl["rate"], duration, wl["mix"], rng, lambda i: pool[i][0].nnz,
                                max_m=wl["m"])
    launches0 = B.chd_kernel_launches()
    # served: continuous batching on 8 streams; one at a time: each request
    # alone on the same path
    srv = serve.Server(pool, workers=8, batching=True)
    srv.warm()
    sampler = ClockSampler(0)
    sampler.start()
    stats, done = serve.replay(srv, trace)
    clocks = sampler.stop()
    launches = B.chd_kernel_launches() - launches0
    srv.free()
    srv = None
    import gc
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    one = serve.Server(pool, workers=1, batching=False)
    one.warm()
    trace2 = [serve.Request(op=r.op, pattern=r.pattern, arrival=r.arrival, data=r.data, m=r.m, rid=r.rid)
              for r in trace]
    stats1, _ = serve.replay(one, trace2)
    h2d = sum(8 * r.m * pool[r.pattern][0].nnz for r in trace if r.op in ("hessian", "inv_hessian"))
    cpu = None if args.no_cpu_baseline else serve_cpu_baseline(pool, trace, os.cpu_count() or 1)
    line = {
        "metric": METRIC, "value": stats["hessian_evals_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": 1, "warmup": args.warmup, "ms_per_step": stats["wall_s"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "trace_seconds": duration, "requests": len(trace),
                   "patterns": len(pool), "workers": 8, "parallelism": "single GPU"},
        "served": stats, "one_at_a_time": stats1,
        "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"],
        "e2e": {"value": stats["hessian_evals_per_s"], "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(h2d)},
        "roofline": None, "cpu_baseline": cpu, "gpu_launches": int(launches), "clocks": clocks,
        "analyze_s": analyze_s,
    }
    print(json.dumps(line), flush=True)


OTHER_KEYS = ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "higher_is_better", "dtype", "config",
              "roofline", "cpu_baseline", "accuracy", "e2e", "gpu_launches", "clocks", "ops_ms", "ops_evals_per_s",
              "autotune", "batched_vs_one_at_a_time", "instances", "completion_forms")


def other_workloads(args, rank, world, local_rank):
    """The 150 x 150 grid (64 right-hand sides) and the 256-instance batch,
    measured in the same run with fewer timed steps, as nested records."""
    import copy
    import gc
    import torch
    out = {}
    for name, steps in (("grid150", 3), ("batch256", 2)):
        a = copy.copy(args)
        a.steps, a.warmup = steps, 3
        try:
            line = run_ours(a, make_workload(name), rank, world, local_rank)
            out[name] = {k: line.get(k) for k in OTHER_KEYS}
        except Exception as e:  # a nested record must not cost the default line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        gc.collect()
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="er5000", choices=["er5000", "band200", "grid150", "batch256", "serve"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="library default tier cutovers instead of the autotuner's")
    ap.add_argument("--tiers", type=int, nargs=3, metavar=("BIG_ROWS", "BIG_COLS", "SPLIT_COLS"), default=None,
                    help="fixed tier cutovers and split width instead of the autotuner's")
    ap.add_argument("--serve-seconds", type=float, default=0.5, help="trace length of the serve workload")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the nested records of the grid and batch workloads (default line only)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    wl = make_workload(args.workload)
    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, wl)
        return
    if "pool" in wl:
        if rank == 0:
            run_serve(args, wl)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        line = run_ours(args, wl, rank, world, local_rank)
        if line is not None and world == 1 and args.workload == "er5000" and not args.no_others:
            line["other_workloads"] = other_workloads(args, rank, world, local_rank)
        if line is not None:
            print(json.dumps(line), flush=True)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
