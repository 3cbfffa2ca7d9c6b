"""Run the operations of the library once on a named synthetic workload, for
a profiler.

    python -m paper_1203_2742_gb300.profile_op WORKLOAD OP [--m M]

WORKLOAD: band200 (band n=200, half-bandwidth 8), er5000 (Erdos-Renyi
n=5000, p=0.001, minimum degree, relax 16), grid150 (5-point 150x150 grid,
nested dissection), dense1500 (dense 1500x1500 pattern), grid3d40 (7-point
40x40x40 grid, nested dissection), band20k_w61 (band n=20000,
half-bandwidth 61: one long chain of thin fronts), batch256 (256 independent band, arrow and
2D-grid instances, n log-uniform in [300, 30000], in one batched symbolic
object).  OP: factor, gradient, hessian,
inv_hessian, completion or all.  M: right-hand sides of the Hessian-type
operations (default: 1, 8, 64, 8, 1 for the workloads above).

Every operation runs twice as warm-up (the second round captures the CUDA
graphs of the launch sequences); then the chosen ones run once more inside
an NVTX range named "timed", so that a profiler can restrict its capture to
them (``ncu --nvtx --nvtx-include "timed/"``), each inside a nested range
named after the operation (``--nvtx-include "timed/hessian/"``).  --no-graphs launches every
kernel directly.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

from . import binding as B  # noqa: E402

DEFAULT_M = {"band200": 1, "er5000": 8, "grid150": 64, "dense1500": 8, "grid3d40": 1, "batch256": 4,
             "band20k_w61": 4}


def symbolic_for(name, **tiers):
    if name == "band200":
        return B.Symbolic(*W.band(200, 8), **tiers)
    if name == "er5000":
        return B.Symbolic(*W.erdos_renyi(5000, 0.001, np.random.default_rng(1)), ordering="mindeg", relax=16,
                          **tiers)
    if name == "grid150":
        return B.Symbolic(*W.grid2d(150, 150), **W.nd_options((150, 150)), **tiers)
    if name == "dense1500":
        return B.Symbolic(*W.band(1500, 1499), **tiers)
    if name == "grid3d40":
        return B.Symbolic(*W.grid3d(40, 40, 40), **W.nd_options((40, 40, 40)), **tiers)
    if name == "band20k_w61":
        return B.Symbolic(*W.band(20000, 61), **tiers)
    if name == "batch256":
        inst = W.batch_mix(256, 3)
        ords = [W.nd_options(W.grid_dims(k, p[0])) if k == "grid" else "natural" for p, _, k in inst]
        return B.SymbolicBatch([p for p, _, _ in inst], orderings=ords, **tiers)
    raise SystemExit(f"unknown workload {name}")


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=sorted(DEFAULT_M))
    ap.add_argument("op", choices=("factor", "gradient", "hessian", "inv_hessian", "completion", "hfactor",
                                   "hfactor_adj", "hfactor_2nz", "hfactor_2nz_sparse", "all"))
    ap.add_argument("--m", type=int, default=None)
    ap.add_argument("--no-graphs", action="store_true", help="launch every kernel directly (no CUDA graphs)")
    ap.add_argument("--big-rows", type=int, default=0, help="dense-tier cutover |J| (0: library default)")
    ap.add_argument("--big-cols", type=int, default=0, help="dense-tier cutover |N| (0: library default)")
    ap.add_argument("--split-cols", type=int, default=0, help="supernode split width (0: library default)")
    ap.add_argument("--chain-runs", type=int, default=1, choices=(0, 1),
                    help="chain tier for runs of one-column band fronts (library default: 1)")
    ap.add_argument("--tc-products", type=int, default=0, choices=(-1, 0, 1),
                    help="dense-tier products on the tensor cores: -1 never, 0 by the cost model, 1 always")
    ap.add_argument("--graph-limit", type=int, default=None,
                    help="longest launch sequence captured into a CUDA graph (library default 8192)")
    ap.add_argument("--completion", default="independent", choices=("independent", "factored"),
                    help="completion form (factored: update matrices propagated from the parents)")
    a = ap.parse_args(argv)
    m = a.m if a.m is not None else DEFAULT_M[a.workload]
    sym = symbolic_for(a.workload, big_rows=a.big_rows, big_cols=a.big_cols, split_cols=a.split_cols,
                       chain_runs=a.chain_runs, completion=a.completion, tc_products=a.tc_products)
    n, cp, ri = sym.n, sym.colptr, sym.rowind
    rng = np.random.default_rng(0)

    def dev(v):
        return torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")

    x = dev(W.diag_dominant(n, cp, ri, rng))
    ys = dev(W.uniform_sym(n, cp, ri, rng, count=m))
    s = dev(W.projected_gram(n, cp, ri, rng.standard_normal((n, 20)), 0.5))
    fac = sym.factor(x)
    g = torch.empty_like(x)
    t = torch.empty_like(ys)
    wr = torch.empty_like(ys)
    # sparse arguments (§5.5): two nonzero lower entries per Y at random positions
    y2 = np.zeros((m, sym.nnz))
    for i in range(m):
        y2[i, rng.choice(sym.nnz, size=2, replace=False)] = rng.uniform(-1.0, 1.0, size=2)
    y2 = dev(y2)
    cfac, _ = sym.complete(s)
    if a.no_graphs:
        fac.set_graphs(False)
        cfac.set_graphs(False)
    if a.graph_limit is not None:
        fac.set_graph_limit(a.graph_limit)
        cfac.set_graph_limit(a.graph_limit)
    ops = {
        "factor": lambda: fac.refactor(x),
        "gradient": lambda: fac.gradient(out=g),
        "hessian": lambda: fac.hessian(ys, out=t),
        "inv_hessian": lambda: fac.inv_hessian(ys, out=t),
        "completion": lambda: cfac.recomplete(s, want_fstar=False),
        "hfactor": lambda: fac.hessian_factor(ys, out=wr),
        "hfactor_adj": lambda: fac.hessian_factor_adj(ys, out=wr),
        "hfactor_2nz": lambda: fac.hessian_factor(y2, out=wr),
        "hfactor_2nz_sparse": lambda: fac.hessian_factor(y2, out=wr, sparse=True),
    }
    import time
    chosen = list(ops) if a.op == "all" else [a.op]
    for rnd in range(2):  # the second round captures the CUDA graphs the timed round replays
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for name in chosen:
            ops[name]()
        torch.cuda.synchronize()
        print(f"  warm-up round {rnd + 1}: {1e3 * (time.perf_counter() - t0):.1f} ms ({a.op})")
    torch.cuda.nvtx.range_push("timed")
    times = {}
    for name in chosen:
        l0 = B.chd_kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(name)  # "timed/<op>" for a profiler's per-operation filter
        e0.record()
        ops[name]()
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        times[name] = (round(e0.elapsed_time(e1), 4), B.chd_kernel_launches() - l0)
    torch.cuda.nvtx.range_pop()
    print(f"{a.workload} {a.op} m={m}: n={n} nnz={sym.nnz} supernodes={sym.nsuper}")
    for name, (ms, nl) in times.items():
        print(f"  {name:12s} {ms:10.3f} ms  {nl:8d} launches")


if __name__ == "__main__":
    main()
