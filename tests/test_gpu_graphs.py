"""CUDA graphs of the launch sequences: repeated calls with the same
arguments replay a captured graph.  Every replay must give bitwise the
results of the direct launches (the graph holds the same kernels in the same
dependency order), and the results must still match the oracle."""
import numpy as np
import pytest

from oracle import dense as OD
import workloads as W
from tests.helpers import lib

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _run_all(B, sym, x, ys, s, graphs, reps):
    """Every operation `reps` times on the same buffers; returns the results of
    each repetition and the launch counts of the last one."""
    import torch
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    xd, yd, sd = dev(x), dev(ys), dev(s)
    fac = sym.factor(xd)
    fac.set_graphs(graphs)
    cfac, _ = sym.complete(sd)
    cfac.set_graphs(graphs)
    g = torch.empty_like(xd)
    t = torch.empty_like(yd)
    yi = torch.empty_like(yd)
    w = torch.empty_like(yd)
    ta = torch.empty_like(yd)
    out = []
    for _ in range(reps):
        l0 = B.chd_kernel_launches()
        fac.refactor(xd)
        fac.gradient(out=g)
        fac.hessian(yd, out=t)
        fac.inv_hessian(yd, out=yi)
        fac.hessian_factor(yd, out=w)
        fac.hessian_factor_adj(w, out=ta)
        cfac.recomplete(sd, want_fstar=False)
        lx, dx = cfac.export()
        torch.cuda.synchronize()
        out.append(dict(logdet=fac.logdet(), g=g.cpu().numpy().copy(), t=t.cpu().numpy().copy(),
                        yi=yi.cpu().numpy().copy(), lx=lx.cpu().numpy().copy(), dx=dx.cpu().numpy().copy(),
                        w=w.cpu().numpy().copy(), ta=ta.cpu().numpy().copy(),
                        launches=B.chd_kernel_launches() - l0))
    return out


@pytest.mark.parametrize("case", ["dense_tier", "mixed_tiers"])
def test_graph_replays_are_bitwise_direct_runs(case):
    B = lib()
    rng = np.random.default_rng(71)
    if case == "dense_tier":
        sym = B.Symbolic(*W.erdos_renyi(500, 0.02, rng), ordering="mindeg", big_rows=48, big_cols=24,
                         split_cols=32)
    else:
        sym = B.Symbolic(*W.permute(W.grid2d(20, 20), W.nested_dissection((20, 20), leaf=6)))
    n, cp, ri = sym.n, sym.colptr, sym.rowind
    x = W.diag_dominant(n, cp, ri, rng)
    ys = W.uniform_sym(n, cp, ri, rng, count=3)
    s = W.projected_gram(n, cp, ri, rng.standard_normal((n, 10)), 0.5)
    direct = _run_all(B, sym, x, ys, s, graphs=False, reps=1)[0]
    replayed = _run_all(B, sym, x, ys, s, graphs=True, reps=4)
    for r in replayed:
        for key in ("g", "t", "yi", "lx", "dx", "w", "ta"):
            assert np.array_equal(r[key], direct[key]), key
        assert r["logdet"] == direct["logdet"]
    # replays count the kernels the graph runs: the same as a direct call
    assert replayed[-1]["launches"] == direct["launches"] > 0
    # and the results are the oracle's
    assert OD.rel_err(n, cp, ri, direct["g"], OD.gradient(n, cp, ri, x)) < TOL
    want = OD.hessian(n, cp, ri, x, list(ys))
    for j in range(3):
        assert OD.rel_err(n, cp, ri, direct["t"][j], want[j]) < TOL


def test_new_buffers_after_a_graph():
    """A call with other buffers runs directly and gives the right result; the
    graph of the earlier buffers is not replayed on them."""
    import torch
    B = lib()
    rng = np.random.default_rng(72)
    sym = B.Symbolic(*W.erdos_renyi(400, 0.02, rng), ordering="mindeg", big_rows=48, big_cols=24)
    n, cp, ri = sym.n, sym.colptr, sym.rowind
    x = W.diag_dominant(n, cp, ri, rng)
    ya = W.uniform_sym(n, cp, ri, rng, count=2)
    yb = W.uniform_sym(n, cp, ri, rng, count=2)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    fac = sym.factor(dev(x))
    yad, ybd = dev(ya), dev(yb)
    ta = torch.empty_like(yad)
    for _ in range(3):
        fac.hessian(yad, out=ta)
    tb = fac.hessian(ybd)
    torch.cuda.synchronize()
    wa = OD.hessian(n, cp, ri, x, list(ya))
    wb = OD.hessian(n, cp, ri, x, list(yb))
    for j in range(2):
        assert OD.rel_err(n, cp, ri, ta[j].cpu().numpy(), wa[j]) < TOL
        assert OD.rel_err(n, cp, ri, tb[j].cpu().numpy(), wb[j]) < TOL
