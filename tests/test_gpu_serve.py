"""Serving: each request's result is the same when it runs alone and when it
runs in a concurrent, continuously batched mix."""
import numpy as np
import pytest

from oracle import dense as OD
import workloads as W
from tests.helpers import lib

pytestmark = pytest.mark.gpu


def _pool(rng):
    B = lib()
    pats = [(W.band(300, 6), {}), (W.permute(W.grid2d(20, 20), W.nested_dissection((20, 20), leaf=6)), {}),
            (W.arrow(250, 40), {}), (W.erdos_renyi(200, 0.03, rng), dict(ordering="mindeg"))]
    pool = []
    for p, kw in pats:
        sym = B.Symbolic(*p, **kw)
        x = W.diag_dominant(sym.n, sym.colptr, sym.rowind, rng)
        s = W.projected_gram(sym.n, sym.colptr, sym.rowind, rng.standard_normal((sym.n, 6)), 0.5)
        pool.append((sym, x, s))
    return pool


@pytest.mark.parametrize("rhs_block", [None, 4])
def test_results_same_alone_and_in_the_mix(rhs_block):
    """In the mix (6 streams, batching; with rhs_block, calls of a fixed
    shape through kept buffers, replayed from CUDA graphs after their second
    call) every result equals the same request served alone on the plain
    path, and the Hessians equal the oracle's."""
    from paper_1203_2742_gb300 import serve
    rng = np.random.default_rng(51)
    pool = _pool(rng)
    mix = {"factor": 0.1, "gradient": 0.2, "hessian": 0.5, "inv_hessian": 0.1, "completion": 0.1}
    trace = serve.poisson_trace(len(pool), 4000.0, 0.05, mix, rng, lambda i: pool[i][0].nnz, max_m=6)
    assert len(trace) > 100
    # in the mix: 6 streams, batching, everything submitted in a burst
    srv = serve.Server(pool, workers=6, batching=True, rhs_block=rhs_block)
    srv.warm()
    for r in trace:
        r.arrival = 0.0
    stats, done = serve.replay(srv, trace)
    assert stats["requests"] == len(trace)
    assert stats["mean_batch"] > 1.0  # some Hessian requests were merged
    # alone: one worker, no batching, one request at a time
    alone = serve.Server(pool, workers=1, batching=False)
    alone.warm()
    for r in trace:
        solo = serve.Request(op=r.op, pattern=r.pattern, arrival=0.0, data=r.data, m=r.m, rid=r.rid)
        alone.run(solo)
        a, b = np.asarray(solo.result, dtype=np.float64), np.asarray(r.result, dtype=np.float64)
        assert a.shape == b.shape, r.op
        if r.op in ("hessian", "inv_hessian"):
            sym = pool[r.pattern][0]
            for j in range(r.m):
                assert OD.rel_err(sym.n, sym.colptr, sym.rowind, b[j], a[j]) < 1e-12, (r.op, r.rid)
        else:
            np.testing.assert_allclose(b, a, rtol=1e-12, atol=0)
    # and the Hessian results are the oracle's
    for r in done[:40]:
        if r.op == "hessian":
            sym, x, _ = pool[r.pattern]
            want = OD.hessian(sym.n, sym.colptr, sym.rowind, x, list(r.data))
            for j in range(r.m):
                assert OD.rel_err(sym.n, sym.colptr, sym.rowind, r.result[j], want[j]) < 1e-10
