"""Many independent patterns in one symbolic object (chd_analyze_batch): the
fronts of all instances share each level's launches.  Every operation must
give, per instance, the oracle's result and exactly the result of running
that instance alone."""
import numpy as np
import pytest

from oracle import dense as OD
from oracle import symbolic as OS
import workloads as W
from tests.helpers import lib

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _instances():
    rng = np.random.default_rng(41)
    pats = [W.band(120, 6), W.arrow(90, 8), W.permute(W.grid2d(12, 12), W.nested_dissection((12, 12), leaf=6)),
            W.erdos_renyi(150, 0.03, rng), W.band(40, 39), W.band(30, 1)]
    ords = ["natural", "natural", "natural", "mindeg", "natural", "natural"]
    return pats, ords


def test_batch_matches_oracle_and_single_runs():
    import torch
    B = lib()
    pats, ords = _instances()
    sb = B.SymbolicBatch(pats, orderings=ords)
    rng = np.random.default_rng(42)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    m = 3
    x = W.diag_dominant(sb.n, sb.colptr, sb.rowind, rng)
    ys = W.uniform_sym(sb.n, sb.colptr, sb.rowind, rng, count=m)
    s = W.projected_gram(sb.n, sb.colptr, sb.rowind, rng.standard_normal((sb.n, 8)), 0.5)
    f = sb.factor(dev(x))
    ld = f.logdet_batch()
    g = f.gradient().cpu().numpy()
    t = f.hessian(dev(ys)).cpu().numpy()
    yi = f.inv_hessian(dev(ys)).cpu().numpy()
    fx, fstar = sb.complete(dev(s))
    ldx = fx.logdet_batch()
    lx, dx = fx.export()
    lx = lx.cpu().numpy()
    torch.cuda.synchronize()
    for i, (p, o) in enumerate(zip(pats, ords)):
        (ni, cp, ri), _ = sb.instance_pattern(i)
        z0, z1 = int(sb.nnz_off[i]), int(sb.nnz_off[i + 1])
        xi, ysi, si = x[z0:z1], ys[:, z0:z1], s[z0:z1]
        err = lambda a, b_: OD.rel_err(ni, cp, ri, a, b_)
        # oracle
        assert abs(ld[i] - OD.logdet(ni, cp, ri, xi)) < TOL * max(1.0, abs(ld[i]))
        assert err(g[z0:z1], OD.gradient(ni, cp, ri, xi)) < TOL
        want = OD.hessian(ni, cp, ri, xi, list(ysi))
        for j in range(m):
            assert err(t[j, z0:z1], want[j]) < TOL
            assert err(yi[j, z0:z1], OD.inv_hessian_dense(ni, cp, ri, xi, [ysi[j]])[0]) < TOL
        I, par = OS.fill(ni, OS.columns_from_csc(ni, cp, ri))
        cl, seps = OS.cliques_and_separators(I, par)
        xh = OD.completion_cliquesum(ni, cp, ri, si, cl, seps)
        assert abs(ldx[i] - OD.logdet(ni, cp, ri, xh)) < TOL * max(1.0, abs(ldx[i]))
        # the same instance alone: identical results
        s1 = B.Symbolic(*p, ordering=o)
        f1 = s1.factor(dev(xi))
        g1 = f1.gradient().cpu().numpy()
        t1 = f1.hessian(dev(ysi)).cpu().numpy()
        fx1, _ = s1.complete(dev(si))
        l1, _ = fx1.export()
        torch.cuda.synchronize()
        assert np.array_equal(g1, g[z0:z1])
        assert np.array_equal(t1, t[:, z0:z1])
        assert np.array_equal(l1.cpu().numpy(), lx[z0:z1])
    # f_* of the union is the sum over instances of (log det Xhat_i - n_i)
    assert abs(fstar - (ldx.sum() - sb.n)) < 1e-9 * max(1.0, abs(fstar))
