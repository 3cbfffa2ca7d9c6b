"""chd_hessian_noalloc: Hessian products with the library's fixed workspace.

The entry point is for callers that must not have a library allocate device
memory while they run (their memory belongs to their own allocator, or
allocator calls are banned after warm-up).  It must give the same products
as chd_hessian, call after call, even though every call reuses one device
array.  This file is collected last so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

from oracle import dense as OD
import workloads as W
from tests.helpers import lib

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _case(pattern, seed, **kw):
    import torch
    B = lib()
    sym = B.Symbolic(*pattern, **kw)
    rng = np.random.default_rng(seed)
    x = W.diag_dominant(sym.n, sym.colptr, sym.rowind, rng)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    fac = sym.factor(dev(x))
    fac.gradient()  # caches the projected inverse the entry point needs
    return B, sym, fac, rng, dev


CASES = {
    "band_chain": lambda: _case(W.band(200, 8), 21),  # the chain tier (library default)
    "band_warp": lambda: _case(W.band(200, 8), 25, chain_runs=False),
    # warp, CTA and dense tiers all in play (low dense-tier thresholds)
    "grid_mixed_tiers": lambda: _case(W.grid2d(16, 16), 22, perm=W.nested_dissection((16, 16), leaf=6),
                                      big_rows=20, big_cols=8),
    # one-column leaves of one parent processed as a leaf group, CTA-tier root
    "arrow_leaf_group": lambda: _case(W.arrow(120, 40), 26),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("side_stream", [False, True])
def test_noalloc_matches_hessian_on_two_calls(name, side_stream):
    """Two calls in a row (the second reuses the workspace the first left
    behind) give the products of chd_hessian, on the default stream and on
    a side stream; the calls change neither the factor's own workspace nor
    the device's free memory."""
    import torch
    B, sym, fac, rng, dev = CASES[name]()
    m = 3
    stream = torch.cuda.Stream() if side_stream else torch.cuda.current_stream()
    ys = [dev(W.uniform_sym(sym.n, sym.colptr, sym.rowind, rng, count=m)) for _ in range(2)]
    got = [torch.full_like(y, float("nan")) for y in ys]
    # one call first: kernels a fresh process has not run yet are loaded now
    warm = torch.empty_like(ys[0])
    with torch.cuda.stream(stream):
        B.chd_hessian_noalloc(fac.handle, ys[0], warm, sym.nnz, stream=stream)
    torch.cuda.synchronize()
    ws0 = fac.workspace_bytes()
    free0, _ = torch.cuda.mem_get_info()
    with torch.cuda.stream(stream):
        for call in range(2):
            B.chd_hessian_noalloc(fac.handle, ys[call], got[call], sym.nnz, stream=stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert fac.workspace_bytes() == ws0
    assert free1 == free0
    for call in range(2):
        want = torch.empty_like(ys[call])
        B.chd_hessian(fac.handle, ys[call], want, sym.nnz)
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got[call].cpu().numpy()
        for i in range(m):
            assert OD.rel_err(sym.n, sym.colptr, sym.rowind, g[i], w[i]) < TOL, (call, i)


def test_noalloc_rejects_what_does_not_fit_and_uncached_factors():
    import torch
    B = lib()
    # without a cached projected inverse the call is refused
    sym = B.Symbolic(*W.band(100, 4))
    rng = np.random.default_rng(23)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    fac = sym.factor(dev(W.diag_dominant(sym.n, sym.colptr, sym.rowind, rng)))
    ys = dev(W.uniform_sym(sym.n, sym.colptr, sym.rowind, rng, count=1))
    out = torch.empty_like(ys)
    with pytest.raises(B.ChdError) as e:
        B.chd_hessian_noalloc(fac.handle, ys, out, sym.nnz)
    assert e.value.code == B.CHD_ERR_INVALID
    # a pattern whose workspace exceeds the fixed 2 Mi doubles is refused
    B2, sym2, fac2, rng2, dev2 = _case(W.grid2d(100, 100), 24, perm=W.nested_dissection((100, 100), leaf=8))
    ys2 = dev2(W.uniform_sym(sym2.n, sym2.colptr, sym2.rowind, rng2, count=4))
    out2 = torch.empty_like(ys2)
    with pytest.raises(B2.ChdError) as e2:
        B2.chd_hessian_noalloc(fac2.handle, ys2, out2, sym2.nnz)
    assert e2.value.code == B2.CHD_ERR_INVALID
    # more right-hand sides than one launch sequence indexes are refused
    B3, sym3, fac3, rng3, dev3 = _case(W.band(4, 1), 27)
    ys3 = torch.zeros((65536, sym3.nnz), dtype=torch.float64, device="cuda")
    out3 = torch.empty_like(ys3)
    with pytest.raises(B3.ChdError) as e3:
        B3.chd_hessian_noalloc(fac3.handle, ys3, out3, sym3.nnz)
    assert e3.value.code == B3.CHD_ERR_INVALID
