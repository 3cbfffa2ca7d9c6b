"""Thin ctypes binding of the C ABI in ``include/chordal_barrier.h``.

Argument marshalling only: every numeric step runs in the CUDA kernels of
``libchordal_barrier.so``.  The functions keep the C names (``chd_analyze``,
``chd_factor_new``, ...); ``Symbolic`` and ``Factor`` are small owners of
the library objects.  Device arrays are torch tensors (float64, CUDA,
contiguous) passed as raw pointers together with the current CUDA stream.
If the shared library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libchordal_barrier.so")

if not os.path.exists(_LIBPATH):
    raise ImportError(
        f"{_LIBPATH} is missing: build it with `python -m paper_1203_2742_gb300.build` "
        "(the library has no fallback implementation)")

_lib = C.CDLL(_LIBPATH)

CHD_OK, CHD_ERR_INVALID, CHD_ERR_NOT_PD, CHD_ERR_NOT_COMPLETABLE, CHD_ERR_OOM, CHD_ERR_CUDA, \
    CHD_ERR_TIMEOUT = range(7)
_STATUS_NAMES = {0: "CHD_OK", 1: "CHD_ERR_INVALID", 2: "CHD_ERR_NOT_PD", 3: "CHD_ERR_NOT_COMPLETABLE",
                 4: "CHD_ERR_OOM", 5: "CHD_ERR_CUDA", 6: "CHD_ERR_TIMEOUT"}
ORDERINGS = {"natural": 0, "user": 1, "mindeg": 2, "nd_geometric": 3}


class ChdError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {_STATUS_NAMES.get(code, code)}")
        self.code = code


class chd_opts(C.Structure):
    _fields_ = [("ordering", C.c_int32), ("user_perm", C.POINTER(C.c_int64)), ("relax", C.c_int32),
                ("tie_last", C.c_int32), ("big_rows", C.c_int32), ("big_cols", C.c_int32),
                ("split_cols", C.c_int32), ("chain_runs", C.c_int32), ("tc_products", C.c_int32),
                ("nd_dims", C.c_int32 * 3), ("nd_leaf", C.c_int32), ("tier_table", C.POINTER(C.c_int32)),
                ("completion", C.c_int32)]


TIER_BUCKETS = 13


def tier_bucket(v):
    """Bucket of a front size in the tier table: its bit length, at most 12."""
    return min(TIER_BUCKETS - 1, int(v).bit_length())


_p = C.c_void_p
_i64 = C.c_int64
_lib.chd_opts_default.argtypes = [C.POINTER(chd_opts)]
_lib.chd_opts_default.restype = None
_lib.chd_analyze.argtypes = [_i64, _p, _p, C.POINTER(chd_opts), C.POINTER(_p)]
_lib.chd_analyze_batch.argtypes = [_i64, _p, _p, _p, _p, C.POINTER(_p)]
_lib.chd_symbolic_batch_info.argtypes = [_p, C.POINTER(_i64), C.POINTER(_p), C.POINTER(_p)]
_lib.chd_logdet_batch.argtypes = [_p, _p]
_lib.chd_symbolic_info.argtypes = [_p, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_p), C.POINTER(_p),
                                   C.POINTER(_p), C.POINTER(_i64)]
_lib.chd_symbolic_supernodes.argtypes = [_p, C.POINTER(_p), C.POINTER(_p), C.POINTER(_p), C.POINTER(_p)]
_lib.chd_symbolic_flops.argtypes = [_p, C.POINTER(C.c_double)]
_lib.chd_completion_flops.argtypes = [_p, C.POINTER(C.c_double)]
_lib.chd_completion_flops.restype = C.c_int
_lib.chd_completion_plan.restype = C.c_int
_lib.chd_symbolic_offsets.restype = C.c_int
_lib.chd_symbolic_free.argtypes = [_p]
_lib.chd_symbolic_free.restype = None
_lib.chd_factor_new.argtypes = [_p, _p, _p, C.POINTER(_p)]
_lib.chd_refactor.argtypes = [_p, _p, _p]
_lib.chd_logdet.argtypes = [_p, C.POINTER(C.c_double)]
_lib.chd_gradient.argtypes = [_p, _p, _p]
_lib.chd_hessian.argtypes = [_p, C.c_int, _p, _i64, _p, _i64, _p]
_lib.chd_inv_hessian.argtypes = [_p, C.c_int, _p, _i64, _p, _i64, _p]
_lib.chd_complete.argtypes = [_p, _p, _p, C.POINTER(_p), C.POINTER(C.c_double)]
_lib.chd_recomplete.argtypes = [_p, _p, _p, C.POINTER(C.c_double)]
_lib.chd_factor_export.argtypes = [_p, _p, _p, _p]
_lib.chd_status_get.argtypes = [_p]
_lib.chd_error_detail.argtypes = [_p, C.POINTER(_i64), C.POINTER(_i64)]
_lib.chd_kernel_launches.argtypes = []
_lib.chd_kernel_launches.restype = _i64
_lib.chd_split_k_launches.argtypes = []
_lib.chd_split_k_launches.restype = _i64
_lib.chd_tc_flops.argtypes = []
_lib.chd_tc_flops.restype = C.c_double
_lib.chd_dgemm_tc.argtypes = [_i64, _i64, _i64, C.c_double, C.c_void_p, _i64, C.c_void_p, _i64, C.c_double,
                              C.c_void_p, _i64, C.c_void_p]
_lib.chd_dgemm_tc.restype = C.c_int
_lib.chd_probe_tc_bf16_peak.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
_lib.chd_probe_tc_bf16_peak.restype = C.c_int
_lib.chd_probe_units.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
_lib.chd_probe_units.restype = C.c_int
_lib.chd_hessian_noalloc.argtypes = [_p, C.c_int, _p, _i64, _p, _i64, _p]
_lib.chd_hessian_noalloc.restype = C.c_int
_lib.chd_probe_fp64_peak.argtypes = [_p, C.POINTER(C.c_double)]
_lib.chd_probe_fp64_peak.restype = C.c_int
_lib.chd_factor_set_workspace_limit.argtypes = [_p, C.c_size_t]
_lib.chd_factor_set_workspace_limit.restype = C.c_int
_lib.chd_factor_release_workspace.argtypes = [_p]
_lib.chd_factor_release_workspace.restype = C.c_int
_lib.chd_factor_workspace_bytes.argtypes = [_p, C.POINTER(C.c_size_t)]
_lib.chd_factor_workspace_bytes.restype = C.c_int
_lib.chd_factor_set_graphs.argtypes = [_p, C.c_int]
_lib.chd_factor_set_graphs.restype = C.c_int
_lib.chd_factor_set_graph_limit.argtypes = [_p, C.c_int64]
_lib.chd_factor_set_graph_limit.restype = C.c_int
_lib.chd_factor_free.argtypes = [_p]
_lib.chd_factor_free.restype = None
_lib.chd_product.argtypes = [_p, _p, _p]
_lib.chd_product.restype = C.c_int
_lib.chd_schur.argtypes = [_p, C.c_int, _p, C.c_int64, _p, C.c_int64, _p, _p]
_lib.chd_schur.restype = C.c_int
_lib.chd_symbolic_schedule.argtypes = [_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)] + [
    C.POINTER(C.POINTER(C.c_int32))] * 4
_lib.chd_symbolic_schedule.restype = C.c_int
for _f in ("chd_hessian_factor", "chd_hessian_factor_adj", "chd_hessian_factor_sparse"):
    getattr(_lib, _f).argtypes = [_p, C.c_int, _p, _i64, _p, _i64, _p]
    getattr(_lib, _f).restype = C.c_int
for _f in ("chd_analyze", "chd_analyze_batch", "chd_symbolic_batch_info", "chd_logdet_batch", "chd_symbolic_info", "chd_symbolic_supernodes", "chd_symbolic_flops",
           "chd_factor_new", "chd_refactor", "chd_logdet", "chd_gradient", "chd_hessian",
           "chd_inv_hessian", "chd_complete", "chd_recomplete", "chd_factor_export", "chd_status_get",
           "chd_error_detail"):
    getattr(_lib, _f).restype = C.c_int


def library_path() -> str:
    return _LIBPATH


def exported_symbols():
    return [n for n in dir(_lib) if n.startswith("chd_")]


def _check(rc, what):
    if rc != CHD_OK:
        raise ChdError(rc, what)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t, what, nnz=None, rows=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{what}: expected a CUDA float64 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    if nnz is not None and t.shape[-1] != nnz:
        raise ValueError(f"{what}: last dimension {t.shape[-1]} != nnz {nnz}")
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# C-named entry points
# ---------------------------------------------------------------------------

def chd_analyze(n, colptr, rowind, **options):
    """Symbolic analysis of one pattern; options as for `_opts`."""
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(rowind, dtype=np.int32)
    o, keep = _opts(**options)
    out = _p()
    rc = _lib.chd_analyze(int(n), colptr.ctypes.data, rowind.ctypes.data, C.byref(o), C.byref(out))
    _check(rc, "chd_analyze")
    del keep
    return out


def _opts(ordering="natural", perm=None, relax=0, tie_last=True, big_rows=0, big_cols=0, split_cols=0,
          chain_runs=True, tc_products=0, tier_table=None, nd_dims=None, nd_leaf=0, completion="independent"):
    """chd_opts from keyword options (and the host arrays it points to).
    ordering: "natural", "mindeg", "nd_geometric" (with nd_dims = grid
    dimensions, one to three of them) or "user" (implied by perm);
    completion: "independent" (every front factors its V_k) or "factored"
    (update matrices propagated from the parents, Algorithm 4.3)."""
    o = chd_opts()
    _lib.chd_opts_default(C.byref(o))
    o.ordering = ORDERINGS[ordering]
    keep = None
    if perm is not None:
        keep = np.ascontiguousarray(perm, dtype=np.int64)
        o.user_perm = keep.ctypes.data_as(C.POINTER(C.c_int64))
        o.ordering = ORDERINGS["user"]
    if ordering == "nd_geometric":
        dims = [int(d) for d in nd_dims] + [1] * (3 - len(nd_dims))
        o.nd_dims[:] = dims
        o.nd_leaf = int(nd_leaf)
    o.relax = int(relax)
    o.tie_last = 1 if tie_last else 0
    o.big_rows = int(big_rows)
    o.big_cols = int(big_cols)
    o.split_cols = int(split_cols)
    o.chain_runs = int(chain_runs)
    o.tc_products = int(tc_products)
    o.completion = {"independent": 0, "factored": 1}[completion]
    if tier_table is not None:
        tt = np.ascontiguousarray(tier_table, dtype=np.int32).reshape(-1)
        if tt.size != TIER_BUCKETS * TIER_BUCKETS:
            raise ValueError("tier_table needs TIER_BUCKETS^2 entries")
        o.tier_table = tt.ctypes.data_as(C.POINTER(C.c_int32))
        keep = (keep, tt)
    return o, keep


def chd_analyze_batch(patterns, orderings=None, perms=None, **shared):
    """Analyse independent patterns together (one block-diagonal union).

    patterns: list of (n, colptr, rowind); orderings / perms: per-instance
    lists (None for natural order; an ordering is a name or a dict of
    ordering options, e.g. {"ordering": "nd_geometric", "nd_dims": (k, k)});
    shared options (relax, big_rows, ...) are taken from the first
    instance's options.
    """
    count = len(patterns)
    orderings = orderings or ["natural"] * count
    perms = perms or [None] * count
    keep = []
    ns = np.array([p[0] for p in patterns], dtype=np.int64)
    cps = [np.ascontiguousarray(p[1], dtype=np.int64) for p in patterns]
    ris = [np.ascontiguousarray(p[2], dtype=np.int32) for p in patterns]
    keep += cps + ris
    OA = chd_opts * count
    oa = OA()
    for i in range(count):
        oi = orderings[i] if isinstance(orderings[i], dict) else {"ordering": orderings[i]}
        o, k = _opts(perm=perms[i], **oi, **shared)
        oa[i] = o
        keep.append(k)
    cp_ptrs = (C.c_void_p * count)(*[c.ctypes.data for c in cps])
    ri_ptrs = (C.c_void_p * count)(*[r.ctypes.data for r in ris])
    out = _p()
    rc = _lib.chd_analyze_batch(count, ns.ctypes.data, C.cast(cp_ptrs, C.c_void_p), C.cast(ri_ptrs, C.c_void_p),
                                C.cast(oa, C.c_void_p), C.byref(out))
    _check(rc, "chd_analyze_batch")
    return out


def chd_symbolic_batch_info(sym):
    cnt = _i64()
    no, zo = _p(), _p()
    _check(_lib.chd_symbolic_batch_info(sym, C.byref(cnt), C.byref(no), C.byref(zo)), "chd_symbolic_batch_info")
    k = cnt.value
    n_off = np.ctypeslib.as_array(C.cast(no, C.POINTER(C.c_int64)), shape=(k + 1,)).copy()
    nnz_off = np.ctypeslib.as_array(C.cast(zo, C.POINTER(C.c_int64)), shape=(k + 1,)).copy()
    return n_off, nnz_off


def chd_logdet_batch(fac, count):
    out = np.zeros(count, dtype=np.float64)
    _check(_lib.chd_logdet_batch(fac, out.ctypes.data), "chd_logdet_batch")
    return out


def chd_symbolic_info(sym):
    n, nnz, ns = _i64(), _i64(), _i64()
    cp, ri, pm = _p(), _p(), _p()
    _check(_lib.chd_symbolic_info(sym, C.byref(n), C.byref(nnz), C.byref(cp), C.byref(ri), C.byref(pm),
                                  C.byref(ns)), "chd_symbolic_info")
    n, nnz = n.value, nnz.value
    colptr = np.ctypeslib.as_array(C.cast(cp, C.POINTER(C.c_int64)), shape=(n + 1,)).copy()
    rowind = np.ctypeslib.as_array(C.cast(ri, C.POINTER(C.c_int32)), shape=(nnz,)).copy()
    perm = np.ctypeslib.as_array(C.cast(pm, C.POINTER(C.c_int64)), shape=(n,)).copy()
    return dict(n=n, nnz=nnz, colptr=colptr, rowind=rowind, perm=perm, nsuper=ns.value)


def chd_symbolic_supernodes(sym, nsuper):
    sp, par, rp, rows = _p(), _p(), _p(), _p()
    _check(_lib.chd_symbolic_supernodes(sym, C.byref(sp), C.byref(par), C.byref(rp), C.byref(rows)),
           "chd_symbolic_supernodes")
    snode_ptr = np.ctypeslib.as_array(C.cast(sp, C.POINTER(C.c_int64)), shape=(nsuper + 1,)).copy()
    snode_par = np.ctypeslib.as_array(C.cast(par, C.POINTER(C.c_int64)), shape=(nsuper,)).copy()
    rows_ptr = np.ctypeslib.as_array(C.cast(rp, C.POINTER(C.c_int64)), shape=(nsuper + 1,)).copy()
    rws = np.ctypeslib.as_array(C.cast(rows, C.POINTER(C.c_int32)), shape=(int(rows_ptr[-1]),)).copy()
    return snode_ptr, snode_par, rows_ptr, rws


def chd_symbolic_flops(sym):
    out = (C.c_double * 5)()
    _check(_lib.chd_symbolic_flops(sym, out), "chd_symbolic_flops")
    return dict(factor=out[0], gradient=out[1], hessian=out[2], inv_hessian=out[3], completion=out[4])


def chd_completion_flops(sym):
    """The two completion forms' differing work: Cholesky of every V_k
    (independent) against the factored propagation, and its level count."""
    out = (C.c_double * 3)()
    _check(_lib.chd_completion_flops(sym, out), "chd_completion_flops")
    return dict(independent=out[0], factored=out[1], levels=int(out[2]))


def chd_symbolic_offsets(sym, nsn):
    """Per-front offsets (nsn + 1 each): f_off (workspace), d_off, v_off."""
    ptrs = [C.POINTER(C.c_int64)() for _ in range(3)]
    _check(_lib.chd_symbolic_offsets(sym, *[C.byref(p) for p in ptrs]), "chd_symbolic_offsets")
    return [np.ctypeslib.as_array(p, shape=(nsn + 1,)).copy() for p in ptrs]


def chd_completion_plan(sym, nsn):
    """The factored completion's plan: dict of numpy arrays fc_off (per
    front), fc_lvl, fc_fronts, fc_big_lvl, fc_big, and fc_total."""
    nl, tot = C.c_int64(), C.c_int64()
    off = C.POINTER(C.c_int64)()
    ptrs = [C.POINTER(C.c_int32)() for _ in range(4)]
    _check(_lib.chd_completion_plan(sym, C.byref(nl), C.byref(tot), C.byref(off), *[C.byref(p) for p in ptrs]),
           "chd_completion_plan")
    L = nl.value
    arr = lambda p, k: np.ctypeslib.as_array(p, shape=(k,)).copy() if k > 0 else np.zeros(0, np.int64)
    lvl, big_lvl = arr(ptrs[0], L + 1), arr(ptrs[2], L + 1)
    return {"fc_off": arr(off, nsn), "fc_lvl": lvl, "fc_fronts": arr(ptrs[1], int(lvl[-1])),
            "fc_big_lvl": big_lvl, "fc_big": arr(ptrs[3], int(big_lvl[-1])), "fc_total": tot.value}


def chd_symbolic_free(sym):
    _lib.chd_symbolic_free(sym)


def chd_factor_new(sym, x, nnz, stream=None):
    out = _p()
    _check(_lib.chd_factor_new(sym, _dptr(x, "x", nnz), _stream_ptr(stream), C.byref(out)), "chd_factor_new")
    return out


def chd_refactor(fac, x, nnz, stream=None):
    _check(_lib.chd_refactor(fac, _dptr(x, "x", nnz), _stream_ptr(stream)), "chd_refactor")


def chd_logdet(fac):
    v = C.c_double()
    _check(_lib.chd_logdet(fac, C.byref(v)), "chd_logdet")
    return v.value


def chd_gradient(fac, g, nnz, stream=None):
    _check(_lib.chd_gradient(fac, _dptr(g, "g", nnz), _stream_ptr(stream)), "chd_gradient")


def _batch(t, nnz, what):
    if t.dim() == 1:
        return 1, nnz
    if t.dim() != 2:
        raise ValueError(f"{what}: expected (m, ld) or (nnz,)")
    return t.shape[0], t.stride(0)


def chd_hessian(fac, y, t, nnz, stream=None):
    m, ldy = _batch(y, nnz, "y")
    m2, ldt = _batch(t, nnz, "t")
    if m != m2:
        raise ValueError("y and t batch sizes differ")
    _check(_lib.chd_hessian(fac, m, _dptr(y, "y"), ldy, _dptr(t, "t"), ldt, _stream_ptr(stream)),
           "chd_hessian")


def chd_hessian_noalloc(fac, y, t, nnz, stream=None):
    """Hessian products with the library's fixed workspace (no allocation)."""
    m, ldy = _batch(y, nnz, "y")
    m2, ldt = _batch(t, nnz, "t")
    if m != m2:
        raise ValueError("y and t batch sizes differ")
    _check(_lib.chd_hessian_noalloc(fac, m, _dptr(y, "y"), ldy, _dptr(t, "t"), ldt, _stream_ptr(stream)),
           "chd_hessian_noalloc")


def chd_hessian_factor(fac, y, w, nnz, stream=None):
    """W = R(Y), H = R^adj o R (Algorithm 5.3)."""
    m, ldy = _batch(y, nnz, "y")
    m2, ldw = _batch(w, nnz, "w")
    if m != m2:
        raise ValueError("y and w batch sizes differ")
    _check(_lib.chd_hessian_factor(fac, m, _dptr(y, "y"), ldy, _dptr(w, "w"), ldw, _stream_ptr(stream)),
           "chd_hessian_factor")


def chd_hessian_factor_sparse(fac, y, w, nnz, stream=None):
    """W = R(Y) with the clique tree pruned per Y (§5.5)."""
    m, ldy = _batch(y, nnz, "y")
    m2, ldw = _batch(w, nnz, "w")
    if m != m2:
        raise ValueError("y and w batch sizes differ")
    _check(_lib.chd_hessian_factor_sparse(fac, m, _dptr(y, "y"), ldy, _dptr(w, "w"), ldw, _stream_ptr(stream)),
           "chd_hessian_factor_sparse")


def chd_hessian_factor_adj(fac, w, t, nnz, stream=None):
    """T = R^adj(W) (Algorithm 5.4)."""
    m, ldw = _batch(w, nnz, "w")
    m2, ldt = _batch(t, nnz, "t")
    if m != m2:
        raise ValueError("w and t batch sizes differ")
    _check(_lib.chd_hessian_factor_adj(fac, m, _dptr(w, "w"), ldw, _dptr(t, "t"), ldt, _stream_ptr(stream)),
           "chd_hessian_factor_adj")


def chd_inv_hessian(fac, t, y, nnz, stream=None):
    m, ldt = _batch(t, nnz, "t")
    m2, ldy = _batch(y, nnz, "y")
    if m != m2:
        raise ValueError("t and y batch sizes differ")
    _check(_lib.chd_inv_hessian(fac, m, _dptr(t, "t"), ldt, _dptr(y, "y"), ldy, _stream_ptr(stream)),
           "chd_inv_hessian")


def chd_complete(sym, s, nnz, stream=None, want_fstar=True):
    out = _p()
    f = C.c_double()
    rc = _lib.chd_complete(sym, _dptr(s, "s", nnz), _stream_ptr(stream), C.byref(out),
                           C.byref(f) if want_fstar else None)
    _check(rc, "chd_complete")
    return out, (f.value if want_fstar else None)


def chd_recomplete(fac, s, nnz, stream=None, want_fstar=True):
    f = C.c_double()
    rc = _lib.chd_recomplete(fac, _dptr(s, "s", nnz), _stream_ptr(stream), C.byref(f) if want_fstar else None)
    _check(rc, "chd_recomplete")
    return f.value if want_fstar else None


def chd_factor_export(fac, l, d, stream=None):
    _check(_lib.chd_factor_export(fac, _dptr(l, "l"), _dptr(d, "d"), _stream_ptr(stream)),
           "chd_factor_export")


def chd_status_get(fac):
    return _lib.chd_status_get(fac)


def chd_error_detail(fac):
    s, c = _i64(), _i64()
    rc = _lib.chd_error_detail(fac, C.byref(s), C.byref(c))
    return rc, s.value, c.value


def chd_kernel_launches():
    return int(_lib.chd_kernel_launches())


def chd_split_k_launches():
    return int(_lib.chd_split_k_launches())


def chd_tc_flops():
    return float(_lib.chd_tc_flops())


def chd_dgemm_tc(a, b, c=None, alpha=1.0, beta=0.0, stream=None):
    """C = beta C + alpha A B on the tensor cores (FP64-level accuracy).
    a (m x k), b (k x n), c (m x n): CUDA float64 tensors in column-major
    order (transposed views of row-major tensors, ``t.T``) or None for c."""
    import torch
    m, k = a.shape
    k2, n = b.shape
    if k2 != k:
        raise ValueError("inner dimensions differ")
    if c is None:
        c = torch.zeros((n, m), dtype=torch.float64, device=a.device).T
    for t_, what in ((a, "a"), (b, "b"), (c, "c")):
        if t_.dtype != torch.float64 or not t_.is_cuda or (t_.numel() and t_.stride(0) != 1):
            raise ValueError(f"{what} must be a column-major CUDA float64 matrix")
    ld = lambda t_: max(1, t_.stride(1) if t_.dim() == 2 and t_.shape[1] > 1 else t_.shape[0])
    _check(_lib.chd_dgemm_tc(m, n, k, float(alpha), a.data_ptr(), ld(a), b.data_ptr(), ld(b), float(beta),
                             c.data_ptr(), ld(c), _stream_ptr(stream)), "chd_dgemm_tc")
    return c


def chd_probe_units(stream=None):
    """dict: fp64_fma_tflops, fp64_mma_tflops, fp32_fma_tflops, fp64_fma_latency_ns."""
    v = (C.c_double * 4)()
    _check(_lib.chd_probe_units(_stream_ptr(stream), v), "chd_probe_units")
    return {"fp64_fma_tflops": v[0], "fp64_mma_tflops": v[1], "fp32_fma_tflops": v[2], "fp64_fma_latency_ns": v[3]}


def chd_probe_tc_bf16_peak(stream=None):
    v = C.c_double()
    _check(_lib.chd_probe_tc_bf16_peak(_stream_ptr(stream), C.byref(v)), "chd_probe_tc_bf16_peak")
    return v.value


def chd_probe_fp64_peak(stream=None):
    v = C.c_double()
    _check(_lib.chd_probe_fp64_peak(_stream_ptr(stream), C.byref(v)), "chd_probe_fp64_peak")
    return v.value


def chd_factor_free(fac):
    _lib.chd_factor_free(fac)


# ---------------------------------------------------------------------------
# owners
# ---------------------------------------------------------------------------

class Symbolic:
    """Owner of a ``chd_symbolic``: the analysed pattern and its clique tree."""

    def __init__(self, n, colptr, rowind, **options):
        """options: ordering ("natural", "mindeg", "nd_geometric" with
        nd_dims and nd_leaf), perm (a user ordering), relax, tie_last,
        big_rows, big_cols, split_cols, chain_runs, tc_products, tier_table
        (the fields of chd_opts)."""
        self._h = chd_analyze(n, colptr, rowind, **options)
        info = chd_symbolic_info(self._h)
        self.n = info["n"]
        self.nnz = info["nnz"]
        self.colptr = info["colptr"]
        self.rowind = info["rowind"]
        self.perm = info["perm"]
        self.nsuper = info["nsuper"]

    @property
    def handle(self):
        return self._h

    @property
    def instances(self):
        """(n_off, nnz_off): column and value ranges of the instances."""
        return chd_symbolic_batch_info(self._h)

    def schedule(self):
        return chd_symbolic_schedule(self._h)

    def supernodes(self):
        return chd_symbolic_supernodes(self._h, self.nsuper)

    def flops(self):
        return chd_symbolic_flops(self._h)

    def completion_flops(self):
        return chd_completion_flops(self._h)

    def completion_plan(self):
        return chd_completion_plan(self._h, self.nsuper)

    def offsets(self):
        """(f_off, d_off, v_off) of the analysis."""
        return chd_symbolic_offsets(self._h, self.nsuper)

    def factor(self, x, stream=None):
        return Factor(self, chd_factor_new(self._h, x, self.nnz, stream))

    def complete(self, s, stream=None):
        h, fstar = chd_complete(self._h, s, self.nnz, stream)
        return Factor(self, h), fstar

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            chd_symbolic_free(h)
            self._h = None


def chd_symbolic_schedule(sym):
    """The analysis' launch schedule: dict of numpy arrays lvl_ptr, lvl_counts
    (nlevels x 5: chain runs |J| <= 32, chain runs |J| <= 64, warp, wide warp,
    dense), task_ptr, task_fronts."""
    nl, nt = C.c_int64(), C.c_int64()
    ptrs = [C.POINTER(C.c_int32)() for _ in range(4)]
    _check(_lib.chd_symbolic_schedule(sym, C.byref(nl), C.byref(nt), *[C.byref(p) for p in ptrs]),
           "chd_symbolic_schedule")
    L, T = nl.value, nt.value
    arr = lambda p, k: np.ctypeslib.as_array(p, shape=(k,)).copy() if k > 0 else np.zeros(0, np.int32)
    task_ptr = arr(ptrs[2], T + 1)
    return {"lvl_ptr": arr(ptrs[0], L + 1), "lvl_counts": arr(ptrs[1], 5 * L).reshape(L, 5),
            "task_ptr": task_ptr, "task_fronts": arr(ptrs[3], int(task_ptr[-1]) if T > 0 else 0)}


class SymbolicBatch(Symbolic):
    """Owner of a batched chd_symbolic: independent patterns run together."""

    def __init__(self, patterns, orderings=None, perms=None, **shared):
        self._h = chd_analyze_batch(patterns, orderings, perms, **shared)
        info = chd_symbolic_info(self._h)
        self.n = info["n"]
        self.nnz = info["nnz"]
        self.colptr = info["colptr"]
        self.rowind = info["rowind"]
        self.perm = info["perm"]
        self.nsuper = info["nsuper"]
        self.n_off, self.nnz_off = chd_symbolic_batch_info(self._h)
        self.count = len(self.n_off) - 1

    def instance_pattern(self, i):
        """Analysed pattern (n_i, colptr_i, rowind_i) and perm_i of instance i."""
        a, b_ = int(self.n_off[i]), int(self.n_off[i + 1])
        z0 = int(self.nnz_off[i])
        cp = self.colptr[a:b_ + 1] - z0
        ri = self.rowind[z0:int(self.nnz_off[i + 1])] - a
        return (b_ - a, cp, ri.astype(np.int32)), self.perm[a:b_] - a


class Factor:
    """Owner of a ``chd_factor`` (device-resident factor and cached blocks)."""

    def __init__(self, sym, handle):
        self.sym = sym
        self._h = handle

    @property
    def handle(self):
        return self._h

    def refactor(self, x, stream=None):
        chd_refactor(self._h, x, self.sym.nnz, stream)

    def logdet(self):
        return chd_logdet(self._h)

    def logdet_batch(self):
        return chd_logdet_batch(self._h, len(self.sym.instances[0]) - 1)

    def recomplete(self, s, stream=None, want_fstar=True):
        return chd_recomplete(self._h, s, self.sym.nnz, stream, want_fstar)

    def gradient(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.sym.nnz, dtype=torch.float64, device="cuda")
        chd_gradient(self._h, out, self.sym.nnz, stream)
        return out

    def hessian(self, y, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(y)
        chd_hessian(self._h, y, out, self.sym.nnz, stream)
        return out

    def hessian_factor(self, y, out=None, stream=None, sparse=False):
        """W = R(Y) with H = R^adj o R (Algorithm 5.3); `sparse` prunes the
        clique tree per Y (§5.5), for Y with few nonzeros."""
        import torch
        if out is None:
            out = torch.empty_like(y)
        (chd_hessian_factor_sparse if sparse else chd_hessian_factor)(self._h, y, out, self.sym.nnz, stream)
        return out

    def hessian_factor_adj(self, w, out=None, stream=None):
        """T = R^adj(W) (Algorithm 5.4); `out` may be `w` itself."""
        import torch
        if out is None:
            out = torch.empty_like(w)
        chd_hessian_factor_adj(self._h, w, out, self.sym.nnz, stream)
        return out

    def inv_hessian(self, t, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(t)
        chd_inv_hessian(self._h, t, out, self.sym.nnz, stream)
        return out

    def schur(self, a, t=None, h=None, stream=None):
        """H_ij = A_i . H(A_j) for the rows A_i of `a` (m x nnz); returns (H, T)."""
        import torch
        a = a if a.dim() == 2 else a.reshape(1, -1)
        m = a.shape[0]
        if t is None:
            t = torch.empty_like(a)
        if h is None:
            h = torch.empty((m, m), dtype=torch.float64, device="cuda")
        _check(_lib.chd_schur(self._h, m, _dptr(a, "a", self.sym.nnz, rows=m), a.stride(0),
                              _dptr(t, "t", self.sym.nnz, rows=m), t.stride(0), _dptr(h, "h"),
                              _stream_ptr(stream)), "chd_schur")
        return h.t(), t

    def product(self, out=None, stream=None):
        """Values on V of L D L^T (Algorithm 3.2): X, or X-hat for a completion."""
        import torch
        if out is None:
            out = torch.empty(self.sym.nnz, dtype=torch.float64, device="cuda")
        _check(_lib.chd_product(self._h, _dptr(out, "out", self.sym.nnz), _stream_ptr(stream)), "chd_product")
        return out

    def export(self, stream=None):
        import torch
        l = torch.empty(self.sym.nnz, dtype=torch.float64, device="cuda")
        d = torch.empty(self.sym.n, dtype=torch.float64, device="cuda")
        chd_factor_export(self._h, l, d, stream)
        return l, d

    def status(self):
        return chd_status_get(self._h)

    def set_workspace_limit(self, nbytes):
        _check(_lib.chd_factor_set_workspace_limit(self._h, int(nbytes)), "chd_factor_set_workspace_limit")

    def release_workspace(self):
        _check(_lib.chd_factor_release_workspace(self._h), "chd_factor_release_workspace")

    def set_graphs(self, on):
        """Replay repeated calls with the same arguments from CUDA graphs (default on)."""
        _check(_lib.chd_factor_set_graphs(self._h, 1 if on else 0), "chd_factor_set_graphs")

    def set_graph_limit(self, launches):
        """Longest launch sequence captured into a graph (default 8192)."""
        _check(_lib.chd_factor_set_graph_limit(self._h, int(launches)), "chd_factor_set_graph_limit")

    def workspace_bytes(self):
        v = C.c_size_t()
        _check(_lib.chd_factor_workspace_bytes(self._h, C.byref(v)), "chd_factor_workspace_bytes")
        return int(v.value)

    def error_detail(self):
        return chd_error_detail(self._h)

    def free(self):
        if self._h:
            chd_factor_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
