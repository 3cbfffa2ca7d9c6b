"""The C ABI library builds, loads and exports every function include/*.h declares."""
import ctypes

from tests.helpers import header_functions, lib


def test_header_declares_the_boundary():
    names = header_functions()
    for want in ("chd_analyze", "chd_symbolic_info", "chd_factor_new", "chd_logdet", "chd_gradient",
                 "chd_hessian", "chd_inv_hessian", "chd_complete", "chd_error_detail",
                 "chd_factor_free", "chd_symbolic_free"):
        assert want in names


def test_library_exports_every_declared_symbol():
    B = lib()
    so = ctypes.CDLL(B.library_path())
    missing = [n for n in header_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_invalid_arguments_are_rejected_without_a_gpu():
    B = lib()
    import numpy as np
    # entry above the diagonal (row < column) is invalid
    colptr = np.array([0, 1, 2], dtype=np.int64)
    rowind = np.array([1, 0], dtype=np.int32)
    try:
        B.chd_analyze(2, colptr, rowind)
        raise AssertionError("expected CHD_ERR_INVALID")
    except B.ChdError as e:
        assert e.code == B.CHD_ERR_INVALID
    # row index out of range
    rowind = np.array([0, 5], dtype=np.int32)
    try:
        B.chd_analyze(2, colptr, rowind)
        raise AssertionError("expected CHD_ERR_INVALID")
    except B.ChdError as e:
        assert e.code == B.CHD_ERR_INVALID
    # user permutation that is not one
    colptr = np.array([0, 1, 2, 3], dtype=np.int64)
    rowind = np.array([0, 1, 2], dtype=np.int32)
    try:
        B.chd_analyze(3, colptr, rowind, perm=np.array([0, 0, 1]))
        raise AssertionError("expected CHD_ERR_INVALID")
    except B.ChdError as e:
        assert e.code == B.CHD_ERR_INVALID


def test_null_handles_are_rejected_without_a_gpu():
    """Every numeric entry point checks its handles before any device work:
    a NULL factor or symbolic object gives CHD_ERR_INVALID."""
    B = lib()
    so = ctypes.CDLL(B.library_path())
    N = None
    i64 = ctypes.c_int64
    one = ctypes.c_int(1)
    out = ctypes.c_void_p()
    calls = {
        "chd_factor_new": (N, N, N, ctypes.byref(out)),
        "chd_refactor": (N, N, N),
        "chd_logdet": (N, ctypes.byref(ctypes.c_double())),
        "chd_logdet_batch": (N, N),
        "chd_gradient": (N, N, N),
        "chd_hessian": (N, one, N, i64(0), N, i64(0), N),
        "chd_hessian_noalloc": (N, one, N, i64(0), N, i64(0), N),
        "chd_inv_hessian": (N, one, N, i64(0), N, i64(0), N),
        "chd_hessian_factor": (N, one, N, i64(0), N, i64(0), N),
        "chd_hessian_factor_adj": (N, one, N, i64(0), N, i64(0), N),
        "chd_hessian_factor_sparse": (N, one, N, i64(0), N, i64(0), N),
        "chd_complete": (N, N, N, ctypes.byref(out), N),
        "chd_recomplete": (N, N, N, N),
        "chd_product": (N, N, N),
        "chd_schur": (N, one, N, i64(0), N, i64(0), N, N),
        "chd_factor_set_graphs": (N, one),
        "chd_factor_set_graph_limit": (N, i64(0)),
        "chd_completion_flops": (N, N),
        "chd_completion_plan": (N,) + (N,) * 7,
        "chd_symbolic_offsets": (N, N, N, N),
        "chd_factor_set_workspace_limit": (N, ctypes.c_size_t(0)),
        "chd_factor_release_workspace": (N,),
        "chd_factor_workspace_bytes": (N, ctypes.byref(ctypes.c_size_t())),
        "chd_symbolic_schedule": (N,) + tuple(ctypes.byref(x) for x in (i64(), i64())) + (N,) * 4,
    }
    for name, args in calls.items():
        f = getattr(so, name)
        f.restype = ctypes.c_int
        assert f(*args) == B.CHD_ERR_INVALID, name
    so.chd_factor_free(N)
    so.chd_symbolic_free(N)
