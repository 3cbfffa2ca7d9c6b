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
