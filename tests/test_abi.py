"""The C-ABI library loads and exports every entry point that include/bo.h
declares (no GPU needed; no compute calls)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "bo.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bo_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_06059_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["bo_create_grid", "bo_set_properties", "bo_assemble", "bo_solve", "bo_step",
                     "bo_get_state", "bo_set_state", "bo_last_error", "bo_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1910_06059_gb300 import _lib
    assert sorted(_declared()) == sorted(_lib.EXPORTED)


def test_binding_refuses_missing_library(tmp_path):
    """No CPU fallback: a missing library is an import error."""
    from paper_1910_06059_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def test_last_error_is_callable_without_gpu(lib):
    lib.bo_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.bo_last_error(), bytes)


def test_null_arguments_are_rejected_without_gpu(lib):
    # argument validation happens before any CUDA call
    out = ctypes.c_void_p()
    st = lib.bo_create_grid(0, 1, 1, None, None, None, ctypes.c_double(0.0), ctypes.byref(out))
    assert st == 1  # BO_ERR_INVALID_ARG
    st = lib.bo_create_grid(2, 2, 2, None, None, None, ctypes.c_double(0.0), None)
    assert st == 1


def _null_args(argtypes):
    return [0.0 if t is ctypes.c_double else (0 if t is ctypes.c_int else None)
            for t in argtypes]


def test_every_entry_point_rejects_a_null_handle(lib):
    """Every call that takes a simulator or ensemble handle returns
    BO_ERR_INVALID_ARG or BO_ERR_STATE for NULL, sets the last-error message
    and touches no device (this runs without a GPU).  bo_destroy(NULL) is a
    no-op, like free(NULL)."""
    from paper_1910_06059_gb300 import _lib
    lib.bo_last_error.restype = ctypes.c_char_p
    checked = []
    for name, argtypes in _lib._SIGS.items():
        if name in ("bo_create_grid", "bo_residual_norms_noalloc", "bo_destroy"):
            continue
        fn = getattr(lib, name)
        fn.argtypes = argtypes
        fn.restype = ctypes.c_int
        st = fn(*_null_args(argtypes))
        assert st in (1, 7), (name, st)
        # the message names the call (the _dev variants share their host twin's)
        assert name.replace("_dev", "").encode() in lib.bo_last_error(), name
        checked.append(name)
    assert len(checked) >= 40
    lib.bo_destroy.argtypes = [ctypes.c_void_p]
    assert lib.bo_destroy(None) == 0


def test_noalloc_arguments_are_checked_without_gpu(lib):
    lib.bo_last_error.restype = ctypes.c_char_p
    f = lib.bo_residual_norms_noalloc
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_double] + [ctypes.c_void_p] * 2
    assert f(None, None, None, 10, 1.0, None, None) == 1
    assert b"NULL" in lib.bo_last_error()
