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
