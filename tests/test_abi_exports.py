"""The C-ABI library builds, loads without a GPU and exports every entry
point include/lmmew.h declares; the binding fails loudly without it."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lmmew.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lm_create", "lm_sensitivity", "lm_forward", "lm_backproject", "lm_osem",
                 "lm_destroy", "lm_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2305_17111_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    from paper_2305_17111_gb300 import _native
    assert set(declared_functions()) == set(_native.SYMBOLS)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2305_17111_gb300 import _native
    old = _native._lib
    _native._lib = None
    try:
        with pytest.raises(RuntimeError, match="missing"):
            _native.load(str(tmp_path / "liblmmew.so"))
    finally:
        _native._lib = old


def test_errors_reported_without_gpu_work():
    """Argument checks run before any CUDA call."""
    from paper_2305_17111_gb300 import _native, build
    build.build()
    lib = _native.load()
    h = ctypes.c_void_p()
    rc = lib.lm_create(None, None, None, None, None, 1, ctypes.byref(h))
    assert rc == -1
    assert b"NULL" in lib.lm_last_error()
    assert lib.lm_destroy(None) == 0


def test_table_streaming_calls_check_their_arguments_without_gpu_work():
    """The streamed-table controls reject bad arguments before any CUDA call;
    the process-wide table budget is a plain host setting."""
    from paper_2305_17111_gb300 import _native, build
    build.build()
    lib = _native.load()
    assert lib.lm_set_table_budget(-1) == -1
    assert lib.lm_set_table_budget(1 << 30) == 0
    assert lib.lm_set_table_budget(0) == 0
    assert lib.lm_set_table_streaming(None, 4) == -1
    slots, nbytes = ctypes.c_int(7), ctypes.c_int64(7)
    assert lib.lm_table_streaming(None, ctypes.byref(slots), ctypes.byref(nbytes)) == -1
    assert b"NULL" in lib.lm_last_error()
