"""The C-ABI library loads and exports every entry point include/swgb.h
declares; host-side validation rejects bad input before touching a GPU."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_08308_gb300 import build
    from paper_2412_08308_gb300 import _native

    build()
    return _native.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "swgb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("sw_db_prepare", "sw_db_free", "sw_queries_prepare", "sw_search_prepared", "sw_search",
                 "sw_last_error"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    from paper_2412_08308_gb300 import _native

    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in _native.SIGNATURES, f"binding lacks {name}"


def test_db_prepare_rejects_bad_input_on_host(lib):
    from paper_2412_08308_gb300 import _native as N

    res = np.array([1, 2, 25, 3], dtype=np.uint8)  # code 25 is invalid
    off = np.array([0, 2, 4], dtype=np.int64)
    h = ctypes.c_void_p()
    rc = lib.sw_db_prepare(res.ctypes.data, off.ctypes.data, 2, None, ctypes.byref(h))
    assert rc == N.SW_EINVAL and b"code" in lib.sw_last_error()
    bad_off = np.array([0, 3, 2], dtype=np.int64)
    rc = lib.sw_db_prepare(res.ctypes.data, bad_off.ctypes.data, 2, None, ctypes.byref(h))
    assert rc == N.SW_EINVAL and b"offsets" in lib.sw_last_error()
    rc = lib.sw_db_prepare(res.ctypes.data, off.ctypes.data, 2, None, None)
    assert rc == N.SW_EINVAL
    off1 = np.array([1, 2], dtype=np.int64)
    rc = lib.sw_db_prepare(res.ctypes.data, off1.ctypes.data, 1, None, ctypes.byref(h))
    assert rc == N.SW_EINVAL


def test_null_handles_rejected(lib):
    from paper_2412_08308_gb300 import _native as N

    assert lib.sw_search_prepared(None, None, None, None) == N.SW_EINVAL
    assert lib.sw_db_free(None) == N.SW_OK
    assert lib.sw_queries_free(None) == N.SW_OK
    q = ctypes.c_void_p()
    assert lib.sw_queries_prepare(None, None, None, 0, None, 10, 2, 1, 0, None, ctypes.byref(q)) == N.SW_EINVAL


def test_product_path_does_not_touch_the_oracle():
    # the CUDA path and the oracle share no code: no source under the package
    # or include/ names the oracle
    for d in ("paper_2412_08308_gb300", "include"):
        for dirpath, _, files in os.walk(os.path.join(ROOT, d)):
            for f in files:
                if f.endswith((".py", ".cu", ".cuh", ".h")):
                    text = open(os.path.join(dirpath, f)).read()
                    assert "import oracle" not in text and "oracle_sw" not in text and "liboracle" not in text, f
