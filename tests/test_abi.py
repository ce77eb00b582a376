"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function include/bvss.h declares; the Python binding mirrors them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bvss.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"typedef struct[^;]*?\{.*?\}[^;]*;", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bvss_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_03301_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_api():
    names = _declared_functions()
    for want in ("bvss_build", "bvss_query", "bvss_query_trace", "bvss_encode", "bvss_free",
                 "bvss_last_error", "bvss_get_codes", "bvss_get_sketches", "bvss_get_counts",
                 "bvss_index_info"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2412_03301_gb300 import bvss
    assert sorted(bvss.SYMBOLS) == _declared_functions()


def test_struct_layouts_match_header():
    from paper_2412_03301_gb300 import bvss
    assert ctypes.sizeof(bvss.bvss_params) == 32
    assert ctypes.sizeof(bvss.bvss_search) == 24
    assert ctypes.sizeof(bvss.bvss_trace) == 8 * ctypes.sizeof(ctypes.c_void_p)
    src = open(HEADER).read()
    for field in ("d", "m", "fanin", "wta_l", "flags"):
        assert re.search(r"int32_t %s;" % field, src)


def test_last_error_is_empty_string_initially(lib):
    lib.bvss_last_error.restype = ctypes.c_char_p
    assert lib.bvss_last_error() == b""


def test_invalid_build_arguments_fail_without_gpu(lib):
    """Argument checks run before any CUDA call, so they work on a CPU machine."""
    from paper_2412_03301_gb300 import bvss
    b = bvss.load()
    out = ctypes.c_void_p()
    p = bvss.bvss_params(d=6, m=128, fanin=2, wta_l=4)      # d not a multiple of 4
    rc = b.bvss_build(ctypes.c_void_p(1), ctypes.c_void_p(1), 1, ctypes.c_void_p(1),
                      ctypes.byref(p), None, ctypes.byref(out))
    assert rc == bvss.BVSS_EINVAL and b"d = 6" in b.bvss_last_error()
    p = bvss.bvss_params(d=8, m=100, fanin=2, wta_l=4)      # m not a multiple of 128
    rc = b.bvss_build(ctypes.c_void_p(1), ctypes.c_void_p(1), 1, ctypes.c_void_p(1),
                      ctypes.byref(p), None, ctypes.byref(out))
    assert rc == bvss.BVSS_EINVAL
    p = bvss.bvss_params(d=8, m=128, fanin=2, wta_l=200)    # L > m
    rc = b.bvss_build(ctypes.c_void_p(1), ctypes.c_void_p(1), 1, ctypes.c_void_p(1),
                      ctypes.byref(p), None, ctypes.byref(out))
    assert rc == bvss.BVSS_EINVAL
    import numpy as np
    off = np.array([0, 2, 2], np.int64)                     # empty second set
    p = bvss.bvss_params(d=8, m=128, fanin=2, wta_l=4)
    rc = b.bvss_build(ctypes.c_void_p(1), ctypes.c_void_p(off.ctypes.data), 2,
                      ctypes.c_void_p(1), ctypes.byref(p), None, ctypes.byref(out))
    assert rc == bvss.BVSS_EINVAL and b"empty" in b.bvss_last_error()
    assert not out.value
