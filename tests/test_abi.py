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


def test_plan_and_fp8_arguments_fail_without_gpu(lib):
    """The plan entry points reject a NULL plan or index, and the FP8 copy's d % 128
    rule is checked with the other build parameters, before any CUDA call."""
    from paper_2412_03301_gb300 import bvss
    b = bvss.load()
    s = bvss.bvss_search(k=1, C=1, A=1, M=1, flags=0)
    out = ctypes.c_void_p()
    rc = b.bvss_plan_create(None, ctypes.byref(s), 1, 1, 1, None, None, None, None, None,
                            ctypes.byref(out))
    assert rc == bvss.BVSS_EINVAL and out.value is None
    assert b.bvss_plan_launch(None, None) == bvss.BVSS_EINVAL
    assert b.bvss_plan_tune(None, 1, None, None) == bvss.BVSS_EINVAL
    assert b.bvss_plan_info(None, None, None) == bvss.BVSS_EINVAL
    kn = (ctypes.c_int32 * 6)(0, 0, 0, 0, 0, 0)
    assert b.bvss_plan_set_knobs(None, kn) == bvss.BVSS_EINVAL
    b.bvss_plan_free(None)                                   # a no-op
    p = bvss.bvss_params(d=64, m=128, fanin=2, wta_l=4, flags=bvss.BVSS_BUILD_FP8)
    rc = b.bvss_build(ctypes.c_void_p(1), ctypes.c_void_p(1), 1, ctypes.c_void_p(1),
                      ctypes.byref(p), None, ctypes.byref(out))
    assert rc == bvss.BVSS_EINVAL and b"BVSS_BUILD_FP8" in b.bvss_last_error()
    p = bvss.bvss_params(d=64, m=128, fanin=2, wta_l=4, flags=8)   # unknown build flag
    rc = b.bvss_build(ctypes.c_void_p(1), ctypes.c_void_p(1), 1, ctypes.c_void_p(1),
                      ctypes.byref(p), None, ctypes.byref(out))
    assert rc == bvss.BVSS_EINVAL


def test_zipf_set_sizes_follow_the_stated_law():
    """The serving load's reading of "Zipf-distributed in 1-128": P(size = k) is
    proportional to 1/k on 1..128 (exponent 1)."""
    import numpy as np
    from paper_2412_03301_gb300 import datagen
    n = 400_000
    z = datagen.zipf_sizes(n, 1, 128, seed=5)
    assert z.min() >= 1 and z.max() <= 128
    k = np.arange(1, 129)
    p = (1.0 / k) / (1.0 / k).sum()
    freq = np.bincount(z, minlength=129)[1:] / n
    # a few standard deviations of a binomial count on the small sizes, and the mean
    for i in range(8):
        assert abs(freq[i] - p[i]) < 5 * np.sqrt(p[i] * (1 - p[i]) / n), i
    assert abs(z.mean() - (k * p).sum()) < 0.2
    assert np.array_equal(z, datagen.zipf_sizes(n, 1, 128, seed=5))   # seeded
