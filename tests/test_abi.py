"""The C ABI library builds for sm_103a, loads without a GPU and exports every
function include/wt.h declares; host-side argument checks need no device."""
import ctypes
import os
import re

import pytest

from paper_1610_05994_gb300 import build as B

HEADER = os.path.join(B.ROOT, "include", "wt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(wt_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    return ctypes.CDLL(B.build_library())


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("wt_build", "wt_build_async", "wt_build_batch", "wt_access", "wt_rank", "wt_select",
                 "wt_query_multi", "wt_free", "wt_info", "wt_level_view", "wt_set_allocator",
                 "wt_last_status", "wt_status_string", "wt_wait", "wt_node_starts", "wt_level_step",
                 "wt_build_matrix_async", "wt_merge_async", "wt_build_chunked"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1610_05994_gb300 import wt
    bound = {name for name, _, _ in wt._SIGNATURES}
    assert set(declared_functions()) <= bound


def test_status_strings_and_argument_checks_without_gpu(lib):
    lib.wt_status_string.restype = ctypes.c_char_p
    assert lib.wt_status_string(0) == b"ok"
    assert lib.wt_status_string(2) == b"symbol out of range"
    lib.wt_build.restype = ctypes.c_void_p
    lib.wt_build.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
    # Invalid widths and alphabets are rejected on the host before any CUDA call.
    for n, sigma, w in ((10, 4, 3), (10, 0, 1), (10, 257, 1), (10, 1 << 17, 2), (10, (1 << 28) + 1, 4)):
        assert lib.wt_build(None, n, sigma, w) is None
        assert lib.wt_last_status() == 1
    assert lib.wt_build(None, 5, 4, 1) is None and lib.wt_last_status() == 1


def test_matrix_merge_and_chunked_argument_checks_without_gpu(lib):
    """The wavelet matrix, merge and buffered-build entry points reject bad
    arguments on the host, before any CUDA call."""
    vp, u64 = ctypes.c_void_p, ctypes.c_uint64
    lib.wt_build_matrix_async.restype = vp
    lib.wt_build_matrix_async.argtypes = [vp, u64, u64, ctypes.c_int, vp]
    lib.wt_merge_async.restype = vp
    lib.wt_merge_async.argtypes = [vp, ctypes.c_uint32, vp]
    lib.wt_build_chunked.restype = vp
    lib.wt_build_chunked.argtypes = [vp, u64, u64, ctypes.c_int, u64, vp]
    for n, sigma, w in ((10, 4, 3), (10, 0, 1), (10, 257, 1)):
        assert lib.wt_build_matrix_async(None, n, sigma, w, None) is None
        assert lib.wt_last_status() == 1
    assert lib.wt_merge_async(None, 0, None) is None and lib.wt_last_status() == 1
    null_parts = (vp * 2)()
    assert lib.wt_merge_async(null_parts, 2, None) is None and lib.wt_last_status() == 1
    buf = (ctypes.c_uint8 * 70000)()
    assert lib.wt_build_chunked(None, 10, 4, 1, 4, None) is None and lib.wt_last_status() == 1
    assert lib.wt_build_chunked(buf, 70000, 4, 1, 0, None) is None and lib.wt_last_status() == 1
    # more than 65536 chunks
    assert lib.wt_build_chunked(buf, 70000, 4, 1, 1, None) is None and lib.wt_last_status() == 1
    assert lib.wt_build_chunked(buf, 70000, 4, 3, 100, None) is None and lib.wt_last_status() == 1
