"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function include/sw_gb300.h declares, and
rejects invalid arguments with status codes before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def swlib():
    from paper_1909_00899_gb300 import build as b
    b.build()
    from paper_1909_00899_gb300 import sw
    return sw


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sw_gb300.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("sw_profile_build", "sw_profile_free", "sw_align_batch",
                     "sw_align_lazyf_batch", "sw_align_pairs", "sw_stream_sync", "sw_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(swlib):
    L = ctypes.CDLL(swlib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(swlib.EXPORTS) == set(declared_functions())


def test_version_and_empty_error(swlib):
    assert swlib.sw_version() == "0.1.0"
    assert isinstance(swlib.sw_last_error(), str)


def test_invalid_arguments_rejected_without_cuda(swlib):
    L = swlib.lib()
    h = ctypes.c_void_p()
    M = (ctypes.c_int8 * 4)(1, -1, -1, 1)
    q = (ctypes.c_uint8 * 3)(0, 1, 0)
    assert L.sw_profile_build(q, -1, M, 2, 0, None, ctypes.byref(h)) == swlib.SW_ERR_INVALID
    assert "qlen" in swlib.sw_last_error()
    assert L.sw_profile_build(q, 3, M, 0, 0, None, ctypes.byref(h)) == swlib.SW_ERR_INVALID
    assert L.sw_profile_build(q, 3, M, 33, 0, None, ctypes.byref(h)) == swlib.SW_ERR_INVALID
    assert L.sw_profile_build(q, 3, None, 2, 0, None, ctypes.byref(h)) == swlib.SW_ERR_INVALID
    assert L.sw_profile_build(q, 3, M, 2, 9, None, ctypes.byref(h)) == swlib.SW_ERR_INVALID
    assert L.sw_profile_build(q, 3, M, 2, 0, None, None) == swlib.SW_ERR_INVALID
    bad = (ctypes.c_uint8 * 3)(0, 5, 0)  # residue >= alphabet
    assert L.sw_profile_build(bad, 3, M, 2, 0, None, ctypes.byref(h)) == swlib.SW_ERR_INVALID
    assert "alphabet" in swlib.sw_last_error()
    # align calls: NULL profile
    assert L.sw_align_batch(None, None, None, 0, 11, 1, None, None) == swlib.SW_ERR_INVALID
    assert L.sw_align_lazyf_batch(None, None, None, 0, 11, 1, None, None) == swlib.SW_ERR_INVALID
    assert L.sw_probe_cell_rate(7, 10, None, None) == swlib.SW_ERR_INVALID
