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
    cps = ctypes.c_double(0.0)
    assert L.sw_probe_cell_rate_pass(1, 3, 10, ctypes.byref(cps), None) == swlib.SW_ERR_INVALID
    assert L.sw_probe_cell_rate_pass(1, 2, 10, ctypes.byref(cps), None) == swlib.SW_ERR_INVALID  # int32: no AC pass
    assert "s16x2" in swlib.sw_last_error()
    assert L.sw_probe_cell_rate_pass(3, 1, 10, ctypes.byref(cps), None) == swlib.SW_ERR_INVALID
    assert "s8x4" in swlib.sw_last_error()
    # batched-launch handle calls: NULL handle
    assert L.sw_multi_set_wait(None, 0, 0) == swlib.SW_ERR_INVALID
    st = ctypes.c_int32(0)
    assert L.sw_multi_status(None, ctypes.byref(st), None) == swlib.SW_ERR_INVALID
    assert L.sw_align_multi(None, 11, 1, None, 0, None) == swlib.SW_ERR_INVALID


def test_plan_query_covers_the_query_host_only(swlib):
    """sw_plan_query (no CUDA call): every lane type's plan covers the query
    with the fewest chunks of its layout; the automatic plan uses the split
    s16x2 lanes, wastes under half a chunk for queries of 128+ residues and
    picks the layouts the measured rates favour at the benchmark lengths."""
    for lane in (0, 1, 2, 3, 4):
        for m in (0, 1, 7, 64, 100, 128, 129, 300, 512, 777, 1024, 2048, 3000, 5000, 12345):
            p = swlib.sw_plan_query(m, lane)
            QC = p["lanes"] * p["seg_len"]
            assert QC > 0
            assert p["chunks"] == (m + QC - 1) // QC
            assert p["lane_type"] == lane if lane else p["lane_type"] in (2, 4)
            if lane == 0 and m >= 128:
                assert m / (p["chunks"] * QC) > 0.5
    picks = {m: swlib.sw_plan_query(m) for m in (128, 512, 2048, 5000)}
    assert picks[128] == dict(lanes=16, seg_len=8, chunks=1, lane_type=4)
    assert picks[512] == dict(lanes=16, seg_len=32, chunks=1, lane_type=4)
    assert picks[2048] == dict(lanes=64, seg_len=32, chunks=1, lane_type=4)
    assert picks[5000] == dict(lanes=32, seg_len=40, chunks=4, lane_type=4)
    # lengths between the benchmark's: the layout whose chunk the query fills
    # best at its measured rate (16 threads x 12/20/24/32, 32 threads x 28)
    mids = {300: (32, 12, 1), 600: (32, 20, 1), 700: (32, 24, 1), 1000: (32, 32, 1), 1700: (64, 28, 1),
            3500: (64, 28, 2)}
    for m, (lanes, seg, chunks) in mids.items():
        assert swlib.sw_plan_query(m) == dict(lanes=lanes, seg_len=seg, chunks=chunks, lane_type=4), m
        assert m / (chunks * lanes * seg) > 0.75
    with pytest.raises(swlib.SwError):
        swlib.sw_plan_query(-1)
    with pytest.raises(swlib.SwError):
        swlib.sw_plan_query(10, 9)


def test_autotune_table_plans_each_query_length():
    """The tuned table keeps every layout's rate per processed cell and picks
    per exact length: a layout whose chunks the query fills beats a faster
    one it would mostly pad (host logic only)."""
    from paper_1909_00899_gb300 import autotune as at
    Q = 4  # split s16x2 lane type
    t = at.Table({4096: [(Q, 64, 20, 5000.0), (Q, 64, 32, 5000.0), (Q, 64, 24, 4800.0)]}, "dev")
    assert t.plan(2100) == (Q, 64, 20)   # 2 chunks of 1280: 82 % real positions
    assert t.plan(3000) == (Q, 64, 24)   # 2 chunks of 1536: 98 %
    assert t.plan(4000) == (Q, 64, 32)   # 2 chunks of 2048: 98 %
    assert t.plan(50) is None            # untuned bin: the library's own plan
    # expected rate: measured rate x real fraction / chunk cost
    assert abs(at.expected_gcups(4000, 64, 32, 5000.0) - 5000.0 * 4000 / 4096 / 1.015) < 1e-9
    assert at.chunks_of(5000, 64, 20) == 4 and not at.admissible(100, 64, 32)
    rt = at.Table.from_json(t.to_json())
    assert all(rt.plan(m) == t.plan(m) for m in (2100, 3000, 4000))
    # tables saved before the per-layout format: one layout per bin
    old = at.Table.from_json({"device": "dev", "entries": {"4096": [Q, 64, 20, 4147.8]}})
    assert old.plan(3000) == (Q, 64, 20)
