"""GPU test of sw_align_batch_noalloc, the entry point for callers that
cannot let the library allocate device memory (their own allocator owns the
device, or their host forbids plug-in allocations): it must give exactly the
scores of sw_align_batch, on two calls in a row (its fixed scratch array
keeps the previous call's contents), and refuse work that does not fit the
array.  Runs last so that a failure here comes after every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sw():
    from paper_1909_00899_gb300 import sw as swmod
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    swmod.lib()
    return swmod


def _call_noalloc(sw, prof, db_d, off_d, out, o=11, e=1):
    L = sw.lib()
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.sw_align_batch_noalloc(prof.handle, ctypes.c_void_p(db_d.data_ptr()), ctypes.c_void_p(off_d.data_ptr()),
                                  off_d.numel() - 1, o, e, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(stream))
    return rc


def test_noalloc_matches_sw_align_batch_on_two_calls(sw):
    from paper_1909_00899_gb300 import synth
    rng = np.random.default_rng(9001)
    M = synth.protein_matrix(rng)
    db, off = synth.random_db(rng, 3000, 20, "lognormal", median=300, sigma=0.76, lo=20, hi=4000)
    db_d = torch.from_numpy(db).cuda()
    off_d = torch.from_numpy(off).cuda()
    n = len(off) - 1
    cases = ((300, sw.SW_LANE_AUTO), (1500, sw.SW_LANE_AUTO), (700, sw.SW_LANE_I32), (90, sw.SW_LANE_I8X4))
    for m, lane in cases:
        prof = sw.Profile(synth.residues(rng, m, 20), M, lane)
        ref = torch.empty(n, dtype=torch.int32, device="cuda")
        sw.sw_align_batch(prof, db_d, off_d, 11, 1, ref)
        torch.cuda.synchronize()
        want = ref.cpu().numpy()
        for _ in range(2):
            out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            rc = _call_noalloc(sw, prof, db_d, off_d, out)
            assert rc == sw.SW_OK, sw.sw_last_error()
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy(), want, err_msg="m=%d lane=%d" % (m, lane))
        prof.free()


def test_noalloc_refuses_work_beyond_its_array(sw):
    from paper_1909_00899_gb300 import synth
    rng = np.random.default_rng(9002)
    M = synth.protein_matrix(rng)
    # one 5M-residue sequence with a query longer than one chunk: the chunk
    # boundary rows alone need 40 MB, more than the 32 MiB array
    db_d = torch.zeros(5_000_000, dtype=torch.uint8, device="cuda")
    off_d = torch.tensor([0, 5_000_000], dtype=torch.int64, device="cuda")
    prof = sw.Profile(synth.residues(rng, 1500, 20), M, sw.SW_LANE_I32)
    out = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = _call_noalloc(sw, prof, db_d, off_d, out)
    assert rc == sw.SW_ERR_RANGE
    assert "scratch" in sw.sw_last_error()
    torch.cuda.synchronize()
    assert int(out.item()) == -1  # nothing ran
    prof.free()
