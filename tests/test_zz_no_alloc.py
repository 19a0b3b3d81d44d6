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
    """Scores equal to the oracle's and to sw_align_batch's, on two calls in
    a row, for one- and multi-chunk queries on packed and int32 lanes.  The
    database holds copies of each query's middle, so that alignments
    overflow the packed lanes (above 127 for s8x4, above the s16 range for
    the 5000-residue query) and go through the int32 rescore list kept in
    the array."""
    import oracle
    from paper_1909_00899_gb300 import synth
    rng = np.random.default_rng(9001)
    M = synth.protein_matrix(rng)
    cases = ((300, sw.SW_LANE_AUTO), (1500, sw.SW_LANE_AUTO), (700, sw.SW_LANE_I32), (90, sw.SW_LANE_I8X4),
             (5000, sw.SW_LANE_AUTO))
    queries = [synth.residues(rng, m, 20) for m, _ in cases]
    base, boff = synth.random_db(rng, 1500, 20, "lognormal", median=300, sigma=0.76, lo=20, hi=4000)
    seqs = [base[boff[i]:boff[i + 1]] for i in range(len(boff) - 1)]
    planted = []
    for q in queries:  # each query's middle 90 % (the longest: all of it), between random flanks
        k = len(q) // 20 if len(q) < 5000 else 0
        planted.append(len(seqs))
        seqs.append(np.concatenate([synth.residues(rng, 40, 20), q[k:len(q) - k], synth.residues(rng, 25, 20)]))
    off = np.zeros(len(seqs) + 1, np.int64)
    np.cumsum([len(x) for x in seqs], out=off[1:])
    db = np.concatenate(seqs).astype(np.uint8)
    db_d = torch.from_numpy(db).cuda()
    off_d = torch.from_numpy(off).cuda()
    n = len(off) - 1
    for (m, lane), q in zip(cases, queries):
        want = oracle.gotoh_batch(q, db, off, M, 11, 1)
        prof = sw.Profile(q, M, lane)
        ref = torch.empty(n, dtype=torch.int32, device="cuda")
        sw.sw_align_batch(prof, db_d, off_d, 11, 1, ref)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ref.cpu().numpy(), want, err_msg="sw_align_batch m=%d lane=%d" % (m, lane))
        for _ in range(2):
            out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            rc = _call_noalloc(sw, prof, db_d, off_d, out)
            assert rc == sw.SW_OK, sw.sw_last_error()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_array_equal(got, want, err_msg="m=%d lane=%d" % (m, lane))
        prof.free()
    # the planted copies did overflow: the s8x4 query's and the long query's
    # scores come from the int32 rescore
    assert want[planted[-1]] > 32767
    s8 = oracle.gotoh_batch(queries[3], db, off, M, 11, 1)
    assert s8[planted[3]] > 127


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
