"""GPU tests of the resident-database API, explicit layouts, the
graph-captured many-query batch, the autotuner, the serving loop and the
bounded stream wait.  Every score is compared bit-exactly with the oracle
(or with a path already compared with it)."""
import time

import numpy as np
import pytest

import oracle
from paper_1909_00899_gb300 import synth

from helpers import db_to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ALL_PLANS = {
    1: [(1, 16), (1, 32), (4, 8), (4, 32), (8, 8), (8, 16), (16, 8), (16, 16), (32, 8), (32, 12), (32, 16),
        (8, 32), (16, 32), (32, 32)],
    2: [(8, 8), (8, 16), (16, 8), (16, 16), (32, 8), (32, 12), (32, 16), (16, 32), (32, 24), (32, 32)],
    3: [(8, 16), (16, 16), (32, 16)],
    4: [(2, 16), (2, 32), (16, 8), (16, 32), (32, 8), (32, 12), (32, 16), (32, 20), (32, 24), (32, 32), (32, 40),
        (64, 8), (64, 16), (64, 20), (64, 24), (64, 28), (64, 32), (64, 40)],
}


@pytest.fixture(scope="module")
def sw():
    from paper_1909_00899_gb300 import sw as swmod
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    swmod.lib()
    return swmod


@pytest.fixture(scope="module")
def small_db():
    rng = np.random.default_rng(2001)
    M = synth.protein_matrix(rng)
    lens = np.concatenate([[0, 1, 5], synth.lengths_lognormal(rng, 400, 300, 0.76, 20, 3000)])
    db, off = synth.pack(lens, rng, 20)
    return dict(M=M, db=db, off=off, rng=rng)


def test_db_handle_matches_batch_and_oracle(sw, small_db):
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    rng = np.random.default_rng(2002)
    for m in (40, 300, 700, 1300):
        q = synth.residues(rng, m, 20)
        want = oracle.gotoh_batch(q, db, off, M, 11, 1)
        prof = sw.Profile(q, M)
        a = torch.empty(h.n, dtype=torch.int32, device="cuda")
        b = torch.empty(h.n, dtype=torch.int32, device="cuda")
        c = torch.empty(h.n, dtype=torch.int32, device="cuda")
        sw.sw_align_db(prof, h, 11, 1, a)
        sw.sw_align_batch(prof, db_d, off_d, 11, 1, b)
        prof32 = sw.Profile(q, M, sw.SW_LANE_I32)
        sw.sw_align_lazyf_db(prof32, h, 11, 1, c)
        # end cells against the handle equal the oracle's
        sc = torch.empty(h.n, dtype=torch.int32, device="cuda")
        qe = torch.empty(h.n, dtype=torch.int32, device="cuda")
        re_ = torch.empty(h.n, dtype=torch.int32, device="cuda")
        sw.sw_align_db_ends(prof, h, 11, 1, sc, qe, re_)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a.cpu().numpy(), want)
        np.testing.assert_array_equal(b.cpu().numpy(), want)
        np.testing.assert_array_equal(c.cpu().numpy(), want)
        ws, wq, wr = oracle.gotoh_end_batch(q, db, off, M, 11, 1)
        np.testing.assert_array_equal(sc.cpu().numpy(), ws)
        np.testing.assert_array_equal(qe.cpu().numpy(), wq)
        np.testing.assert_array_equal(re_.cpu().numpy(), wr)
    h.free()


@pytest.mark.parametrize("lane", [1, 2, 3, 4])
def test_every_compiled_layout_is_exact(sw, small_db, lane):
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db[: off[120]], off[:121])
    rng = np.random.default_rng(2003 + lane)
    out = torch.empty(120, dtype=torch.int32, device="cuda")
    for m in (37, 300, 1100):
        q = synth.residues(rng, m, 20)
        want = oracle.gotoh_batch(q, db[: off[120]], off[:121], M, 11, 1)
        want_ends = oracle.gotoh_end_batch(q, db[: off[120]], off[:121], M, 11, 1) if lane == 4 else None
        for (L, S) in ALL_PLANS[lane]:
            prof = sw.Profile(q, M, lane, lanes=L, seg_len=S)
            sw.sw_align_batch(prof, db_d, off_d, 11, 1, out)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy(), want, err_msg="lane %d L=%d S=%d m=%d" % (lane, L, S, m))
            if lane in (1, 2, 4):  # lazy-F runs on these layouts too
                out.fill_(-7)
                sw.sw_align_lazyf_batch(prof, db_d, off_d, 11, 1, out)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(out.cpu().numpy(), want,
                                              err_msg="lazy-F lane %d L=%d S=%d m=%d" % (lane, L, S, m))
            if lane == 4:  # end cells on the split layouts
                qe = torch.empty(120, dtype=torch.int32, device="cuda")
                re_ = torch.empty(120, dtype=torch.int32, device="cuda")
                sw.sw_align_batch_ends(prof, db_d, off_d, 11, 1, out, qe, re_)
                torch.cuda.synchronize()
                ws, wq, wr = want_ends
                np.testing.assert_array_equal(out.cpu().numpy(), ws)
                np.testing.assert_array_equal(re_.cpu().numpy(), wr, err_msg="ends L=%d S=%d m=%d" % (L, S, m))
                np.testing.assert_array_equal(qe.cpu().numpy(), wq, err_msg="ends L=%d S=%d m=%d" % (L, S, m))
            prof.free()


def test_unknown_layout_rejected(sw):
    M = synth.dna_matrix()
    with pytest.raises(sw.SwError) as ei:
        sw.Profile(np.zeros(10, np.uint8), M, sw.SW_LANE_I32, lanes=32, seg_len=5)
    assert ei.value.code == sw.SW_ERR_INVALID
    with pytest.raises(sw.SwError):
        sw.Profile(np.zeros(10, np.uint8), M, sw.SW_LANE_I8X4, lanes=8, seg_len=8)


def test_profile_free_async_in_stream_order(sw, small_db):
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    s = torch.cuda.Stream()
    rng = np.random.default_rng(2004)
    q = synth.residues(rng, 200, 20)
    out = torch.empty(len(off) - 1, dtype=torch.int32, device="cuda")
    for _ in range(3):
        prof = sw.Profile(q, M, stream=s)
        sw.sw_align_batch(prof, db_d, off_d, 11, 1, out, stream=s)
        prof.free_async(s)
    s.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.gotoh_batch(q, db, off, M, 11, 1))


def test_graph_captured_ragged_batch(sw, small_db):
    from paper_1909_00899_gb300.batch import BatchAligner
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    rng = np.random.default_rng(2005)
    qlens = synth.lengths_loguniform(rng, 24, 32, 1500)
    queries = [synth.residues(rng, int(m), 20) for m in qlens]
    for mode in ("multi", "per_query"):
        out = torch.full((len(queries), h.n), -1, dtype=torch.int32, device="cuda")
        ba = BatchAligner(h, M, 11, 1, mode=mode).prepare(queries, out)
        assert (ba.multi is not None) == (mode == "multi")
        out.fill_(-1)
        ba.run()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for i, q in enumerate(queries):
            np.testing.assert_array_equal(got[i], oracle.gotoh_batch(q, db, off, M, 11, 1),
                                          err_msg="query %d, %s" % (i, mode))
        out.fill_(-1)
        ba.run()  # replays give the same result
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), got)
        ba.free()


def _multi_case(sw, M, o, e, seqs, queries, layouts, items_per_group=0):
    """sw_align_multi on a padded score matrix, eagerly and replayed from a
    CUDA graph, every row against the oracle."""
    from helpers import pack_list
    db, off = pack_list(seqs)
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    profs = []
    for q, lay in zip(queries, layouts):
        if lay is None:
            profs.append(sw.Profile(q, M))
        else:
            profs.append(sw.Profile(q, M, sw.SW_LANE_I16X2Q, lanes=lay[0], seg_len=lay[1]))
    batch = sw.Multi(profs, h, items_per_group=items_per_group)
    n = h.n
    out = torch.full((len(queries), n + 5), -7, dtype=torch.int32, device="cuda")  # padded rows
    sw.sw_align_multi(batch, o, e, out)
    torch.cuda.synchronize()
    assert sw.sw_multi_status(batch) == 0  # no bounded wait gave up
    got = out.cpu().numpy()
    for i, q in enumerate(queries):
        want = oracle.gotoh_batch(q, db, off, M, o, e)
        np.testing.assert_array_equal(got[i, :n], want, err_msg="query %d (m=%d, layout %s)"
                                      % (i, len(q), layouts[i]))
        assert np.all(got[i, n:] == -7)  # padding untouched
    # captured into a graph and replayed: the same scores
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st, capture_error_mode="thread_local"):
        sw.sw_align_multi(batch, o, e, out, stream=st)
    out.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy()[:, :n], got[:, :n])
    batch.free()
    for p in profs:
        p.free()
    h.free()
    return got[:, :n], db, off


def test_long_query_on_db_handle_captures_into_a_graph(sw, small_db):
    """A 5000-residue query (several chunks, boundary rows sized from the
    handle's cached residue count) through sw_align_db is captured into a
    CUDA graph with no host synchronisation, and the replay equals the
    oracle; single-chunk sw_align_batch calls capture too."""
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    rng = np.random.default_rng(2013)
    q_long = synth.residues(rng, 5000, 20)
    q_short = synth.residues(rng, 400, 20)
    p_long = sw.Profile(q_long, M)
    p_short = sw.Profile(q_short, M)
    assert p_long.plan()["chunks"] > 1 and p_short.plan()["chunks"] == 1
    a = torch.full((h.n,), -7, dtype=torch.int32, device="cuda")
    b = torch.full((h.n,), -7, dtype=torch.int32, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):  # eager once (kernel attributes, pool)
        sw.sw_align_db(p_long, h, 11, 1, a, stream=st)
        sw.sw_align_batch(p_short, db_d, off_d, 11, 1, b, stream=st)
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st, capture_error_mode="thread_local"):
        sw.sw_align_db(p_long, h, 11, 1, a, stream=st)
        sw.sw_align_batch(p_short, db_d, off_d, 11, 1, b, stream=st)
    a.fill_(-1)
    b.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.cpu().numpy(), oracle.gotoh_batch(q_long, db, off, M, 11, 1))
    np.testing.assert_array_equal(b.cpu().numpy(), oracle.gotoh_batch(q_short, db, off, M, 11, 1))
    p_long.free()
    p_short.free()
    h.free()


def test_batched_launch_every_layout_exact(sw):
    """One persistent launch per layout over every (query, tile) unit:
    queries on every split layout of 16+ virtual lanes (one and several
    chunks, the chunk boundary rows in per-group slots), empty and
    one-residue queries and sequences, copies of long queries planted in
    long sequences (pairs whose score could pass the packed lanes' range
    go to the int32 launch, here above 28,543), scores into padded rows."""
    rng = np.random.default_rng(2010)
    M = synth.protein_matrix(rng)
    lens = np.concatenate([[0, 1, 2, 5], synth.lengths_lognormal(rng, 150, 300, 0.76, 20, 3000)])
    seqs = [synth.residues(rng, int(x), 20) for x in lens]
    layouts = [(16, 8), (16, 32), (32, 8), (32, 12), (32, 16), (32, 20), (32, 24), (32, 32), (32, 40), (64, 8),
               (64, 16), (64, 20), (64, 24), (64, 28), (64, 32), (64, 40)]
    queries, lays = [], []
    for k, lay in enumerate(layouts):
        for m in (max(1, lay[0] * lay[1] - 3), 2 * lay[0] * lay[1] + 5):  # one chunk, three chunks
            queries.append(synth.residues(rng, int(m), 20))
            lays.append(lay)
    long_q = synth.residues(rng, 6000, 20)
    queries += [np.zeros(0, np.uint8), synth.residues(rng, 1, 20), synth.residues(rng, 2700, 20), long_q]
    lays += [None, None, None, None]
    seqs.append(np.concatenate([synth.residues(rng, 30, 20), long_q[1000:5200], synth.residues(rng, 20, 20)]))
    seqs.append(np.concatenate([queries[-2][100:2650], synth.residues(rng, 400, 20)]))
    got, db, off = _multi_case(sw, M, 11, 1, seqs, queries, lays)
    assert got[-1, -2] > 32767  # overflowed the packed lanes, rescored by the int32 launch
    assert got[-2, -1] > 2550 * 4
    # the fused-chunk tiles (items_per_group > 0) on the multi-chunk queries
    got2, _, _ = _multi_case(sw, M, 11, 1, seqs, queries, lays, items_per_group=3)
    np.testing.assert_array_equal(got2, got)


def test_batched_launch_general_pass_and_dna(sw):
    """The batched launch with mismatch scores below -o (the general
    corrected pass) and with DNA scoring (most h below zero: the always-
    corrected pass's floor on the diagonal), gap extension 0 (carries that
    never decay) and e = o, query-side insertions across many lanes and
    chunks."""
    from helpers import gap_adversary
    rng = np.random.default_rng(2011)
    queries, refs = gap_adversary(rng, 4, 20, ylo=60, yhi=500)
    refs += [synth.residues(rng, int(n), 4) for n in (1, 7, 900, 2500)]
    queries = queries[:6] + [synth.residues(rng, n, 4) for n in (70, 700, 2100, 4000)]
    for o, e, mm in ((6, 1, -4), (3, 1, -5), (5, 5, -2), (4, 0, -2), (2, 0, -5)):
        M = synth.dna_matrix(match=2, mismatch=mm)
        got, _, _ = _multi_case(sw, M, o, e, refs, queries, [None] * len(queries))
        if mm < -o:  # the general pass in the fused-chunk tiles as well
            got2, _, _ = _multi_case(sw, M, o, e, refs, queries, [None] * len(queries), items_per_group=2)
            np.testing.assert_array_equal(got2, got)


def test_batched_launch_wait_bound_sets_status(sw, small_db):
    """The chunk walk's bounded wait: with every wait made to await a mark
    no phase writes, each runs out, the status word reads 1 (then clears),
    the launch ends and the context stays usable; with the bound restored
    the next call on the same handle is exact and reads 0."""
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    q = synth.residues(np.random.default_rng(2014), 700, 20)
    p = sw.Profile(q, M, sw.SW_LANE_I16X2Q, lanes=16, seg_len=8)  # 128 positions a chunk: 6 chunks
    assert p.plan()["chunks"] > 1
    batch = sw.Multi([p], h)
    out = torch.full((1, h.n), -1, dtype=torch.int32, device="cuda")
    sw.sw_multi_set_wait(batch, 64, unreachable=True)
    t0 = time.time()
    sw.sw_align_multi(batch, 11, 1, out)
    torch.cuda.synchronize()
    assert time.time() - t0 < 30
    assert sw.sw_multi_status(batch) == 1
    assert sw.sw_multi_status(batch) == 0  # read clears it
    sw.sw_multi_set_wait(batch, 0)
    out.fill_(-1)
    sw.sw_align_multi(batch, 11, 1, out)
    torch.cuda.synchronize()
    assert sw.sw_multi_status(batch) == 0
    np.testing.assert_array_equal(out.cpu().numpy()[0], oracle.gotoh_batch(q, db, off, M, 11, 1))
    batch.free()
    p.free()
    h.free()


def test_batched_launch_empty_batch_and_empty_database(sw, small_db):
    """No queries, an empty database, and a batch of only empty queries:
    the calls succeed, launch nothing that writes outside the score rows,
    and empty queries score 0."""
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    none = sw.Multi([], h)
    out = torch.full((1, h.n), -3, dtype=torch.int32, device="cuda")
    sw.sw_align_multi(none, 11, 1, out)
    torch.cuda.synchronize()
    assert (out == -3).all()
    assert sw.sw_multi_status(none) == 0
    none.free()
    empties = [sw.Profile(np.zeros(0, np.uint8), M) for _ in range(2)]
    batch = sw.Multi(empties, h)
    out2 = torch.full((2, h.n + 3), -3, dtype=torch.int32, device="cuda")
    sw.sw_align_multi(batch, 11, 1, out2)
    torch.cuda.synchronize()
    got = out2.cpu().numpy()
    assert (got[:, :h.n] == 0).all() and (got[:, h.n:] == -3).all()
    batch.free()
    empty_db = sw.Database(torch.zeros(0, dtype=torch.uint8, device="cuda"),
                           torch.zeros(1, dtype=torch.int64, device="cuda"))
    q = sw.Profile(synth.residues(np.random.default_rng(2016), 3000, 20), M)
    b2 = sw.Multi([q], empty_db)
    sw.sw_align_multi(b2, 11, 1, torch.empty((1, 1), dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    assert sw.sw_multi_status(b2) == 0
    b2.free()
    for p in empties + [q]:
        p.free()
    empty_db.free()
    h.free()


def test_batch_aligner_falls_back_to_per_query_calls(sw, small_db):
    """Gap costs beyond the packed lanes of the batched launch (o > 127) and
    profiles on other lane types: the aligner captures per-query calls
    instead, with the same exact scores."""
    from paper_1909_00899_gb300.batch import BatchAligner
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    rng = np.random.default_rng(2017)
    queries = [synth.residues(rng, m, 20) for m in (40, 300, 1500)]
    for o, e, lane in ((150, 3, sw.SW_LANE_AUTO), (11, 1, sw.SW_LANE_I32)):
        out = torch.full((len(queries), h.n), -1, dtype=torch.int32, device="cuda")
        ba = BatchAligner(h, M, o, e, lane=lane).prepare(queries, out)
        assert ba.multi is None and ba.mode == "per_query"
        ba.run()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for i, q in enumerate(queries):
            np.testing.assert_array_equal(got[i], oracle.gotoh_batch(q, db, off, M, o, e), err_msg="o=%d" % o)
        ba.free()
    h.free()


def test_batched_launch_rejects_what_it_cannot_run(sw, small_db):
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    q = synth.residues(np.random.default_rng(2012), 300, 20)
    p32 = sw.Profile(q, M, sw.SW_LANE_I32)
    with pytest.raises(sw.SwError):
        sw.Multi([p32], h)  # not the split lane type
    pa = sw.Profile(q, M)
    batch = sw.Multi([pa], h)
    out = torch.zeros((1, h.n), dtype=torch.int32, device="cuda")
    with pytest.raises(sw.SwError) as ex:
        sw.sw_align_multi(batch, 200, 1, out)  # gap open beyond the packed lanes
    assert ex.value.code == sw.SW_ERR_RANGE
    with pytest.raises(sw.SwError):
        sw.sw_align_multi(batch, 11, 12, out)  # e > o
    batch.free()
    p32.free()
    pa.free()


def test_autotuner_table_is_exact(sw, small_db):
    from paper_1909_00899_gb300 import autotune
    from paper_1909_00899_gb300.batch import BatchAligner
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    table = autotune.tune(h, M, 11, 1, lengths=[100, 600], reps=1)
    assert table.plan(100) is not None and table.plan(600) is not None
    rt = autotune.Table.from_json(table.to_json())
    assert rt.plan(600) == table.plan(600)
    rng = np.random.default_rng(2006)
    queries = [synth.residues(rng, m, 20) for m in (90, 120, 500, 600)]
    out = torch.empty((len(queries), h.n), dtype=torch.int32, device="cuda")
    ba = BatchAligner(h, M, 11, 1, table=table).prepare(queries, out)
    ba.run()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i, q in enumerate(queries):
        np.testing.assert_array_equal(got[i], oracle.gotoh_batch(q, db, off, M, 11, 1))
    ba.free()


def test_autotuner_batched_timing_is_exact(sw, small_db):
    """The tuner's batched timing (one sw_align_multi over k queries per
    layout) gives a table whose plans the batched launch runs exactly."""
    from paper_1909_00899_gb300 import autotune
    from paper_1909_00899_gb300.batch import BatchAligner
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    table = autotune.tune(h, M, 11, 1, lengths=[150, 1500], reps=1, lanes=(sw.SW_LANE_I16X2Q,), batched=2)
    for m in (150, 1500):
        assert table.plan(m) is not None and table.plan(m)[0] == sw.SW_LANE_I16X2Q
        assert all(c[3] > 0 for c in table.entries[autotune.bin_of(m)])
    rng = np.random.default_rng(2015)
    queries = [synth.residues(rng, m, 20) for m in (120, 150, 1400, 1500)]
    out = torch.empty((len(queries), h.n), dtype=torch.int32, device="cuda")
    ba = BatchAligner(h, M, 11, 1, table=table).prepare(queries, out)
    assert ba.multi is not None
    ba.run()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i, q in enumerate(queries):
        np.testing.assert_array_equal(got[i], oracle.gotoh_batch(q, db, off, M, 11, 1))
    ba.free()
    h.free()


def test_serving_admits_by_available_device_memory(sw, small_db, monkeypatch):
    """Admission also checks the memory the device has now: with the query
    reporting too little, requests wait while others of the server run and
    are refused when nothing of its own is running to free memory; with the
    real query every request is served, and sw_mem_available is at most the
    device's total."""
    from paper_1909_00899_gb300 import serve
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    rng = np.random.default_rng(2014)
    queries = [synth.residues(rng, int(m), 20) for m in (60, 300, 900, 120)]
    avail = sw.sw_mem_available()
    assert 0 < avail <= torch.cuda.get_device_properties(0).total_memory
    srv = serve.Server(h, M, 11, 1, slots=2)
    reqs = srv.run(queries)
    assert srv.rejected == 0 and all(r.scores is not None for r in reqs)
    # a device that has only a few bytes left: nothing can be admitted
    monkeypatch.setattr(serve.sw, "sw_mem_available", lambda: 1024)
    srv2 = serve.Server(h, M, 11, 1, slots=2)
    reqs2 = srv2.run(queries)
    assert srv2.rejected == len(queries) and all(r.scores is None for r in reqs2)
    # memory short only while the first request runs: the others wait, then run
    state = {"calls": 0}

    def flaky():
        state["calls"] += 1
        return avail if state["calls"] == 1 or srv3.in_use == 0 else 1024

    monkeypatch.setattr(serve.sw, "sw_mem_available", flaky)
    srv3 = serve.Server(h, M, 11, 1, slots=4)
    reqs3 = srv3.run(queries)
    assert srv3.rejected == 0 and srv3.waited_for_memory > 0
    for a, b in zip(reqs, reqs3):
        np.testing.assert_array_equal(a.scores, b.scores)
    h.free()


def test_serving_results_same_alone_and_in_the_mix(sw, small_db):
    from paper_1909_00899_gb300 import serve
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    rng = np.random.default_rng(2007)
    qlens = synth.lengths_loguniform(rng, 30, 50, 2000)
    queries = [synth.residues(rng, int(m), 20) for m in qlens]
    # alone: one request at a time
    alone = serve.Server(h, M, 11, 1, slots=1).run(queries)
    # in the mix: Poisson arrivals, 4 slots, overlapping on the device
    srv = serve.Server(h, M, 11, 1, slots=4)
    mixed = srv.run(queries, serve.poisson_arrivals(rng, len(queries), rate=400.0))
    for a, b in zip(alone, mixed):
        np.testing.assert_array_equal(a.scores, b.scores)
    for i in (0, 7, 19):
        np.testing.assert_array_equal(mixed[i].scores, oracle.gotoh_batch(queries[i], db, off, M, 11, 1))
    st = serve.latency_stats(mixed)
    assert st["n"] == len(queries) and st["p99_ms"] >= st["p50_ms"] > 0
    assert srv.in_use == 0


def test_serving_memory_budget_admission(sw, small_db):
    from paper_1909_00899_gb300 import serve
    M, db, off = small_db["M"], small_db["db"], small_db["off"]
    db_d, off_d = db_to_dev(db, off)
    h = sw.Database(db_d, off_d)
    rng = np.random.default_rng(2008)
    queries = [synth.residues(rng, m, 20) for m in (100, 200, 150, 120)]
    probe = serve.Server(h, M, 11, 1, slots=4)
    one = max(probe.request_bytes(len(q)) for q in queries)
    srv = serve.Server(h, M, 11, 1, slots=4, mem_budget=one)  # one request at a time
    reqs = srv.run(queries)
    for r, q in zip(reqs, queries):
        np.testing.assert_array_equal(r.scores, oracle.gotoh_batch(q, db, off, M, 11, 1))
    # a request that can never fit is refused, the others are served
    tiny = serve.Server(h, M, 11, 1, slots=2, mem_budget=probe.request_bytes(100))
    reqs = tiny.run([queries[0], synth.residues(rng, 3000, 20)])
    assert reqs[0].scores is not None and reqs[1].scores is None and tiny.rejected == 1


def test_stream_sync_times_out_while_busy(sw):
    """A bounded wait on a busy stream returns SW_ERR_TIMEOUT (no fault, the
    context stays usable), then a long enough wait succeeds."""
    rng = np.random.default_rng(2009)
    M = synth.protein_matrix(rng)
    db, off = synth.random_db(rng, 20000, 20, "uniform", lo=800, hi=1200)
    db_d, off_d = db_to_dev(db, off)
    s = torch.cuda.Stream()
    prof = sw.Profile(synth.residues(rng, 4000, 20), M, stream=s)
    out = torch.empty(20000, dtype=torch.int32, device="cuda")
    sw.sw_align_batch(prof, db_d, off_d, 11, 1, out, stream=s)
    with pytest.raises(sw.SwError) as ei:
        sw.sw_stream_sync(s, 0)
    assert ei.value.code == sw.SW_ERR_TIMEOUT
    sw.sw_stream_sync(s, 120_000)
