"""GPU tests of the resident-database API, explicit layouts, the
graph-captured many-query batch, the autotuner, the serving loop and the
bounded stream wait.  Every score is compared bit-exactly with the oracle
(or with a path already compared with it)."""
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
    4: [(2, 16), (2, 32), (16, 8), (32, 8), (32, 12), (32, 16), (32, 20), (32, 24), (32, 32), (32, 40), (64, 8),
        (64, 16), (64, 20), (64, 24), (64, 28), (64, 32), (64, 40)],
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
    out = torch.full((len(queries), h.n), -1, dtype=torch.int32, device="cuda")
    ba = BatchAligner(h, M, 11, 1).prepare(queries, out)
    out.fill_(-1)
    ba.run()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i, q in enumerate(queries):
        np.testing.assert_array_equal(got[i], oracle.gotoh_batch(q, db, off, M, 11, 1), err_msg="query %d" % i)
    out.fill_(-1)
    ba.run()  # replays give the same result
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), got)
    ba.free()


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
