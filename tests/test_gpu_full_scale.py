"""GPU parity at the benchmark's full sizes, in the launch configuration the
benchmark times (automatic layouts, the four queries spread over side
streams): sampled outputs against the oracle one by one, the longest
database sequences included, and properties of every output (scan-F equal
to lazy-F, bounds that hold at any size)."""
import numpy as np
import pytest

import oracle
from paper_1909_00899_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sw():
    from paper_1909_00899_gb300 import sw as swmod
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    swmod.lib()
    return swmod


def _subset(db, off, ids):
    parts = [db[off[i]:off[i + 1]] for i in ids]
    sub_off = np.zeros(len(ids) + 1, dtype=np.int64)
    np.cumsum([len(p) for p in parts], out=sub_off[1:])
    return np.concatenate(parts).astype(np.uint8), sub_off


@pytest.fixture(scope="module")
def scale():
    """Queries m = 128, 512, 2048, 5000 vs 100,000 log-normal sequences
    (40 M residues): the benchmark step."""
    return synth.workload_protein_scale()


@pytest.mark.parametrize("lane", ["auto", "i32"])
def test_scale_step_sampled_and_properties(sw, scale, lane):
    """The benchmark step at full size on the automatic lanes (split s16x2
    with int32 rescore) and on int32 lanes throughout (the plain method's
    own lane type, which the benchmark times beside it)."""
    lane_type = {"auto": sw.SW_LANE_AUTO, "i32": sw.SW_LANE_I32}[lane]
    w = scale
    M, o, e = w["M"], w["o"], w["e"]
    n = len(w["off"]) - 1
    db_d = torch.from_numpy(w["db"]).cuda()
    off_d = torch.from_numpy(w["off"]).cuda()
    main = torch.cuda.current_stream()
    side = [torch.cuda.Stream() for _ in range(4)]
    scan = [torch.full((n,), -7, dtype=torch.int32, device="cuda") for _ in w["queries"]]
    lazy = [torch.full((n,), -7, dtype=torch.int32, device="cuda") for _ in w["queries"]]
    profs = []
    fork = torch.cuda.Event()
    fork.record(main)
    for i, q in enumerate(w["queries"]):
        st = side[i]
        st.wait_event(fork)
        p = sw.Profile(q, M, lane_type, stream=st)
        sw.sw_align_batch(p, db_d, off_d, o, e, scan[i], stream=st)
        profs.append(p)
    torch.cuda.synchronize()
    lens = np.diff(w["off"])
    rng = np.random.default_rng(77)
    ids = np.unique(np.concatenate([rng.choice(n, 96, replace=False), np.argsort(lens)[-8:]]))
    sub_db, sub_off = _subset(w["db"], w["off"], ids)
    maxdiag = int(M.max())
    for i, q in enumerate(w["queries"]):
        got = scan[i].cpu().numpy()
        want = oracle.gotoh_batch(q, sub_db, sub_off, M, o, e)
        np.testing.assert_array_equal(got[ids], want, err_msg="m=%d lane=%s" % (len(q), lane))
        # every output: 0 <= score <= max(M) * min(m, n)
        assert got.min() >= 0
        assert np.all(got <= maxdiag * np.minimum(len(q), lens))
        # every output: lazy-F (the plain method, on its own kernel) agrees
        p32 = sw.Profile(q, M, sw.SW_LANE_I16X2)
        sw.sw_align_lazyf_batch(p32, db_d, off_d, o, e, lazy[i])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(lazy[i].cpu().numpy(), got, err_msg="scan vs lazy m=%d" % len(q))
        p32.free()
    for p in profs:
        p.free()


def test_reads_vs_windows_full_size_sampled(sw):
    """1M reads vs their own 2 kbp windows through the automatic pair lane:
    2000 sampled pairs against the oracle, every pair against lazy-F."""
    w = synth.workload_reads(n_pairs=1_000_000)
    n = len(w["q_off"]) - 1
    qd, qo = torch.from_numpy(w["q"]).cuda(), torch.from_numpy(w["q_off"]).cuda()
    rd, ro = torch.from_numpy(w["r"]).cuda(), torch.from_numpy(w["r_off"]).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    sw.sw_align_pairs(qd, qo, rd, ro, w["M"], w["o"], w["e"], out)
    got = out.cpu().numpy()
    ids = np.sort(np.random.default_rng(78).choice(n, 2000, replace=False))
    q = [w["q"][w["q_off"][i]:w["q_off"][i + 1]] for i in ids]
    r = [w["r"][w["r_off"][i]:w["r_off"][i + 1]] for i in ids]
    qo_s = np.zeros(len(ids) + 1, np.int64)
    ro_s = np.zeros(len(ids) + 1, np.int64)
    np.cumsum([len(x) for x in q], out=qo_s[1:])
    np.cumsum([len(x) for x in r], out=ro_s[1:])
    want = oracle.gotoh_pairs(np.concatenate(q), qo_s, np.concatenate(r), ro_s, w["M"], w["o"], w["e"])
    np.testing.assert_array_equal(got[ids], want)
    lz = torch.empty(n, dtype=torch.int32, device="cuda")
    sw.sw_align_lazyf_pairs(qd, qo, rd, ro, w["M"], w["o"], w["e"], lz)
    np.testing.assert_array_equal(lz.cpu().numpy(), got)
    assert got.max() > 127  # the packed lanes overflowed somewhere and were rescored


def _sampled_check(got, q, db, off, M, o, e, ids, err):
    sub_db, sub_off = _subset(db, off, ids)
    want = oracle.gotoh_batch(q, sub_db, sub_off, M, o, e)
    np.testing.assert_array_equal(got[ids], want, err_msg=err)


def test_ragged_batch_full_size_sampled(sw):
    """The ragged batch at its full database size (200k log-normal
    sequences, 80 M residues) in the benchmark's launch configuration:
    length-stratified queries from the 10,000 (32..4096), an autotuned
    split layout per length bin, one batched launch per layout (and the
    int32 launch of the longest pairs) in one graph.  Sampled outputs against the oracle (the longest sequences
    included), every output against the direct database call and within
    0 <= score <= max(M) * min(m, n)."""
    from paper_1909_00899_gb300 import autotune
    from paper_1909_00899_gb300.batch import BatchAligner
    rng = synth.rng_for(3)
    M = synth.protein_matrix(rng)
    qlens_all = synth.lengths_loguniform(rng, 10_000, 32, 4096)
    db, off = synth.random_db(rng, 200_000, 20, "lognormal", median=300, sigma=0.76, lo=20, hi=35000)
    order = np.argsort(qlens_all, kind="stable")
    pick = order[np.linspace(0, len(order) - 1, 10).astype(int)]
    queries = [synth.residues(np.random.default_rng([5, int(i)]), int(qlens_all[i]), 20) for i in pick]
    db_d, off_d = torch.from_numpy(db).cuda(), torch.from_numpy(off).cuda()
    h = sw.Database(db_d, off_d)
    table = autotune.tune(h, M, 11, 1, lengths=[48, 400, 3200], reps=1, lanes=(sw.SW_LANE_I16X2Q,))
    out = torch.full((len(queries), h.n), -7, dtype=torch.int32, device="cuda")
    ba = BatchAligner(h, M, 11, 1, table=table, streams=4).prepare(queries, out)
    assert ba.multi is not None  # one batched launch per layout
    ba.run()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    lens = np.diff(off)
    ids = np.unique(np.concatenate([np.random.default_rng(79).choice(h.n, 80, replace=False),
                                    np.argsort(lens)[-4:]]))
    direct = torch.empty(h.n, dtype=torch.int32, device="cuda")
    for i, q in enumerate(queries):
        _sampled_check(got[i], q, db, off, M, 11, 1, ids, "query %d (m=%d)" % (i, len(q)))
        p = sw.Profile(q, M)
        sw.sw_align_db(p, h, 11, 1, direct)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got[i], direct.cpu().numpy(), err_msg="graph vs direct, m=%d" % len(q))
        p.free()
        assert got[i].min() >= 0 and np.all(got[i] <= int(M.max()) * np.minimum(len(q), lens))
    ba.free()


def test_serving_full_size_sampled(sw):
    """Serving against the full resident database (1M log-normal sequences,
    about 350 M residues) in the benchmark's configuration (four slots, a
    48 GB budget, Poisson arrivals): every request's scores the same alone
    and in the mix, and sampled against the oracle."""
    from paper_1909_00899_gb300 import serve
    rng = synth.rng_for(4)
    M = synth.protein_matrix(rng)
    db, off = synth.random_db(rng, 1_000_000, 20, "lognormal", median=300, sigma=0.555, lo=20, hi=35000)
    assert 3.0e8 < off[-1] < 4.0e8
    db_d, off_d = torch.from_numpy(db).cuda(), torch.from_numpy(off).cuda()
    h = sw.Database(db_d, off_d)
    r = np.random.default_rng([6, 99])
    qlens = synth.lengths_loguniform(r, 6, 50, 10_000)
    queries = [synth.residues(r, int(m), 20) for m in qlens]
    alone = serve.Server(h, M, 11, 1, slots=1, mem_budget=48 << 30).run(queries)
    srv = serve.Server(h, M, 11, 1, slots=4, mem_budget=48 << 30)
    mixed = srv.run(queries, serve.poisson_arrivals(np.random.default_rng(9), len(queries), 20.0))
    lens = np.diff(off)
    ids = np.unique(np.concatenate([np.random.default_rng(80).choice(h.n, 60, replace=False),
                                    np.argsort(lens)[-3:]]))
    for k, (a, b) in enumerate(zip(alone, mixed)):
        np.testing.assert_array_equal(a.scores, b.scores, err_msg="request %d alone vs mixed" % k)
        _sampled_check(b.scores, queries[k], db, off, M, 11, 1, ids, "request %d (m=%d)" % (k, len(queries[k])))
    assert srv.in_use == 0
