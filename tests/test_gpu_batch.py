"""GPU parity of sw_align_batch (scan-F, every lane type) and
sw_align_lazyf_batch against the CPU oracle: bit-exact int32 scores."""
import numpy as np
import pytest

import oracle
from paper_1909_00899_gb300 import synth

from helpers import db_to_dev, gap_adversary, pack_list

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LANES = ["i32", "i16x2", "i16x2q", "i8x4", "auto", "lazyf", "lazyf16", "lazyf16q"]


@pytest.fixture(scope="module")
def sw():
    from paper_1909_00899_gb300 import sw as swmod
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    swmod.lib()
    return swmod


def run(sw, kind, query, M, db_d, off_d, o, e):
    lane = {"i32": sw.SW_LANE_I32, "i16x2": sw.SW_LANE_I16X2, "i16x2q": sw.SW_LANE_I16X2Q,
            "i8x4": sw.SW_LANE_I8X4, "auto": sw.SW_LANE_AUTO, "lazyf": sw.SW_LANE_I32,
            "lazyf16": sw.SW_LANE_I16X2, "lazyf16q": sw.SW_LANE_I16X2Q}[kind]
    prof = sw.Profile(query, M, lane)
    n = off_d.numel() - 1
    out = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    if kind.startswith("lazyf"):
        sw.sw_align_lazyf_batch(prof, db_d, off_d, o, e, out)
    else:
        sw.sw_align_batch(prof, db_d, off_d, o, e, out)
    torch.cuda.synchronize()
    res = out[:n].cpu().numpy()
    prof.free()
    return res


@pytest.mark.parametrize("kind", LANES)
def test_protein_query256_vs_1000(sw, kind):
    """One protein query of 256 vs 1000 sequences of length U{50..500}."""
    w = synth.workload_protein_small()
    db_d, off_d = db_to_dev(w["db"], w["off"])
    want = oracle.gotoh_batch(w["query"], w["db"], w["off"], w["M"], w["o"], w["e"])
    got = run(sw, kind, w["query"], w["M"], db_d, off_d, w["o"], w["e"])
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("kind", LANES)
def test_query_lengths_span_plans_and_chunks(sw, kind):
    """Query lengths around every plan boundary (32/64/128/256/512 positions)
    and multi-chunk queries, against a ragged db with empty and 1-residue
    sequences."""
    rng = np.random.default_rng(1001)
    M = synth.protein_matrix(rng)
    lens = np.concatenate([[0, 1, 2, 3, 0, 17], rng.integers(1, 700, 120)])
    db, off = synth.pack(lens.astype(np.int64), rng, 20)
    db_d, off_d = db_to_dev(db, off)
    for qlen in (1, 7, 31, 33, 64, 100, 129, 255, 257, 511, 512, 513, 1100, 1600):
        q = synth.residues(rng, qlen, 20)
        want = oracle.gotoh_batch(q, db, off, M, 11, 1)
        got = run(sw, kind, q, M, db_d, off_d, 11, 1)
        np.testing.assert_array_equal(got, want, err_msg="qlen=%d" % qlen)


@pytest.mark.parametrize("kind", ["auto", "i32", "i16x2", "lazyf16q"])
def test_long_queries_many_chunks(sw, kind):
    """Queries of 12,000 and 20,000 residues (10 to 33 chunk launches,
    depending on the lane type) against a ragged database that also holds a
    3000-residue slice of each query: high scores carried across every chunk
    boundary, near the packed lanes' ceiling (flagged and rescored there)."""
    rng = np.random.default_rng(1010)
    M = synth.protein_matrix(rng)
    for qlen in (12_000, 20_000):
        q = synth.residues(rng, qlen, 20)
        lens = np.concatenate([[0, 1], rng.integers(1, 800, 40)]).astype(np.int64)
        seqs = [synth.residues(rng, int(x), 20) for x in lens]
        start = int(rng.integers(0, qlen - 3000))
        seqs.append(np.concatenate([synth.residues(rng, 50, 20), q[start:start + 3000],
                                    synth.residues(rng, 50, 20)]))
        db, off = pack_list(seqs)
        db_d, off_d = db_to_dev(db, off)
        want = oracle.gotoh_batch(q, db, off, M, 11, 1)
        assert want[-1] > 15_000  # the planted slice
        got = run(sw, kind, q, M, db_d, off_d, 11, 1)
        np.testing.assert_array_equal(got, want, err_msg="qlen=%d" % qlen)


def _piece_geometry(m, maxM, e):
    """Pieces of a long sequence for a single-chunk query of length m: the
    widest span of a positive-scoring local alignment, the piece length and
    the stride between piece starts (the library's rule)."""
    span = m + (m * maxM - 1) // e
    plen = max(2 * span, 2048)
    return span, plen, plen - span + 1


@pytest.mark.parametrize("kind", LANES)
def test_long_sequences_split_into_pieces(sw, kind):
    """Short queries against sequences several pieces long: copies of the
    query planted across piece boundaries (straddling the overlap, at its
    edges and inside), with and without a horizontal gap, in protein and DNA
    scoring; beside them ordinary short sequences, empty ones, and long ones
    with nothing planted.  Scores equal the oracle's on every lane type."""
    rng = np.random.default_rng(1011)
    for M, o, e, A, m in ((synth.protein_matrix(rng), 11, 1, 20, 60), (synth.dna_matrix(), 6, 1, 4, 150)):
        span, plen, stride = _piece_geometry(m, int(M.max()), e)
        q = synth.residues(rng, m, A)
        seqs = [synth.residues(rng, int(x), A) for x in rng.integers(0, 400, 30)] + [np.zeros(0, np.uint8)]
        for k, shift in enumerate((-m // 2, 0, span - m - 1, stride - 1, -1, plen - stride)):
            L = plen * 3 + 500 + 37 * k
            ref = synth.residues(rng, L, A)
            at = (k % 2 + 1) * stride + shift  # near the start of the second or third piece
            at = min(max(at, 0), L - m - 40)
            ref[at:at + m] = q
            if k % 3 == 2:  # a horizontal gap of 25 inside the copy
                ref = np.concatenate([ref[:at + m // 2], synth.residues(rng, 25, A), ref[at + m // 2:]])
            seqs.append(ref)
        seqs.append(synth.residues(rng, plen * 4 + 11, A))  # long, nothing planted
        db, off = pack_list(seqs)
        db_d, off_d = db_to_dev(db, off)
        want = oracle.gotoh_batch(q, db, off, M, o, e)
        assert (want[-7:-1] >= m // 2).all()  # the planted copies score
        got = run(sw, kind, q, M, db_d, off_d, o, e)
        np.testing.assert_array_equal(got, want, err_msg="A=%d m=%d" % (A, m))


@pytest.mark.parametrize("kind", ["auto", "i32", "i16x2", "lazyf16q"])
def test_piece_slots_run_out(sw, kind):
    """More pieces than slots (at most one per database sequence): a few long
    sequences with a planted copy each, among fewer short ones, so that some
    long sequences must stay whole.  Every score equals the oracle's, split
    or not."""
    rng = np.random.default_rng(1012)
    M, o, e, m = synth.protein_matrix(rng), 11, 1, 60
    span, plen, stride = _piece_geometry(m, int(M.max()), e)
    q = synth.residues(rng, m, 20)
    seqs = []
    for k in range(4):  # 4 long sequences of 3-4 pieces each, 2 short ones: 6 slots
        ref = synth.residues(rng, plen + stride * (2 + k % 2) + 17 * k, 20)
        at = stride * (1 + k % 2) - m // 3
        ref[at:at + m] = q
        seqs.append(ref)
    seqs += [synth.residues(rng, 90, 20), synth.residues(rng, 5, 20)]
    db, off = pack_list(seqs)
    db_d, off_d = db_to_dev(db, off)
    want = oracle.gotoh_batch(q, db, off, M, o, e)
    assert (want[:4] >= 4 * m).all()
    got = run(sw, kind, q, M, db_d, off_d, o, e)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("kind", LANES)
def test_gap_adversary_dna(sw, kind):
    """Long query-side insertions (vertical gaps through many segments) with
    DNA scoring; each query is aligned against every reference."""
    rng = np.random.default_rng(1002)
    M = synth.dna_matrix()
    queries, refs = gap_adversary(rng, 4, 40)
    db, off = pack_list(refs)
    db_d, off_d = db_to_dev(db, off)
    for q in queries[:6]:
        want = oracle.gotoh_batch(q, db, off, M, 6, 1)
        got = run(sw, kind, q, M, db_d, off_d, 6, 1)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("kind", LANES)
def test_random_gap_costs(sw, kind):
    rng = np.random.default_rng(1003)
    M = synth.protein_matrix(rng)
    db, off = synth.random_db(rng, 200, 20, "uniform", lo=1, hi=300)
    db_d, off_d = db_to_dev(db, off)
    for o, e in ((1, 0), (1, 1), (3, 3), (5, 0), (7, 2), (11, 1), (12, 12), (20, 5)):
        q = synth.residues(rng, int(rng.integers(20, 600)), 20)
        want = oracle.gotoh_batch(q, db, off, M, o, e)
        got = run(sw, kind, q, M, db_d, off_d, o, e)
        np.testing.assert_array_equal(got, want, err_msg="o=%d e=%d" % (o, e))


@pytest.mark.parametrize("kind", ["i32", "i16x2", "i16x2q", "auto", "lazyf16q"])
def test_both_corrected_passes(sw, kind):
    """The scan-F kernels take a shorter corrected pass when the smallest
    substitution score allows it (>= -(o+e) for int32 lanes, >= -o for
    s16x2 lanes) and the general pass otherwise: mismatch scores on both
    sides of both boundaries, several e, query-side insertions across many
    segments and multi-chunk queries."""
    rng = np.random.default_rng(1010)
    queries, refs = gap_adversary(rng, 4, 24, ylo=60, yhi=400)
    refs += [synth.residues(rng, int(n), 4) for n in (1, 5, 300, 2500)]
    db, off = pack_list(refs)
    db_d, off_d = db_to_dev(db, off)
    queries = queries[:4] + [synth.residues(rng, n, 4) for n in (70, 700, 2100)]
    for o in (3, 5):
        for e in (0, 1, o):
            for mm in sorted({-(o + e + 1), -(o + e), -(o + 1), -o, -o + 1}):
                M = synth.dna_matrix(match=2, mismatch=mm)
                for q in queries:
                    want = oracle.gotoh_batch(q, db, off, M, o, e)
                    got = run(sw, kind, q, M, db_d, off_d, o, e)
                    np.testing.assert_array_equal(got, want, err_msg="o=%d e=%d mismatch=%d m=%d"
                                                  % (o, e, mm, len(q)))


AC_LAYOUTS = [(16, 8), (16, 32), (32, 8), (32, 16), (32, 24), (32, 32), (32, 40), (64, 8), (64, 16), (64, 24),
              (64, 28), (64, 32), (64, 40)]


@pytest.mark.parametrize("layout", AC_LAYOUTS)
def test_always_corrected_pass(sw, layout):
    """The split layouts that run the always-corrected pass (every column
    corrected, the zero floor of H taken on the diagonal instead of h):
    DNA scoring, where most h are below zero and the floor decides the
    diagonal; mismatch scores at the pass's condition (-o, -o + 1); e = 0,
    1 and o; one-chunk and multi-chunk queries, with query-side insertions
    that carry F across many lanes and a copy of the query's middle planted
    across chunk boundaries."""
    L, S = layout
    rng = np.random.default_rng(1012 + L * 100 + S)
    QC = L * S
    queries, refs = gap_adversary(rng, 4, 12, ylo=40, yhi=300)
    q_long = synth.residues(rng, 3 * QC + 17, 4)
    refs += [synth.residues(rng, int(n), 4) for n in (1, 2, 90, 1500)]
    refs.append(np.concatenate([synth.residues(rng, 50, 4), q_long[QC - 40: 2 * QC + 40],
                                synth.residues(rng, 30, 4)]))
    db, off = pack_list(refs)
    db_d, off_d = db_to_dev(db, off)
    out = torch.empty(len(refs), dtype=torch.int32, device="cuda")
    qs = queries[:3] + [synth.residues(rng, QC, 4), synth.residues(rng, QC + 1, 4), q_long]
    # the last case (mismatch below -o) runs the general pass on the same layout
    for o, e, mm in ((6, 1, -4), (5, 0, -5), (4, 4, -3), (3, 1, -3), (7, 2, -1), (3, 1, -4)):
        M = synth.dna_matrix(match=2 if mm > -4 else 1, mismatch=mm)
        for q in qs:
            want = oracle.gotoh_batch(q, db, off, M, o, e)
            prof = sw.Profile(q, M, sw.SW_LANE_I16X2Q, lanes=L, seg_len=S)
            out.fill_(-7)
            sw.sw_align_batch(prof, db_d, off_d, o, e, out)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy(), want, err_msg="L=%d S=%d o=%d e=%d mm=%d m=%d"
                                          % (L, S, o, e, mm, len(q)))
            prof.free()


@pytest.mark.parametrize("kind", LANES)
def test_unknown_database_residues(sw, kind):
    """Database codes >= A score the smallest matrix entry on every lane
    type (the oracle's convention): DNA and protein matrices, both sides of
    the shorter corrected pass's condition, one- and multi-chunk queries."""
    rng = np.random.default_rng(1011)
    for M, o, e in ((synth.dna_matrix(match=2, mismatch=-3), 5, 1),
                    (synth.dna_matrix(match=2, mismatch=-3), 2, 1),
                    (synth.protein_matrix(rng), 11, 1)):
        A = M.shape[0]
        lens = np.concatenate([[1, 3], rng.integers(20, 900, 60)]).astype(np.int64)
        db, off = synth.pack(lens, rng, A)
        hit = rng.random(len(db)) < 0.08
        db[hit] = rng.choice(np.array([A, A + 1, 255], np.uint8), int(hit.sum()))
        db_d, off_d = db_to_dev(db, off)
        for qlen in (150, 700, 2300):
            q = synth.residues(rng, qlen, A)
            want = oracle.gotoh_batch(q, db, off, M, o, e)
            got = run(sw, kind, q, M, db_d, off_d, o, e)
            np.testing.assert_array_equal(got, want, err_msg="A=%d o=%d m=%d" % (A, o, qlen))


@pytest.mark.parametrize("kind", LANES)
def test_overflow_boundaries_rescored_exactly(sw, kind):
    """Identical DNA stretches whose true score sits just below, at and above
    the s8 (127) and s16 (32767) ceilings: packed lanes must flag them and
    the int32 rescore must return the exact value."""
    rng = np.random.default_rng(1004)
    M = synth.dna_matrix()
    base = synth.residues(rng, 33000, 4)
    q = base[:600]
    seqs = [base[:k] for k in (120, 121, 126, 127, 128, 129, 140, 300, 600)]
    seqs += [synth.residues(rng, 50, 4)]
    db, off = pack_list(seqs)
    db_d, off_d = db_to_dev(db, off)
    want = oracle.gotoh_batch(q, db, off, M, 6, 1)
    assert want[3] == 127 and want[4] == 128
    got = run(sw, kind, q, M, db_d, off_d, 6, 1)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("kind", ["i16x2", "i16x2q", "auto"])
def test_int16_ceiling(sw, kind):
    """True scores around 32767 - max(M) and above 32767 (identical
    sequences with a +11 diagonal) are rescored exactly."""
    M = np.full((20, 20), -4, np.int8)
    np.fill_diagonal(M, 11)
    rng = np.random.default_rng(1005)
    q = synth.residues(rng, 3100, 20)
    seqs = [q[:k] for k in (2975, 2977, 2978, 2979, 3000, 3100)]
    db, off = pack_list(seqs)
    db_d, off_d = db_to_dev(db, off)
    want = oracle.gotoh_batch(q, db, off, M, 11, 1)
    assert want.max() > 32767
    got = run(sw, kind, q, M, db_d, off_d, 11, 1)
    np.testing.assert_array_equal(got, want)


def test_int16_ceiling_end_cells(sw):
    """Alignments whose score leaves the s16x2 range are flagged and their
    end cells recomputed exactly with int32 lanes (split layout, AUTO)."""
    M = np.full((20, 20), -4, np.int8)
    np.fill_diagonal(M, 11)
    rng = np.random.default_rng(1006)
    q = synth.residues(rng, 3100, 20)
    seqs = [q[:k] for k in (2975, 2979, 3000, 3100)] + [synth.residues(rng, 500, 20)]
    seqs.append(np.concatenate([synth.residues(rng, 40, 20), q[:3050]]))
    db, off = pack_list(seqs)
    db_d, off_d = db_to_dev(db, off)
    ws, wq, wr = oracle.gotoh_end_batch(q, db, off, M, 11, 1)
    assert ws.max() > 32767
    gs, gq, gr = _ends(sw, q, M, sw.SW_LANE_AUTO, db_d, off_d, len(seqs), 11, 1)
    np.testing.assert_array_equal(gs, ws)
    np.testing.assert_array_equal(gr, wr)
    np.testing.assert_array_equal(gq, wq)


def test_empty_inputs(sw):
    rng = np.random.default_rng(1006)
    M = synth.protein_matrix(rng)
    db, off = synth.random_db(rng, 10, 20, "uniform", lo=0, hi=40)
    db_d, off_d = db_to_dev(db, off)
    got = run(sw, "i32", np.zeros(0, np.uint8), M, db_d, off_d, 11, 1)
    assert (got == 0).all()
    prof = sw.Profile(synth.residues(rng, 50, 20), M)
    empty_off = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    sw.sw_align_batch(prof, db_d, empty_off, 11, 1, out)
    torch.cuda.synchronize()


def test_gap_cost_errors(sw):
    rng = np.random.default_rng(1007)
    M = synth.protein_matrix(rng)
    db, off = synth.random_db(rng, 4, 20, "uniform", lo=5, hi=9)
    db_d, off_d = db_to_dev(db, off)
    prof = sw.Profile(synth.residues(rng, 50, 20), M)
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    for o, e in ((0, 0), (5, 6), (3, -1)):
        with pytest.raises(sw.SwError) as ei:
            sw.sw_align_batch(prof, db_d, off_d, o, e, out)
        assert ei.value.code == sw.SW_ERR_INVALID


def test_stream_sync_and_scores_independent_of_stream(sw):
    rng = np.random.default_rng(1008)
    M = synth.protein_matrix(rng)
    db, off = synth.random_db(rng, 300, 20, "uniform", lo=10, hi=400)
    db_d, off_d = db_to_dev(db, off)
    q = synth.residues(rng, 300, 20)
    s = torch.cuda.Stream()
    prof = sw.Profile(q, M, sw.SW_LANE_AUTO, stream=s)
    out = torch.zeros(300, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(s):
        sw.sw_align_batch(prof, db_d, off_d, 11, 1, out, stream=s)
    sw.sw_stream_sync(s, 30_000)
    want = oracle.gotoh_batch(q, db, off, M, 11, 1)
    np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_cell_rate_probe_runs(sw):
    for lane in (sw.SW_LANE_I32, sw.SW_LANE_I16X2, sw.SW_LANE_I8X4):
        r = sw.sw_probe_cell_rate(lane, 256)
        assert r > 1e9
    # the corrected pass does more per cell than the plain one
    for lane in (sw.SW_LANE_I32, sw.SW_LANE_I16X2):
        plain = sw.sw_probe_cell_rate_pass(lane, 0, 1024)
        corr = sw.sw_probe_cell_rate_pass(lane, 1, 1024)
        assert 1e9 < corr < plain
    # the always-corrected pass (s16x2 only) also does more than the plain one
    ac = sw.sw_probe_cell_rate_pass(sw.SW_LANE_I16X2Q, 2, 1024)
    assert 1e9 < ac < sw.sw_probe_cell_rate_pass(sw.SW_LANE_I16X2, 0, 1024)


# ---------------------------------------------------------------------------
# sw_align_pairs: each pair with its own query
# ---------------------------------------------------------------------------

PAIR_LANES = ["i32", "i16x2", "i16x2q", "i8x4", "auto"]


def run_pairs(sw, kind, q, q_off, r, r_off, M, o, e):
    lane = {"i32": sw.SW_LANE_I32, "i16x2": sw.SW_LANE_I16X2, "i16x2q": sw.SW_LANE_I16X2Q,
            "i8x4": sw.SW_LANE_I8X4, "auto": sw.SW_LANE_AUTO}[kind]
    qd, qo = db_to_dev(q, q_off)
    rd, ro = db_to_dev(r, r_off)
    n = len(q_off) - 1
    out = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    sw.sw_align_pairs(qd, qo, rd, ro, M, o, e, out, lane_type=lane)
    torch.cuda.synchronize()
    return out[:n].cpu().numpy()


@pytest.mark.parametrize("kind", PAIR_LANES)
def test_pairs_reads_vs_windows(sw, kind):
    """DNA reads (95%/99% copies, 40-200 bp indels) against their own 2 kbp
    windows, match +1 mismatch -4, o=6 e=1."""
    w = synth.workload_reads(n_pairs=1500)
    want = oracle.gotoh_pairs(w["q"], w["q_off"], w["r"], w["r_off"], w["M"], w["o"], w["e"])
    got = run_pairs(sw, kind, w["q"], w["q_off"], w["r"], w["r_off"], w["M"], w["o"], w["e"])
    np.testing.assert_array_equal(got, want)
    assert want.max() > 127  # the 8-bit lanes must have overflowed and been rescored


@pytest.mark.parametrize("kind", PAIR_LANES)
def test_pairs_mixed_query_lengths(sw, kind):
    """Query lengths 0..512 across every class, ragged references (some
    empty), protein scoring."""
    rng = np.random.default_rng(1101)
    M = synth.protein_matrix(rng)
    qlens = np.concatenate([[0, 1, 2, 512, 511, 160, 161, 128, 129, 256, 257],
                            rng.integers(0, 513, 300)]).astype(np.int64)
    rlens = rng.integers(0, 700, len(qlens)).astype(np.int64)
    rlens[:3] = 0
    q, q_off = synth.pack(qlens, rng, 20)
    r, r_off = synth.pack(rlens, rng, 20)
    want = oracle.gotoh_pairs(q, q_off, r, r_off, M, 11, 1)
    got = run_pairs(sw, kind, q, q_off, r, r_off, M, 11, 1)
    np.testing.assert_array_equal(got, want)


def test_pairs_query_too_long(sw):
    rng = np.random.default_rng(1102)
    M = synth.dna_matrix()
    q, q_off = synth.pack(np.array([100, 600], np.int64), rng, 4)
    r, r_off = synth.pack(np.array([200, 200], np.int64), rng, 4)
    with pytest.raises(sw.SwError) as ei:
        run_pairs(sw, "auto", q, q_off, r, r_off, M, 6, 1)
    assert ei.value.code == sw.SW_ERR_RANGE


@pytest.mark.parametrize("kind", PAIR_LANES)
def test_pairs_gap_adversary(sw, kind):
    rng = np.random.default_rng(1103)
    M = synth.dna_matrix()
    queries, refs = gap_adversary(rng, 4, 400, xlo=20, xhi=120, ylo=40, yhi=200)
    queries = [x[:512] for x in queries]
    q, q_off = pack_list(queries)
    r, r_off = pack_list(refs)
    want = oracle.gotoh_pairs(q, q_off, r, r_off, M, 6, 1)
    got = run_pairs(sw, kind, q, q_off, r, r_off, M, 6, 1)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("kind", ["i32", "i16x2", "i16x2q"])
def test_pairs_both_corrected_passes(sw, kind):
    """Pairs with mismatch scores on both sides of the shorter corrected
    pass's conditions (>= -(o+e) int32, >= -o s16x2)."""
    rng = np.random.default_rng(1104)
    queries, refs = gap_adversary(rng, 4, 120, xlo=20, xhi=120, ylo=40, yhi=300)
    queries = [x[:512] for x in queries]
    q, q_off = pack_list(queries)
    r, r_off = pack_list(refs)
    o = 4
    for e in (0, 1, 4):
        for mm in sorted({-(o + e + 1), -(o + e), -(o + 1), -o, -o + 1}):
            M = synth.dna_matrix(match=2, mismatch=mm)
            want = oracle.gotoh_pairs(q, q_off, r, r_off, M, o, e)
            got = run_pairs(sw, kind, q, q_off, r, r_off, M, o, e)
            np.testing.assert_array_equal(got, want, err_msg="e=%d mismatch=%d" % (e, mm))


@pytest.mark.parametrize("kind", PAIR_LANES)
def test_pairs_unknown_residues(sw, kind):
    """Codes >= A in the reads and in the windows score the smallest matrix
    entry, as in the oracle."""
    rng = np.random.default_rng(1105)
    M = synth.dna_matrix(match=2, mismatch=-3)
    qlens = rng.integers(1, 400, 300).astype(np.int64)
    rlens = rng.integers(1, 900, 300).astype(np.int64)
    q, q_off = synth.pack(qlens, rng, 4)
    r, r_off = synth.pack(rlens, rng, 4)
    for s in (q, r):
        hit = rng.random(len(s)) < 0.05
        s[hit] = rng.choice(np.array([4, 5, 255], np.uint8), int(hit.sum()))
    for o, e in ((5, 1), (2, 2)):
        want = oracle.gotoh_pairs(q, q_off, r, r_off, M, o, e)
        got = run_pairs(sw, kind, q, q_off, r, r_off, M, o, e)
        np.testing.assert_array_equal(got, want, err_msg="o=%d e=%d" % (o, e))


@pytest.mark.parametrize("kind", ["auto", "i16x2q", "i32", "i16x2"])
def test_pairs_end_cells(sw, kind):
    """sw_align_pairs_ends: scores and end cells of every pair equal the
    oracle's (first cell in column order), reads vs windows with planted
    copies, ties from a +1/-1 matrix, and a +100 diagonal whose scores leave
    the s16x2 range (flagged pairs rescored with int32 end cells)."""
    lane = {"auto": sw.SW_LANE_AUTO, "i16x2q": sw.SW_LANE_I16X2Q, "i32": sw.SW_LANE_I32,
            "i16x2": sw.SW_LANE_I16X2}[kind]
    rng = np.random.default_rng(1106)
    w = synth.workload_reads(n_pairs=300)
    cases = [(w["q"], w["q_off"], w["r"], w["r_off"], w["M"], w["o"], w["e"])]
    qlens = rng.integers(1, 513, 200).astype(np.int64)
    rlens = rng.integers(1, 700, 200).astype(np.int64)
    q, q_off = synth.pack(qlens, rng, 4)
    r, r_off = synth.pack(rlens, rng, 4)
    cases.append((q, q_off, r, r_off, synth.dna_matrix(match=1, mismatch=-1), 2, 1))
    big = np.full((4, 4), -20, np.int8)
    np.fill_diagonal(big, 100)
    qs = [synth.residues(rng, int(n), 4) for n in (400, 500, 512)]
    rs = [np.concatenate([synth.residues(rng, 30, 4), x, synth.residues(rng, 30, 4)]) for x in qs]
    qb, qbo = pack_list(qs)
    rb, rbo = pack_list(rs)
    cases.append((qb, qbo, rb, rbo, big, 20, 2))
    for (q, q_off, r, r_off, M, o, e) in cases:
        n = len(q_off) - 1
        ws, wq, wr = oracle.gotoh_end_pairs(q, q_off, r, r_off, M, o, e)
        qd, qo = db_to_dev(q, q_off)
        rd, ro = db_to_dev(r, r_off)
        sc = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        qe = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        re_ = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        sw.sw_align_pairs_ends(qd, qo, rd, ro, M, o, e, sc, qe, re_, lane_type=lane)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(sc.cpu().numpy(), ws)
        np.testing.assert_array_equal(re_.cpu().numpy(), wr)
        np.testing.assert_array_equal(qe.cpu().numpy(), wq)
    assert ws.max() > 32767


def test_lazyf_pairs_on_the_split_layout(sw):
    """Lazy-F on the split s16x2 pair kernel equals the oracle (reads vs
    windows, the gap adversary, both corrected-pass conditions) and counts
    its correction steps."""
    rng = np.random.default_rng(1107)
    w = synth.workload_reads(n_pairs=400)
    queries, refs = gap_adversary(rng, 4, 100, xlo=20, xhi=120, ylo=40, yhi=200)
    qa, qao = pack_list([x[:512] for x in queries])
    ra, rao = pack_list(refs)
    for (q, q_off, r, r_off, M, o, e) in ((w["q"], w["q_off"], w["r"], w["r_off"], w["M"], w["o"], w["e"]),
                                          (qa, qao, ra, rao, synth.dna_matrix(), 6, 1),
                                          (qa, qao, ra, rao, synth.dna_matrix(match=2, mismatch=-5), 3, 1)):
        want = oracle.gotoh_pairs(q, q_off, r, r_off, M, o, e)
        qd, qo = db_to_dev(q, q_off)
        rd, ro = db_to_dev(r, r_off)
        out = torch.full((len(q_off) - 1,), -7, dtype=torch.int32, device="cuda")
        steps = torch.zeros(1, dtype=torch.int64, device="cuda")
        sw.sw_align_lazyf_pairs(qd, qo, rd, ro, M, o, e, out, lazy_steps=steps, lane_type=sw.SW_LANE_I16X2Q)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        assert steps.item() > 0


def test_lazyf_pairs_exact_and_counts_steps(sw):
    """Lazy-F pairs equal the oracle; its correction loop (the corrective
    factor C of Sec. I) runs far more on related read/window pairs (long
    high-scoring paths keep carried F alive) than on unrelated ones."""
    w = synth.workload_reads(n_pairs=1200)
    want = oracle.gotoh_pairs(w["q"], w["q_off"], w["r"], w["r_off"], w["M"], w["o"], w["e"])
    qd, qo = db_to_dev(w["q"], w["q_off"])
    rd, ro = db_to_dev(w["r"], w["r_off"])
    out = torch.empty(1200, dtype=torch.int32, device="cuda")
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    sw.sw_align_lazyf_pairs(qd, qo, rd, ro, w["M"], w["o"], w["e"], out, lazy_steps=steps)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    related = int(steps.item())
    # the same reads against the windows of other pairs (unrelated)
    r_off = w["r_off"]
    win = np.roll(w["r"].reshape(1200, -1), 1, axis=0).reshape(-1)
    rd2, _ = db_to_dev(win, r_off)
    steps.zero_()
    sw.sw_align_lazyf_pairs(qd, qo, rd2, ro, w["M"], w["o"], w["e"], out, lazy_steps=steps)
    torch.cuda.synchronize()
    unrelated = int(steps.item())
    assert related > 3 * unrelated


def _ends(sw, q, M, kind, db_d, off_d, n, o, e):
    prof = sw.Profile(q, M, kind)
    sc = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    qe = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    re_ = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    sw.sw_align_batch_ends(prof, db_d, off_d, o, e, sc, qe, re_)
    torch.cuda.synchronize()
    prof.free()
    return sc.cpu().numpy(), qe.cpu().numpy(), re_.cpu().numpy()


END_LANES = ["auto", "i32", "i16x2q", "i16x2"]


@pytest.mark.parametrize("lane", END_LANES)
def test_end_cells_with_ties(sw, lane):
    """Many cells reach the same maximum (DNA, +1/-1, cheap gaps, repeated
    copies): the reported end cell is the first in column order, then the
    smallest query position, as in the oracle; matrices on both sides of the
    shorter corrected pass's condition; one- and multi-chunk queries."""
    rng = np.random.default_rng(1203)
    kind = {"auto": sw.SW_LANE_AUTO, "i32": sw.SW_LANE_I32, "i16x2q": sw.SW_LANE_I16X2Q,
            "i16x2": sw.SW_LANE_I16X2}[lane]
    for M, o, e in ((synth.dna_matrix(match=1, mismatch=-1), 2, 1), (synth.dna_matrix(match=1, mismatch=-3), 2, 1)):
        for qlen in (30, 700, 2600):
            q = synth.residues(rng, qlen, 4)
            refs = [synth.residues(rng, int(n), 4) for n in rng.integers(1, 400, 40)]
            refs += [np.concatenate([q[:50], synth.residues(rng, 30, 4), q[:50]]) for _ in range(5)]
            refs += [np.concatenate([synth.residues(rng, 20, 4), q[qlen // 2:qlen // 2 + 60]] * 3) for _ in range(5)]
            db, off = pack_list(refs)
            db_d, off_d = db_to_dev(db, off)
            n = len(off) - 1
            ws, wq, wr = oracle.gotoh_end_batch(q, db, off, M, o, e)
            gs, gq, gr = _ends(sw, q, M, kind, db_d, off_d, n, o, e)
            msg = "min M %d m=%d" % (M.min(), qlen)
            np.testing.assert_array_equal(gs, ws, err_msg=msg)
            np.testing.assert_array_equal(gr, wr, err_msg=msg)
            np.testing.assert_array_equal(gq, wq, err_msg=msg)


@pytest.mark.parametrize("lane", ["auto", "i32"])
def test_end_cells_with_unknown_residues(sw, lane):
    """End cells when database codes >= A (unknown residues, scored as the
    smallest matrix entry) sit inside and around the best alignments."""
    rng = np.random.default_rng(1204)
    kind = {"auto": sw.SW_LANE_AUTO, "i32": sw.SW_LANE_I32}[lane]
    M = synth.dna_matrix(match=2, mismatch=-3)
    for qlen in (40, 900, 2600):
        q = synth.residues(rng, qlen, 4)
        refs = [np.concatenate([synth.residues(rng, int(rng.integers(0, 100)), 4), q[: min(qlen, 300)],
                                synth.residues(rng, 50, 4)]) for _ in range(30)]
        refs += [synth.residues(rng, int(n), 4) for n in rng.integers(1, 500, 30)]
        db, off = pack_list(refs)
        hit = rng.random(len(db)) < 0.05
        db[hit] = rng.choice(np.array([4, 7, 255], np.uint8), int(hit.sum()))
        db_d, off_d = db_to_dev(db, off)
        ws, wq, wr = oracle.gotoh_end_batch(q, db, off, M, 5, 1)
        gs, gq, gr = _ends(sw, q, M, kind, db_d, off_d, len(refs), 5, 1)
        np.testing.assert_array_equal(gs, ws)
        np.testing.assert_array_equal(gr, wr)
        np.testing.assert_array_equal(gq, wq)


@pytest.mark.parametrize("lane", END_LANES)
def test_end_cells_match_oracle(sw, lane):
    """Scores and end cells of every alignment equal the oracle's (first
    cell in column order), across single- and multi-chunk queries."""
    rng = np.random.default_rng(1201)
    M = synth.protein_matrix(rng)
    lens = np.concatenate([[0, 1, 3], rng.integers(1, 600, 150)])
    db, off = synth.pack(lens.astype(np.int64), rng, 20)
    db_d, off_d = db_to_dev(db, off)
    n = len(off) - 1
    kind = {"auto": sw.SW_LANE_AUTO, "i32": sw.SW_LANE_I32, "i16x2q": sw.SW_LANE_I16X2Q,
            "i16x2": sw.SW_LANE_I16X2}[lane]
    for qlen in (1, 40, 300, 700, 1500, 3000, 5200):
        q = synth.residues(rng, qlen, 20)
        ws, wq, wr = oracle.gotoh_end_batch(q, db, off, M, 11, 1)
        prof = sw.Profile(q, M, kind)
        sc = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        qe = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        re_ = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        sw.sw_align_batch_ends(prof, db_d, off_d, 11, 1, sc, qe, re_)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(sc.cpu().numpy(), ws, err_msg="qlen=%d" % qlen)
        np.testing.assert_array_equal(re_.cpu().numpy(), wr, err_msg="qlen=%d" % qlen)
        np.testing.assert_array_equal(qe.cpu().numpy(), wq, err_msg="qlen=%d" % qlen)
        prof.free()


def test_end_cells_of_planted_local_matches(sw):
    """Reads planted inside random references: the end cell is where the
    planted copy ends (DNA scoring, high identity)."""
    rng = np.random.default_rng(1202)
    M = synth.dna_matrix()
    q = synth.residues(rng, 120, 4)
    refs, ends = [], []
    for k in range(50):
        pre = int(rng.integers(0, 300))
        refs.append(np.concatenate([synth.residues(rng, pre, 4), q, synth.residues(rng, 200, 4)]))
        ends.append(pre + 120)
    db, off = pack_list(refs)
    db_d, off_d = db_to_dev(db, off)
    prof = sw.Profile(q, M)
    sc = torch.empty(50, dtype=torch.int32, device="cuda")
    qe = torch.empty(50, dtype=torch.int32, device="cuda")
    re_ = torch.empty(50, dtype=torch.int32, device="cuda")
    sw.sw_align_batch_ends(prof, db_d, off_d, 6, 1, sc, qe, re_)
    torch.cuda.synchronize()
    assert (sc.cpu().numpy() == 120).all()
    assert (qe.cpu().numpy() == 120).all()
    np.testing.assert_array_equal(re_.cpu().numpy(), np.array(ends))
