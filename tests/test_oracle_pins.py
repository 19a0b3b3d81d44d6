"""Pins of the CPU oracle against facts fixed by the paper and by the
mathematics, not by the oracle itself.

 - brute-force enumeration of every local alignment on tiny inputs, with
   asymmetric random matrices (catches a dropped term, a wrong sign or index
   and a transposed operand in the recurrence)
 - hand-derived golden cases (tests/golden/hand_cases.ini)
 - closed forms: identical sequences, one-residue query, gap open so large
   that only ungapped diagonals remain (max-sum segment per diagonal),
   all-mismatch, empty inputs
 - invariants: score >= 0, symmetry for symmetric matrices, transpose rule
   for asymmetric ones
 - the striped CPU variants of Alg. 1 (lazy-F) and Alg. 6 (scan) equal the
   scalar recurrence for every lane count p (the transformations of Sec. II
   are claimed to be equivalences)
"""
import numpy as np
import pytest

import oracle
from paper_1909_00899_gb300 import synth

from golden_cases import load as load_golden


def _rand_case(rng, A, mmax, nmax, lo=-6, hi=6):
    M = rng.integers(lo, hi + 1, size=(A, A)).astype(np.int8)
    m = int(rng.integers(0, mmax + 1))
    n = int(rng.integers(0, nmax + 1))
    return M, rng.integers(0, A, m).astype(np.uint8), rng.integers(0, A, n).astype(np.uint8)


@pytest.mark.parametrize("A", [2, 4, 20])
def test_gotoh_equals_brute_force(A):
    rng = np.random.default_rng([7, A])
    cases = 3000 if A != 20 else 2000
    for _ in range(cases):
        M, q, r = _rand_case(rng, A, 6, 6)
        o = int(rng.integers(1, 13))
        e = int(rng.integers(0, o + 1))
        assert oracle.gotoh(q, r, M, o, e) == oracle.brute(q, r, M, o, e), (q, r, M, o, e)


def test_gotoh_equals_brute_force_length7():
    rng = np.random.default_rng(77)
    for _ in range(300):
        A = int(rng.choice([2, 4, 20]))
        M = rng.integers(-5, 6, size=(A, A)).astype(np.int8)
        q = rng.integers(0, A, 7).astype(np.uint8)
        r = rng.integers(0, A, 7).astype(np.uint8)
        o = int(rng.integers(1, 13))
        e = int(rng.integers(0, o + 1))
        assert oracle.gotoh(q, r, M, o, e) == oracle.brute(q, r, M, o, e)


def test_gotoh_config_matrices_brute_force():
    rng = np.random.default_rng(79)
    Mp = synth.protein_matrix(rng)
    Md = synth.dna_matrix()
    for _ in range(800):
        for M, A, o, e in ((Mp, 20, 11, 1), (Md, 4, 6, 1)):
            q = rng.integers(0, A, int(rng.integers(1, 8))).astype(np.uint8)
            r = rng.integers(0, A, int(rng.integers(1, 8))).astype(np.uint8)
            assert oracle.gotoh(q, r, M, o, e) == oracle.brute(q, r, M, o, e)


@pytest.mark.parametrize("case", load_golden(), ids=lambda c: c["name"])
def test_golden_hand_cases(case):
    got = oracle.gotoh(case["q"], case["r"], case["M"], case["o"], case["e"])
    assert got == case["score"], case["cite"]
    # every lane count of both striped variants reaches the same value
    for p in (1, 2, 3, 4, 8, 16, 32):
        assert oracle.striped_lazyf(case["q"], case["r"], case["M"], case["o"], case["e"], p) == case["score"]
        assert oracle.striped_scan(case["q"], case["r"], case["M"], case["o"], case["e"], p) == case["score"]
    if len(case["q"]) <= 9 and len(case["r"]) <= 9:
        assert oracle.brute(case["q"], case["r"], case["M"], case["o"], case["e"]) == case["score"]


def test_identical_sequences_score_diagonal_sum():
    """With every off-diagonal entry below every diagonal entry (the seeded
    protein matrix: off <= 3 < 4 <= diag), M[x][y] <= (M[x][x]+M[y][y])/2, so
    no alignment of a sequence against itself beats the full diagonal."""
    rng = np.random.default_rng(80)
    for k in range(20):
        M = synth.protein_matrix(rng)
        q = synth.residues(rng, int(rng.integers(1, 400)), 20)
        assert oracle.gotoh(q, q, M, 11, 1) == int(M[q, q].sum())
    Md = synth.dna_matrix()
    read = synth.residues(rng, 150, 4)
    assert oracle.gotoh(read, read, Md, 6, 1) == 150


def test_one_residue_query():
    rng = np.random.default_rng(81)
    for _ in range(200):
        A = int(rng.choice([4, 20]))
        M = rng.integers(-8, 9, size=(A, A)).astype(np.int8)
        q = rng.integers(0, A, 1).astype(np.uint8)
        r = rng.integers(0, A, int(rng.integers(1, 50))).astype(np.uint8)
        expect = max(0, int(M[q[0], r].max()))
        assert oracle.gotoh(q, r, M, int(rng.integers(1, 12)), 1) == expect


def _kadane_diagonals(q, r, M):
    best = 0
    m, n = len(q), len(r)
    for d in range(-(m - 1), n):
        run = 0
        for i in range(m):
            j = i + d
            if 0 <= j < n:
                run = max(0, run + int(M[q[i], r[j]]))
                best = max(best, run)
    return best


def test_huge_gap_open_reduces_to_diagonal_max_segments():
    rng = np.random.default_rng(82)
    for _ in range(200):
        A = int(rng.choice([4, 20]))
        M = rng.integers(-6, 7, size=(A, A)).astype(np.int8)
        q = rng.integers(0, A, int(rng.integers(1, 40))).astype(np.uint8)
        r = rng.integers(0, A, int(rng.integers(1, 40))).astype(np.uint8)
        assert oracle.gotoh(q, r, M, 1_000_000, 1) == _kadane_diagonals(q, r, M)


def test_all_mismatch_is_zero_and_empty_inputs():
    Md = synth.dna_matrix()
    q = np.zeros(30, np.uint8)
    r = np.full(40, 2, np.uint8)
    assert oracle.gotoh(q, r, Md, 6, 1) == 0
    assert oracle.gotoh(q[:0], r, Md, 6, 1) == 0
    assert oracle.gotoh(q, r[:0], Md, 6, 1) == 0
    assert oracle.striped_scan(q[:0], r, Md, 6, 1, 4) == 0
    assert oracle.striped_lazyf(q, r[:0], Md, 6, 1, 4) == 0


def test_nonnegative_symmetry_and_transpose():
    rng = np.random.default_rng(83)
    for _ in range(300):
        A = int(rng.choice([4, 20]))
        Ms = synth.protein_matrix(rng) if A == 20 else synth.dna_matrix()
        Ma = rng.integers(-6, 7, size=(A, A)).astype(np.int8)
        q = rng.integers(0, A, int(rng.integers(0, 60))).astype(np.uint8)
        r = rng.integers(0, A, int(rng.integers(0, 60))).astype(np.uint8)
        o = int(rng.integers(1, 13))
        e = int(rng.integers(0, o + 1))
        s = oracle.gotoh(q, r, Ms, o, e)
        assert s >= 0
        assert s == oracle.gotoh(r, q, Ms, o, e)
        assert oracle.gotoh(q, r, Ma, o, e) == oracle.gotoh(r, q, np.ascontiguousarray(Ma.T), o, e)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 8, 16, 32, 64])
def test_striped_variants_match_scalar(p):
    """Alg. 1 and Alg. 6 on the CPU equal the definition for every p,
    including gap-heavy inputs where carries cross many segments."""
    rng = np.random.default_rng([84, p])
    Mp = synth.protein_matrix(rng)
    Md = synth.dna_matrix()
    for t in range(60):
        if t % 2:
            M, A, o, e = Mp, 20, 11, 1
        else:
            M, A, o, e = Md, 4, 6, 1
        if t % 5 == 0:
            o = int(rng.integers(1, 13))
            e = int(rng.integers(0, o + 1))
        X = rng.integers(0, A, int(rng.integers(3, 50))).astype(np.uint8)
        Y = rng.integers(0, A, int(rng.integers(0, 90))).astype(np.uint8)
        Z = rng.integers(0, A, int(rng.integers(3, 50))).astype(np.uint8)
        if t % 3 == 0:
            q, r = np.concatenate([X, Y, Z]), np.concatenate([X, Z])
        elif t % 3 == 1:
            q, r = np.concatenate([X, Z]), np.concatenate([X, Y, Z])
        else:
            q, r = np.concatenate([X, Y]), np.concatenate([Z, Y, X])
        want = oracle.gotoh(q, r, M, o, e)
        assert oracle.striped_lazyf(q, r, M, o, e, p) == want
        assert oracle.striped_scan(q, r, M, o, e, p) == want


def test_lazyf_worst_case_needs_more_rounds():
    """A long query-only insertion makes the lazy-F loop run many steps
    (the corrective factor C of Sec. I grows with p)."""
    rng = np.random.default_rng(85)
    Md = synth.dna_matrix()
    X = synth.residues(rng, 60, 4)
    Y = synth.residues(rng, 150, 4)
    Z = synth.residues(rng, 60, 4)
    q = np.concatenate([X, Y, Z])
    r = np.concatenate([X, Z])
    _, steps_adv = oracle.striped_lazyf(q, r, Md, 6, 1, 16, return_steps=True)
    qr = synth.residues(rng, len(q), 4)
    _, steps_rand = oracle.striped_lazyf(qr, r, Md, 6, 1, 16, return_steps=True)
    assert steps_adv > steps_rand


def test_threaded_batch_and_pairs_equal_single_calls():
    rng = np.random.default_rng(86)
    M = synth.protein_matrix(rng)
    q = synth.residues(rng, 97, 20)
    db, off = synth.random_db(rng, 50, 20, "uniform", lo=0, hi=120)
    out = oracle.gotoh_batch(q, db, off, M, 11, 1, nthreads=4)
    for k in range(50):
        assert out[k] == oracle.gotoh(q, db[off[k]:off[k + 1]], M, 11, 1)
    qs, qoff = synth.random_db(rng, 50, 20, "uniform", lo=0, hi=80)
    outp = oracle.gotoh_pairs(qs, qoff, db, off, M, 11, 1, nthreads=3)
    for k in range(50):
        assert outp[k] == oracle.gotoh(qs[qoff[k]:qoff[k + 1]], db[off[k]:off[k + 1]], M, 11, 1)


@pytest.mark.parametrize("A", [2, 4, 20])
def test_end_cell_equals_brute_force(A):
    """The end cell (first in column order among cells whose H is the score)
    of the recurrence equals the end of the best enumerated alignment."""
    rng = np.random.default_rng([90, A])
    for _ in range(2000):
        M, q, r = _rand_case(rng, A, 6, 6)
        o = int(rng.integers(1, 13))
        e = int(rng.integers(0, o + 1))
        assert oracle.gotoh_end(q, r, M, o, e) == oracle.brute_end(q, r, M, o, e)


@pytest.mark.parametrize("case", [c for c in load_golden() if c["end"] is not None], ids=lambda c: c["name"])
def test_golden_end_cells(case):
    s, qe, re_ = oracle.gotoh_end(case["q"], case["r"], case["M"], case["o"], case["e"])
    assert s == case["score"] and (qe, re_) == case["end"], case["cite"]


def test_end_cell_of_a_prefix_match():
    """A query that is a prefix of the reference (identical residues, the
    seeded protein matrix): the alignment ends at the query's last residue,
    reference position m."""
    rng = np.random.default_rng(91)
    for _ in range(20):
        M = synth.protein_matrix(rng)
        q = synth.residues(rng, int(rng.integers(5, 80)), 20)
        r = np.concatenate([q, synth.residues(rng, int(rng.integers(0, 50)), 20)])
        s, qe, re_ = oracle.gotoh_end(q, r, M, 11, 1)
        assert s == int(M[q, q].sum()) and qe == len(q)
        assert re_ >= len(q)  # an equal score cannot end earlier than the full diagonal
        assert oracle.gotoh(q, r[:re_], M, 11, 1) == s
        assert oracle.gotoh(q, r[:re_ - 1], M, 11, 1) < s


def test_end_batch_matches_single():
    rng = np.random.default_rng(92)
    M = synth.protein_matrix(rng)
    q = synth.residues(rng, 70, 20)
    db, off = synth.random_db(rng, 40, 20, "uniform", lo=0, hi=90)
    s, qe, re_ = oracle.gotoh_end_batch(q, db, off, M, 11, 1, nthreads=3)
    for k in range(40):
        assert (s[k], qe[k], re_[k]) == oracle.gotoh_end(q, db[off[k]:off[k + 1]], M, 11, 1)


def _extend_alphabet(q, r, M):
    """Codes >= A mapped to one extra code A whose row and column hold the
    smallest entry of M: the unknown-residue convention as a plain
    (A+1)-letter problem, with no code outside the extended alphabet."""
    A = M.shape[0]
    Mx = np.full((A + 1, A + 1), M.min(), dtype=np.int8)
    Mx[:A, :A] = M
    return np.minimum(q, A).astype(np.uint8), np.minimum(r, A).astype(np.uint8), Mx


@pytest.mark.parametrize("seed", range(4))
def test_unknown_residues_score_the_smallest_entry(seed):
    """A code >= A on either side scores min(M) against anything: the same
    as an extra alphabet letter with that row and column (checked by the
    recurrence and, on tiny inputs, by enumeration), and identical in the
    striped variants."""
    rng = np.random.default_rng(600 + seed)
    M = synth.dna_matrix(match=2, mismatch=-3) if seed % 2 == 0 else synth.protein_matrix(rng)
    A = M.shape[0]
    unk = np.array([A, A + 1, 200, 255], dtype=np.uint8)
    for _ in range(30):
        q = synth.residues(rng, int(rng.integers(1, 40)), A)
        r = synth.residues(rng, int(rng.integers(1, 60)), A)
        for s in (q, r):
            k = rng.integers(0, len(s) // 3 + 1)
            s[rng.integers(0, len(s), k)] = rng.choice(unk, k)
        qx, rx, Mx = _extend_alphabet(q, r, M)
        for o, e in ((5, 1), (3, 3), (11, 1)):
            want = oracle.gotoh(qx, rx, Mx, o, e)
            assert oracle.gotoh(q, r, M, o, e) == want
            assert oracle.striped_scan(q, r, M, o, e, 4) == want
            assert oracle.striped_lazyf(q, r, M, o, e, 4) == want
            assert oracle.gotoh_end(q, r, M, o, e) == oracle.gotoh_end(qx, rx, Mx, o, e)
    for _ in range(40):
        q = rng.integers(0, A + 2, int(rng.integers(1, 7))).astype(np.uint8)
        r = rng.integers(0, A + 2, int(rng.integers(1, 7))).astype(np.uint8)
        qx, rx, Mx = _extend_alphabet(q, r, M)
        assert oracle.gotoh(q, r, M, 4, 1) == oracle.brute(qx, rx, Mx, 4, 1)


def test_unknown_residue_all_positive_matrix():
    """With a matrix of only positive entries an unknown residue still
    scores min(M) > 0 and extends the alignment (it is a residue, not a
    gap or a stop)."""
    M = np.array([[3, 1], [1, 2]], dtype=np.int8)
    q = np.array([0, 9, 1], dtype=np.uint8)
    r = np.array([0, 0, 1], dtype=np.uint8)
    assert oracle.gotoh(q, r, M, 5, 1) == 3 + 1 + 2


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_windows_overlapping_by_the_span_keep_the_score(seed):
    """The score of a query against a long sequence equals the maximum over
    windows of 2*span columns every span + 1 columns, where span = m +
    floor((m * max M - 1) / e) bounds the columns of any positive-scoring
    local alignment (the rule the batch plan splits long sequences by);
    windows overlapping by less can miss the optimum.  Copies of the query
    (some with a horizontal gap) are planted across window boundaries."""
    rng = np.random.default_rng([12, seed])
    A = 4 if seed % 2 else 20
    M = synth.dna_matrix() if A == 4 else synth.protein_matrix(rng)
    o, e = (6, 1 + seed % 3) if A == 4 else (11, 1 + seed % 3)
    m = int(rng.integers(6, 14))
    q = synth.residues(rng, m, A)
    span = m + (m * int(M.max()) - 1) // e
    plen, stride = 2 * span, span + 1
    refs = []
    for k in range(12):
        ref = synth.residues(rng, 6 * plen + int(rng.integers(0, 50)), A)
        at = int(rng.integers(1, 5)) * stride + int(rng.integers(-m, span - m))
        ref[at:at + m] = q
        if k % 3 == 0:
            gap = int(rng.integers(1, 6))
            ref = np.concatenate([ref[:at + m // 2], synth.residues(rng, gap, A), ref[at + m // 2:]])
        refs.append(ref)
    for ref in refs:
        whole = oracle.gotoh(q, ref, M, o, e)
        starts = list(range(0, max(1, len(ref) - plen + stride), stride))
        wins = [ref[s:s + plen] for s in starts]
        assert starts[-1] + plen >= len(ref)
        assert max(oracle.gotoh(q, w, M, o, e) for w in wins) == whole


def test_windows_without_overlap_miss_a_straddling_copy():
    """The converse check of the span rule: windows that do not overlap cut a
    copy of the query planted across their boundary, and their maximum falls
    below the sequence's score (so the overlap is what keeps it exact)."""
    rng = np.random.default_rng(1213)
    M = synth.dna_matrix()
    q = synth.residues(rng, 40, 4)
    ref = synth.residues(rng, 3000, 4)
    plen = 1000
    ref[plen - 20:plen + 20] = q
    whole = oracle.gotoh(q, ref, M, 6, 1)
    cut = max(oracle.gotoh(q, ref[s:s + plen], M, 6, 1) for s in range(0, len(ref), plen))
    assert whole == 40 and cut < whole


def test_gap_adversary_workload_is_what_it_claims():
    """The lazy-F worst-case workload: every query is X + Y + Z and its
    reference X + Z (|X|, |Z| >= 60, |Y| in 40..200), so the oracle's score is
    at least that of aligning X and Z across one vertical gap of |Y|
    (|X| + |Z| - o - (|Y| - 1) e) and at least the longer of X and Z alone."""
    w = synth.workload_gap_adversary(n_pairs=40)
    M, o, e = w["M"], w["o"], w["e"]
    q, qo, r, ro = w["q"], w["q_off"], w["r"], w["r_off"]
    for i in range(40):
        qi, ri = q[qo[i]:qo[i + 1]], r[ro[i]:ro[i + 1]]
        y = len(qi) - len(ri)
        assert 40 <= y <= 200
        pre = next((k for k in range(len(ri)) if qi[k] != ri[k]), len(ri))
        suf = next((k for k in range(len(ri)) if qi[len(qi) - 1 - k] != ri[len(ri) - 1 - k]), len(ri))
        assert pre >= 60 and suf >= 60  # X and Z are shared (at least)
        s = oracle.gotoh(qi, ri, M, o, e)
        assert s >= max(len(ri) - o - (y - 1) * e, pre, suf)  # an exact common run of k scores k
