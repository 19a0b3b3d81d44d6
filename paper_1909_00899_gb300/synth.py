"""Seeded synthetic inputs for the alignment workloads.

This module draws residues, lengths and substitution matrices; it holds none
of the alignment arithmetic.  Both the oracle-side checks and the CUDA path
consume what it returns, so it stays free of anything either side computes.

Workloads (all seeded; residue codes 0..A-1, uint8):
  protein_matrix   symmetric 20x20, diagonal U{4..11}, off-diagonal U{-4..3}
  dna_matrix       4x4, match +1, mismatch -4
  random_db        n sequences, lengths uniform or log-normal, iid residues
  read_windows     DNA reads vs their own reference windows, with mutated
                   copies and long indels (the mate-rescue stand-in)
"""
import numpy as np

BASE_SEED = 1909_00899
PROTEIN_A = 20
DNA_A = 4


def rng_for(config_index: int, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng([BASE_SEED + config_index, salt])


def protein_matrix(rng: np.random.Generator) -> np.ndarray:
    """Symmetric 20x20: diagonal uniform in [4, 11], off-diagonal in [-4, 3]."""
    A = PROTEIN_A
    M = rng.integers(-4, 4, size=(A, A))
    M = np.triu(M, 1)
    M = M + M.T
    M[np.arange(A), np.arange(A)] = rng.integers(4, 12, size=A)
    return M.astype(np.int8)


def dna_matrix(match: int = 1, mismatch: int = -4) -> np.ndarray:
    M = np.full((DNA_A, DNA_A), mismatch, dtype=np.int8)
    M[np.arange(DNA_A), np.arange(DNA_A)] = match
    return M


def residues(rng: np.random.Generator, n: int, A: int) -> np.ndarray:
    return rng.integers(0, A, size=int(n), dtype=np.uint8)


def lengths_uniform(rng, n, lo, hi):
    return rng.integers(lo, hi + 1, size=int(n)).astype(np.int64)


def lengths_lognormal(rng, n, median, sigma, lo, hi):
    x = rng.lognormal(mean=np.log(median), sigma=sigma, size=int(n))
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def lengths_loguniform(rng, n, lo, hi):
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), size=int(n)))
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def pack(lengths: np.ndarray, rng, A: int):
    """Concatenated residues (uint8) and offsets (int64, n+1, offsets[0]=0)."""
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return residues(rng, int(off[-1]), A), off


def random_db(rng, n, A, dist="uniform", **kw):
    if dist == "uniform":
        L = lengths_uniform(rng, n, kw["lo"], kw["hi"])
    elif dist == "lognormal":
        L = lengths_lognormal(rng, n, kw.get("median", 300), kw.get("sigma", 0.76),
                              kw.get("lo", 20), kw.get("hi", 35000))
    elif dist == "loguniform":
        L = lengths_loguniform(rng, n, kw["lo"], kw["hi"])
    else:
        raise ValueError(dist)
    return pack(L, rng, A)


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

def workload_protein_small(seed_salt: int = 0, n_db: int = 1000, qlen: int = 256):
    """One protein query (256) vs 1000 db sequences, lengths U{50..500}."""
    rng = rng_for(0, seed_salt)
    M = protein_matrix(rng)
    q = residues(rng, qlen, PROTEIN_A)
    db, off = random_db(rng, n_db, PROTEIN_A, "uniform", lo=50, hi=500)
    return dict(M=M, query=q, db=db, off=off, o=11, e=1)


def workload_protein_scale(seed_salt: int = 0, n_db: int = 100_000,
                           qlens=(128, 512, 2048, 5000), sigma: float = 0.76):
    """Protein queries of the given lengths vs n_db log-normal sequences
    (median 300, clipped to [20, 35000]); sigma 0.76 gives ~40M residues at
    100k sequences."""
    rng = rng_for(1, seed_salt)
    M = protein_matrix(rng)
    queries = [residues(rng, m, PROTEIN_A) for m in qlens]
    db, off = random_db(rng, n_db, PROTEIN_A, "lognormal", median=300,
                        sigma=sigma, lo=20, hi=35000)
    return dict(M=M, queries=queries, db=db, off=off, o=11, e=1)


def _substitute(rng, reads, identity, A):
    """Each base of `reads` (any shape) replaced, with probability
    1 - identity, by one of the other A - 1 bases."""
    hit = rng.random(reads.shape) >= identity
    shift = rng.integers(1, A, size=reads.shape, dtype=np.uint8)
    return np.where(hit, (reads + shift) % A, reads).astype(np.uint8)


def workload_gap_adversary(seed_salt: int = 0, n_pairs: int = 200_000, xlo: int = 60, xhi: int = 150,
                           ylo: int = 40, yhi: int = 200):
    """The lazy-F worst case as read/window pairs: query = X + Y + Z against
    reference = X + Z (X, Z iid DNA of xlo..xhi bases, Y of ylo..yhi random
    bases inserted into the query), so the best alignment carries a vertical
    gap of |Y| through many query segments.  DNA +1/-4, o=6, e=1."""
    rng = rng_for(5, seed_salt)
    A = DNA_A
    n = int(n_pairs)
    xl = rng.integers(xlo, xhi + 1, n)
    yl = rng.integers(ylo, yhi + 1, n)
    zl = rng.integers(xlo, xhi + 1, n)
    qs, rs = [], []
    for i in range(n):
        X = residues(rng, int(xl[i]), A)
        Y = residues(rng, int(yl[i]), A)
        Z = residues(rng, int(zl[i]), A)
        qs.append(np.concatenate([X, Y, Z]))
        rs.append(np.concatenate([X, Z]))
    q_off = np.zeros(n + 1, dtype=np.int64)
    r_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum([len(x) for x in qs], out=q_off[1:])
    np.cumsum([len(x) for x in rs], out=r_off[1:])
    return dict(q=np.concatenate(qs).astype(np.uint8), q_off=q_off, r=np.concatenate(rs).astype(np.uint8),
                r_off=r_off, M=dna_matrix(), o=6, e=1)


def workload_reads(seed_salt: int = 0, n_pairs: int = 1_000_000,
                   read_len: int = 150, win_len: int = 2000):
    """DNA reads vs their own reference windows (mate-rescue stand-in).

    Classes: 30% copies at 95% identity, 10% with a 40-200 bp indel (half
    deletions vs the window -- the read spans a gap of 40-200 bp in the
    window -- and half insertions of 40-100 random bases into the read),
    60% copies at 99% identity.  Copies start at a uniform offset in the
    window; indels are placed at least 25 bases from either read end.
    """
    rng = rng_for(2, seed_salt)
    A = DNA_A
    n = int(n_pairs)
    windows = rng.integers(0, A, size=(n, win_len), dtype=np.uint8)
    u = rng.random(n)
    kinds = np.where(u < 0.30, 0, np.where(u < 0.40, 1, 3)).astype(np.int8)
    ins = (kinds == 1) & (rng.random(n) < 0.5)
    kinds[ins] = 2
    cols = np.arange(read_len)
    # copies (kinds 0 and 3)
    start = rng.integers(0, win_len - read_len + 1, size=n)
    copies = windows[np.arange(n)[:, None], start[:, None] + cols[None, :]]
    ident = np.where(kinds == 0, 0.95, 0.99)[:, None]
    hit = rng.random(copies.shape) >= ident
    shift = rng.integers(1, A, size=copies.shape, dtype=np.uint8)
    reads = np.where(hit, (copies + shift) % A, copies).astype(np.uint8)
    # deletions vs the window (kind 1): read = window[s:s+left] + window[s+left+dl : s+read_len+dl]
    d_idx = np.flatnonzero(kinds == 1)
    if d_idx.size:
        dl = rng.integers(40, 201, size=d_idx.size)
        s0 = (rng.random(d_idx.size) * (win_len - read_len - dl + 1)).astype(np.int64)
        left = rng.integers(25, read_len - 25 + 1, size=d_idx.size)
        src = s0[:, None] + cols[None, :] + np.where(cols[None, :] < left[:, None], 0, dl[:, None])
        reads[d_idx] = _substitute(rng, windows[d_idx[:, None], src], 0.99, A)
    qlen = np.full(n, read_len, dtype=np.int64)
    # insertions into the read (kind 2): ragged lengths read_len + 40..100
    i_idx = np.flatnonzero(kinds == 2)
    il = rng.integers(40, 101, size=i_idx.size)
    qlen[i_idx] = read_len + il
    q_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(qlen, out=q_off[1:])
    q = np.empty(int(q_off[-1]), dtype=np.uint8)
    regular = np.flatnonzero(kinds != 2)
    # fixed-length reads go in with one gather
    pos = q_off[regular][:, None] + cols[None, :]
    q[pos] = reads[regular]
    for k, i in enumerate(i_idx):
        cut = int(rng.integers(25, read_len - 25 + 1))
        piece = np.concatenate([reads[i, :cut], rng.integers(0, A, int(il[k]), dtype=np.uint8), reads[i, cut:]])
        q[q_off[i]:q_off[i + 1]] = piece
    r_off = np.arange(n + 1, dtype=np.int64) * win_len
    return dict(M=dna_matrix(), q=q, q_off=q_off, r=windows.reshape(-1), r_off=r_off, kinds=kinds, o=6, e=1)
