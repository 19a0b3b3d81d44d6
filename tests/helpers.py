"""Shared helpers of the GPU tests: device copies and oracle expectations."""
import numpy as np

import oracle


def to_dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def db_to_dev(db, off):
    import torch
    return to_dev(db, torch.uint8), to_dev(off, torch.int64)


def expect_batch(query, db, off, M, o, e):
    return oracle.gotoh_batch(query, db, off, M, o, e)


def gap_adversary(rng, A, n_pairs, xlo=20, xhi=80, ylo=40, yhi=200):
    """Query-side insertions: query = X+Y+Z, reference = X+Z (the lazy-F
    worst case: a vertical gap crossing many segments)."""
    refs, queries = [], []
    for _ in range(n_pairs):
        X = rng.integers(0, A, int(rng.integers(xlo, xhi))).astype(np.uint8)
        Y = rng.integers(0, A, int(rng.integers(ylo, yhi))).astype(np.uint8)
        Z = rng.integers(0, A, int(rng.integers(xlo, xhi))).astype(np.uint8)
        queries.append(np.concatenate([X, Y, Z]))
        refs.append(np.concatenate([X, Z]))
    return queries, refs


def pack_list(seqs):
    off = np.zeros(len(seqs) + 1, dtype=np.int64)
    np.cumsum([len(s) for s in seqs], out=off[1:])
    flat = np.concatenate(seqs).astype(np.uint8) if len(seqs) else np.zeros(0, np.uint8)
    return flat, off
