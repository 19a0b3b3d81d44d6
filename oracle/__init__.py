"""ctypes front of the C oracle (oracle/sw_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg, never by the product package.  Every function
takes numpy arrays of residue codes (uint8), a substitution matrix (int8,
A*A row-major, indexed [query residue][reference residue]) and the gap costs
(gap of length k costs o + (k-1)*e) and returns exact int32 scores.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_i8p = ctypes.POINTER(ctypes.c_int8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name in ("oracle_gotoh", "oracle_brute"):
            f = getattr(L, name)
            f.restype = _i32
            f.argtypes = [_u8p, _i32, _u8p, _i32, _i8p, _i32, _i32, _i32]
        L.oracle_striped_lazyf.restype = _i32
        L.oracle_striped_lazyf.argtypes = [_u8p, _i32, _u8p, _i32, _i8p, _i32,
                                           _i32, _i32, _i32, _i64p]
        L.oracle_striped_scan.restype = _i32
        L.oracle_striped_scan.argtypes = [_u8p, _i32, _u8p, _i32, _i8p, _i32,
                                          _i32, _i32, _i32]
        L.oracle_gotoh_batch.restype = None
        L.oracle_gotoh_batch.argtypes = [_u8p, _i32, _u8p, _i64p, _i64, _i8p,
                                         _i32, _i32, _i32, _i32p, _i32]
        for name in ("oracle_gotoh_end", "oracle_brute_end"):
            f = getattr(L, name)
            f.restype = _i32
            f.argtypes = [_u8p, _i32, _u8p, _i32, _i8p, _i32, _i32, _i32, _i32p, _i32p]
        L.oracle_gotoh_end_batch.restype = None
        L.oracle_gotoh_end_batch.argtypes = [_u8p, _i32, _u8p, _i64p, _i64, _i8p, _i32, _i32, _i32,
                                             _i32p, _i32p, _i32p, _i32]
        L.oracle_gotoh_pairs.restype = None
        L.oracle_gotoh_pairs.argtypes = [_u8p, _i64p, _u8p, _i64p, _i64, _i8p,
                                         _i32, _i32, _i32, _i32p, _i32]
        _lib = L
    return _lib


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(_u8p)


def _mat(M):
    M = np.ascontiguousarray(M, dtype=np.int8)
    assert M.ndim == 2 and M.shape[0] == M.shape[1]
    return M, M.ctypes.data_as(_i8p), M.shape[0]


def gotoh(q, r, M, o, e):
    """Plain textbook score (the definition)."""
    q, qp = _u8(q)
    r, rp = _u8(r)
    M, Mp, A = _mat(M)
    return lib().oracle_gotoh(qp, len(q), rp, len(r), Mp, A, o, e)


def brute(q, r, M, o, e):
    """Enumerates every local alignment; lengths <= 9 only."""
    q, qp = _u8(q)
    r, rp = _u8(r)
    M, Mp, A = _mat(M)
    if len(q) > 9 or len(r) > 9:
        raise ValueError("brute force is limited to lengths <= 9")
    return lib().oracle_brute(qp, len(q), rp, len(r), Mp, A, o, e)


def striped_lazyf(q, r, M, o, e, p, return_steps=False):
    """Alg. 1 (striped, lazy-F loop) with p lanes."""
    q, qp = _u8(q)
    r, rp = _u8(r)
    M, Mp, A = _mat(M)
    steps = ctypes.c_int64(0)
    s = lib().oracle_striped_lazyf(qp, len(q), rp, len(r), Mp, A, o, e, p,
                                   ctypes.byref(steps))
    return (s, steps.value) if return_steps else s


def striped_scan(q, r, M, o, e, p):
    """Alg. 6 (striped, max-plus scan of F) with p lanes."""
    q, qp = _u8(q)
    r, rp = _u8(r)
    M, Mp, A = _mat(M)
    return lib().oracle_striped_scan(qp, len(q), rp, len(r), Mp, A, o, e, p)


def gotoh_batch(query, db, db_off, M, o, e, nthreads=None):
    """One query against every db sequence; returns int32[n_db]."""
    query, qp = _u8(query)
    db, dp = _u8(db)
    off = np.ascontiguousarray(db_off, dtype=np.int64)
    M, Mp, A = _mat(M)
    n = len(off) - 1
    out = np.zeros(n, dtype=np.int32)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    lib().oracle_gotoh_batch(qp, len(query), dp, off.ctypes.data_as(_i64p), n,
                             Mp, A, o, e, out.ctypes.data_as(_i32p), nthreads)
    return out


def gotoh_pairs(q, q_off, r, r_off, M, o, e, nthreads=None):
    """Pair k: q[q_off[k]:q_off[k+1]] vs r[r_off[k]:r_off[k+1]]."""
    q, qp = _u8(q)
    r, rp = _u8(r)
    qo = np.ascontiguousarray(q_off, dtype=np.int64)
    ro = np.ascontiguousarray(r_off, dtype=np.int64)
    assert len(qo) == len(ro)
    M, Mp, A = _mat(M)
    n = len(qo) - 1
    out = np.zeros(n, dtype=np.int32)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    lib().oracle_gotoh_pairs(qp, qo.ctypes.data_as(_i64p), rp,
                             ro.ctypes.data_as(_i64p), n, Mp, A, o, e,
                             out.ctypes.data_as(_i32p), nthreads)
    return out


def gotoh_end(q, r, M, o, e):
    """(score, q_end, r_end): the first cell in column order (1-based) whose
    H equals the score; (-1, -1) when the score is 0."""
    q, qp = _u8(q)
    r, rp = _u8(r)
    M, Mp, A = _mat(M)
    qe, re_ = ctypes.c_int32(), ctypes.c_int32()
    s = lib().oracle_gotoh_end(qp, len(q), rp, len(r), Mp, A, o, e, ctypes.byref(qe), ctypes.byref(re_))
    return s, qe.value, re_.value


def brute_end(q, r, M, o, e):
    q, qp = _u8(q)
    r, rp = _u8(r)
    M, Mp, A = _mat(M)
    if len(q) > 9 or len(r) > 9:
        raise ValueError("brute force is limited to lengths <= 9")
    qe, re_ = ctypes.c_int32(), ctypes.c_int32()
    s = lib().oracle_brute_end(qp, len(q), rp, len(r), Mp, A, o, e, ctypes.byref(qe), ctypes.byref(re_))
    return s, qe.value, re_.value


def gotoh_end_pairs(q, q_off, r, r_off, M, o, e):
    """Scores, q_end, r_end (int32[n] each) of pair k: q[q_off[k]:q_off[k+1]]
    against r[r_off[k]:r_off[k+1]], one oracle_gotoh_end call per pair."""
    n = len(q_off) - 1
    out = np.zeros(n, dtype=np.int32)
    qe = np.zeros(n, dtype=np.int32)
    re_ = np.zeros(n, dtype=np.int32)
    for k in range(n):
        out[k], qe[k], re_[k] = gotoh_end(q[q_off[k]:q_off[k + 1]], r[r_off[k]:r_off[k + 1]], M, o, e)
    return out, qe, re_


def gotoh_end_batch(query, db, db_off, M, o, e, nthreads=None):
    """Scores, q_end, r_end (int32[n_db] each) of one query against every
    db sequence."""
    query, qp = _u8(query)
    db, dp = _u8(db)
    off = np.ascontiguousarray(db_off, dtype=np.int64)
    M, Mp, A = _mat(M)
    n = len(off) - 1
    out = np.zeros(n, dtype=np.int32)
    qe = np.zeros(n, dtype=np.int32)
    re_ = np.zeros(n, dtype=np.int32)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    lib().oracle_gotoh_end_batch(qp, len(query), dp, off.ctypes.data_as(_i64p), n, Mp, A, o, e,
                                 out.ctypes.data_as(_i32p), qe.ctypes.data_as(_i32p),
                                 re_.ctypes.data_as(_i32p), nthreads)
    return out, qe, re_
