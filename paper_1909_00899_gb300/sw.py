"""ctypes binding of libsw_gb300.so (include/sw_gb300.h), same names as the
C entry points.  Argument marshalling only: tensors are passed by
``data_ptr()``, streams by ``torch.cuda.Stream.cuda_stream``; every compute
step runs in the library's CUDA kernels.

The library is loaded on first use; if it is missing or cannot be loaded the
call raises (there is no CPU fallback).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsw_gb300.so")

SW_OK = 0
SW_ERR_INVALID = -1
SW_ERR_CUDA = -2
SW_ERR_NOMEM = -3
SW_ERR_TIMEOUT = -4
SW_ERR_RANGE = -5

SW_LANE_AUTO = 0
SW_LANE_I32 = 1
SW_LANE_I16X2 = 2
SW_LANE_I8X4 = 3
SW_LANE_I16X2Q = 4

# every function declared in include/sw_gb300.h
EXPORTS = (
    "sw_profile_build", "sw_profile_build_ex", "sw_profile_free", "sw_profile_free_async", "sw_profile_plan",
    "sw_align_batch", "sw_align_lazyf_batch", "sw_align_pairs", "sw_stream_sync", "sw_last_error",
    "sw_probe_cell_rate", "sw_probe_cell_rate_pass", "sw_version", "sw_db_create", "sw_db_free", "sw_align_db",
    "sw_align_db_ends", "sw_align_lazyf_db", "sw_align_lazyf_pairs", "sw_align_lazyf_db_stats",
    "sw_align_batch_noalloc", "sw_align_batch_ends", "sw_plan_query", "sw_align_pairs_ends",
    "sw_align_lazyf_pairs_lane", "sw_multi_create", "sw_align_multi", "sw_multi_free", "sw_multi_status",
    "sw_multi_set_wait", "sw_mem_available",
)


class SwError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


def lib():
    """Load the library (raises OSError if it is missing: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libsw_gb300.so is not built (run __graft_entry__.build()); "
                          "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        L.sw_profile_build.restype = ctypes.c_int
        L.sw_profile_build.argtypes = [_vp, _i32, _vp, _i32, _i32, _vp, ctypes.POINTER(_vp)]
        L.sw_profile_build_ex.restype = ctypes.c_int
        L.sw_profile_build_ex.argtypes = [_vp, _i32, _vp, _i32, _i32, _i32, _i32, _vp, ctypes.POINTER(_vp)]
        L.sw_profile_free.restype = ctypes.c_int
        L.sw_profile_free.argtypes = [_vp]
        L.sw_profile_free_async.restype = ctypes.c_int
        L.sw_profile_free_async.argtypes = [_vp, _vp]
        L.sw_profile_plan.restype = ctypes.c_int
        L.sw_profile_plan.argtypes = [_vp] + [ctypes.POINTER(_i32)] * 4
        L.sw_plan_query.restype = ctypes.c_int
        L.sw_plan_query.argtypes = [_i32, _i32] + [ctypes.POINTER(_i32)] * 4
        for name in ("sw_align_batch", "sw_align_lazyf_batch", "sw_align_batch_noalloc"):
            f = getattr(L, name)
            f.restype = ctypes.c_int
            f.argtypes = [_vp, _vp, _vp, _i64, _i32, _i32, _vp, _vp]
        L.sw_align_batch_ends.restype = ctypes.c_int
        L.sw_align_batch_ends.argtypes = [_vp, _vp, _vp, _i64, _i32, _i32, _vp, _vp, _vp, _vp]
        L.sw_align_pairs.restype = ctypes.c_int
        L.sw_align_pairs.argtypes = [_vp, _vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _i32, _vp, _vp]
        L.sw_align_pairs_ends.restype = ctypes.c_int
        L.sw_align_pairs_ends.argtypes = [_vp, _vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp]
        L.sw_db_create.restype = ctypes.c_int
        L.sw_db_create.argtypes = [_vp, _vp, _i64, _vp, ctypes.POINTER(_vp)]
        L.sw_db_free.restype = ctypes.c_int
        L.sw_db_free.argtypes = [_vp]
        for name in ("sw_align_db", "sw_align_lazyf_db"):
            f = getattr(L, name)
            f.restype = ctypes.c_int
            f.argtypes = [_vp, _vp, _i32, _i32, _vp, _vp]
        L.sw_align_db_ends.restype = ctypes.c_int
        L.sw_align_db_ends.argtypes = [_vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp]
        L.sw_align_lazyf_pairs.restype = ctypes.c_int
        L.sw_align_lazyf_pairs.argtypes = [_vp, _vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _vp, _vp, _vp]
        L.sw_align_lazyf_pairs_lane.restype = ctypes.c_int
        L.sw_align_lazyf_pairs_lane.argtypes = [_vp, _vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _i32, _vp, _vp,
                                                _vp]
        L.sw_align_lazyf_db_stats.restype = ctypes.c_int
        L.sw_align_lazyf_db_stats.argtypes = [_vp, _vp, _i32, _i32, _vp, _vp, _vp]
        L.sw_multi_create.restype = ctypes.c_int
        L.sw_multi_create.argtypes = [_vp, _i32, _vp, _i32, _vp, ctypes.POINTER(_vp)]
        L.sw_align_multi.restype = ctypes.c_int
        L.sw_align_multi.argtypes = [_vp, _i32, _i32, _vp, _i64, _vp]
        L.sw_multi_free.restype = ctypes.c_int
        L.sw_multi_free.argtypes = [_vp]
        L.sw_multi_status.restype = ctypes.c_int
        L.sw_multi_status.argtypes = [_vp, ctypes.POINTER(_i32), _vp]
        L.sw_multi_set_wait.restype = ctypes.c_int
        L.sw_multi_set_wait.argtypes = [_vp, _i32, _i32]
        L.sw_mem_available.restype = ctypes.c_int
        L.sw_mem_available.argtypes = [ctypes.POINTER(_i64)]
        L.sw_stream_sync.restype = ctypes.c_int
        L.sw_stream_sync.argtypes = [_vp, _i64]
        L.sw_last_error.restype = ctypes.c_char_p
        L.sw_last_error.argtypes = []
        L.sw_version.restype = ctypes.c_char_p
        L.sw_version.argtypes = []
        L.sw_probe_cell_rate.restype = ctypes.c_int
        L.sw_probe_cell_rate.argtypes = [_i32, _i32, ctypes.POINTER(ctypes.c_double), _vp]
        L.sw_probe_cell_rate_pass.restype = ctypes.c_int
        L.sw_probe_cell_rate_pass.argtypes = [_i32, _i32, _i32, ctypes.POINTER(ctypes.c_double), _vp]
        _lib = L
    return _lib


def _check(rc):
    if rc != SW_OK:
        raise SwError(rc, lib().sw_last_error().decode(errors="replace"))
    return rc


def _stream(stream):
    """A torch stream, an int handle or None (current torch stream)."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(t, dtype_name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype) != "torch." + dtype_name:
        raise TypeError("expected dtype %s, got %s" % (dtype_name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


class Profile:
    """Owns a device profile built by sw_profile_build."""

    def __init__(self, query, subst_matrix, lane_type=SW_LANE_AUTO, stream=None, lanes=0, seg_len=0):
        q = np.ascontiguousarray(query, dtype=np.uint8)
        M = np.ascontiguousarray(subst_matrix, dtype=np.int8)
        if M.ndim != 2 or M.shape[0] != M.shape[1]:
            raise ValueError("subst_matrix must be square")
        self.qlen = int(q.size)
        self.alphabet = int(M.shape[0])
        h = _vp()
        _check(lib().sw_profile_build_ex(q.ctypes.data if q.size else None, self.qlen,
                                         M.ctypes.data, self.alphabet, lane_type, int(lanes),
                                         int(seg_len), _stream(stream), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def plan(self):
        vals = [_i32() for _ in range(4)]
        _check(lib().sw_profile_plan(self._h, *[ctypes.byref(v) for v in vals]))
        return dict(lanes=vals[0].value, seg_len=vals[1].value, chunks=vals[2].value,
                    lane_type=vals[3].value)

    def free(self):
        """Waits for the device, then releases the profile."""
        if getattr(self, "_h", None):
            lib().sw_profile_free(self._h)
            self._h = None

    def free_async(self, stream=None):
        """Releases the profile in stream order (no wait)."""
        if getattr(self, "_h", None):
            _check(lib().sw_profile_free_async(self._h, _stream(stream)))
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sw_profile_build(query, subst_matrix, lane_type=SW_LANE_AUTO, stream=None):
    return Profile(query, subst_matrix, lane_type, stream)


def sw_profile_build_ex(query, subst_matrix, lane_type, lanes, seg_len, stream=None):
    return Profile(query, subst_matrix, lane_type, stream, lanes, seg_len)


def sw_profile_free(profile):
    profile.free()


def sw_profile_free_async(profile, stream=None):
    profile.free_async(stream)


def _align(fn, profile, db_residues, db_offsets, gap_open, gap_extend, scores_out, stream):
    n_db = int(db_offsets.numel()) - 1
    if n_db < 0:
        raise ValueError("db_offsets needs n_db + 1 entries")
    if scores_out.numel() < n_db:
        raise ValueError("scores_out too small")
    _check(fn(profile.handle, _dev_ptr(db_residues, "uint8"), _dev_ptr(db_offsets, "int64"),
              n_db, int(gap_open), int(gap_extend), _dev_ptr(scores_out, "int32"), _stream(stream)))
    return scores_out


def sw_align_batch(profile, db_residues, db_offsets, gap_open, gap_extend, scores_out, stream=None):
    """Scan-F (Alg. 6) scores of profile's query against every db sequence."""
    return _align(lib().sw_align_batch, profile, db_residues, db_offsets, gap_open, gap_extend,
                  scores_out, stream)


def sw_align_batch_ends(profile, db_residues, db_offsets, gap_open, gap_extend, scores_out, q_end_out,
                        r_end_out, stream=None):
    """Scores and end cells (1-based query / reference position of the first
    cell in column order reaching the score; -1 when the score is 0)."""
    n_db = int(db_offsets.numel()) - 1
    for t in (scores_out, q_end_out, r_end_out):
        if t.numel() < n_db:
            raise ValueError("output too small")
    _check(lib().sw_align_batch_ends(profile.handle, _dev_ptr(db_residues, "uint8"),
                                     _dev_ptr(db_offsets, "int64"), n_db, int(gap_open), int(gap_extend),
                                     _dev_ptr(scores_out, "int32"), _dev_ptr(q_end_out, "int32"),
                                     _dev_ptr(r_end_out, "int32"), _stream(stream)))
    return scores_out, q_end_out, r_end_out


def sw_align_lazyf_batch(profile, db_residues, db_offsets, gap_open, gap_extend, scores_out, stream=None):
    """Lazy-F (Alg. 1) scores, the plain-method comparison."""
    return _align(lib().sw_align_lazyf_batch, profile, db_residues, db_offsets, gap_open, gap_extend,
                  scores_out, stream)


def sw_align_batch_noalloc(profile, db_residues, db_offsets, gap_open, gap_extend, scores_out, stream=None):
    """sw_align_batch without device allocation: scratch comes from the
    library's fixed device array (SW_NOALLOC_SCRATCH_BYTES); concurrent calls
    must be serialised by the caller."""
    return _align(lib().sw_align_batch_noalloc, profile, db_residues, db_offsets, gap_open, gap_extend,
                  scores_out, stream)


def sw_align_pairs(q, q_off, r, r_off, subst_matrix, gap_open, gap_extend, scores_out,
                   lane_type=SW_LANE_AUTO, stream=None):
    """Pair k: q[q_off[k]:q_off[k+1]] against r[r_off[k]:r_off[k+1]]."""
    M = np.ascontiguousarray(subst_matrix, dtype=np.int8)
    n = int(q_off.numel()) - 1
    if int(r_off.numel()) - 1 != n:
        raise ValueError("q_off and r_off must have the same length")
    _check(lib().sw_align_pairs(_dev_ptr(q, "uint8"), _dev_ptr(q_off, "int64"), _dev_ptr(r, "uint8"),
                                _dev_ptr(r_off, "int64"), n, M.ctypes.data, int(M.shape[0]),
                                int(gap_open), int(gap_extend), int(lane_type),
                                _dev_ptr(scores_out, "int32"), _stream(stream)))
    return scores_out


def sw_align_pairs_ends(q, q_off, r, r_off, subst_matrix, gap_open, gap_extend, scores_out, q_end_out, r_end_out,
                        lane_type=SW_LANE_AUTO, stream=None):
    """sw_align_pairs plus the 1-based end cell (q_end_out, r_end_out) of
    each pair's best alignment (-1, -1 when the score is 0)."""
    M = np.ascontiguousarray(subst_matrix, dtype=np.int8)
    n = int(q_off.numel()) - 1
    if int(r_off.numel()) - 1 != n:
        raise ValueError("q_off and r_off must have the same length")
    _check(lib().sw_align_pairs_ends(_dev_ptr(q, "uint8"), _dev_ptr(q_off, "int64"), _dev_ptr(r, "uint8"),
                                     _dev_ptr(r_off, "int64"), n, M.ctypes.data, int(M.shape[0]),
                                     int(gap_open), int(gap_extend), int(lane_type),
                                     _dev_ptr(scores_out, "int32"), _dev_ptr(q_end_out, "int32"),
                                     _dev_ptr(r_end_out, "int32"), _stream(stream)))
    return scores_out, q_end_out, r_end_out


class Database:
    """A device-resident database (sw_db): keeps references to the residue
    and offset tensors, which must stay alive while the handle exists."""

    def __init__(self, db_residues, db_offsets, stream=None):
        self.residues = db_residues
        self.offsets = db_offsets
        self.n = int(db_offsets.numel()) - 1
        h = _vp()
        _check(lib().sw_db_create(_dev_ptr(db_residues, "uint8"), _dev_ptr(db_offsets, "int64"),
                                  self.n, _stream(stream), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def free(self):
        if getattr(self, "_h", None):
            lib().sw_db_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sw_db_create(db_residues, db_offsets, stream=None):
    return Database(db_residues, db_offsets, stream)


def sw_db_free(db):
    db.free()


def sw_align_db(profile, db, gap_open, gap_extend, scores_out, stream=None):
    """Scan-F scores against a resident database (graph-capturable)."""
    if scores_out.numel() < db.n:
        raise ValueError("scores_out too small")
    _check(lib().sw_align_db(profile.handle, db.handle, int(gap_open), int(gap_extend),
                             _dev_ptr(scores_out, "int32"), _stream(stream)))
    return scores_out


def sw_align_db_ends(profile, db, gap_open, gap_extend, scores_out, q_end_out, r_end_out, stream=None):
    """Scores and end cells against a resident database (as sw_align_batch_ends)."""
    for t in (scores_out, q_end_out, r_end_out):
        if t.numel() < db.n:
            raise ValueError("output too small")
    _check(lib().sw_align_db_ends(profile.handle, db.handle, int(gap_open), int(gap_extend),
                                  _dev_ptr(scores_out, "int32"), _dev_ptr(q_end_out, "int32"),
                                  _dev_ptr(r_end_out, "int32"), _stream(stream)))
    return scores_out, q_end_out, r_end_out


def sw_align_lazyf_db(profile, db, gap_open, gap_extend, scores_out, stream=None):
    if scores_out.numel() < db.n:
        raise ValueError("scores_out too small")
    _check(lib().sw_align_lazyf_db(profile.handle, db.handle, int(gap_open), int(gap_extend),
                                   _dev_ptr(scores_out, "int32"), _stream(stream)))
    return scores_out


def sw_align_lazyf_pairs(q, q_off, r, r_off, subst_matrix, gap_open, gap_extend, scores_out,
                         lazy_steps=None, stream=None, lane_type=None):
    """Lazy-F (Alg. 1) pair scores; lazy_steps: optional int64 CUDA tensor
    of one element that accumulates the correction loop's j-steps.
    lane_type: None (int32 lanes, sw_align_lazyf_pairs) or a lane type
    (sw_align_lazyf_pairs_lane: SW_LANE_I16X2Q runs on the split layout)."""
    M = np.ascontiguousarray(subst_matrix, dtype=np.int8)
    n = int(q_off.numel()) - 1
    if int(r_off.numel()) - 1 != n:
        raise ValueError("q_off and r_off must have the same length")
    steps = _dev_ptr(lazy_steps, "int64") if lazy_steps is not None else None
    if lane_type is None:
        _check(lib().sw_align_lazyf_pairs(_dev_ptr(q, "uint8"), _dev_ptr(q_off, "int64"), _dev_ptr(r, "uint8"),
                                          _dev_ptr(r_off, "int64"), n, M.ctypes.data, int(M.shape[0]),
                                          int(gap_open), int(gap_extend), _dev_ptr(scores_out, "int32"),
                                          steps, _stream(stream)))
    else:
        _check(lib().sw_align_lazyf_pairs_lane(_dev_ptr(q, "uint8"), _dev_ptr(q_off, "int64"), _dev_ptr(r, "uint8"),
                                               _dev_ptr(r_off, "int64"), n, M.ctypes.data, int(M.shape[0]),
                                               int(gap_open), int(gap_extend), int(lane_type),
                                               _dev_ptr(scores_out, "int32"), steps, _stream(stream)))
    return scores_out


def sw_align_lazyf_db_stats(profile, db, gap_open, gap_extend, scores_out, lazy_steps=None, stream=None):
    if scores_out.numel() < db.n:
        raise ValueError("scores_out too small")
    steps = _dev_ptr(lazy_steps, "int64") if lazy_steps is not None else None
    _check(lib().sw_align_lazyf_db_stats(profile.handle, db.handle, int(gap_open), int(gap_extend),
                                         _dev_ptr(scores_out, "int32"), steps, _stream(stream)))
    return scores_out


class Multi:
    """A batch of profiled queries against one resident database
    (sw_multi): keeps references to the profiles and the database, which
    must stay alive while the handle exists."""

    def __init__(self, profiles, db, stream=None, items_per_group=0):
        self.profiles = list(profiles)
        self.db = db
        arr = (_vp * max(1, len(self.profiles)))(*[p.handle for p in self.profiles])
        h = _vp()
        _check(lib().sw_multi_create(arr, len(self.profiles), db.handle, int(items_per_group), _stream(stream),
                                     ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def free(self):
        if getattr(self, "_h", None):
            lib().sw_multi_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sw_multi_create(profiles, db, items_per_group=0, stream=None):
    return Multi(profiles, db, stream, items_per_group)


def sw_multi_free(batch):
    batch.free()


def sw_multi_status(batch, stream=None):
    """The batch's status word (then cleared): 0, or 1 when a bounded wait
    of the chunk-phase walk gave up since the last read."""
    out = _i32(0)
    _check(lib().sw_multi_status(batch.handle, ctypes.byref(out), _stream(stream)))
    return int(out.value)


def sw_multi_set_wait(batch, max_polls=0, unreachable=False):
    """Bound of the chunk-phase walk's waits (polls of about 256 ns; 0: the
    default, about a second); unreachable=True makes every wait run out
    (a test of the bound: the status word is set, the scores undefined)."""
    _check(lib().sw_multi_set_wait(batch.handle, int(max_polls), 1 if unreachable else 0))


def sw_align_multi(batch, gap_open, gap_extend, scores_out, stream=None):
    """Scores of every query of the batch against the database: scores_out
    is a 2-D int32 CUDA tensor [n_queries, >= n_db] (rows may be padded);
    one persistent launch per layout, graph-capturable."""
    if scores_out.dim() != 2 or scores_out.shape[0] < len(batch.profiles) or scores_out.shape[1] < batch.db.n:
        raise ValueError("scores_out must be [n_queries, >= n_db]")
    if scores_out.stride(1) != 1:
        raise ValueError("scores_out rows must be contiguous")
    if str(scores_out.dtype) != "torch.int32" or not scores_out.is_cuda:
        raise TypeError("expected an int32 CUDA tensor")
    _check(lib().sw_align_multi(batch.handle, int(gap_open), int(gap_extend), scores_out.data_ptr(),
                                int(scores_out.stride(0)), _stream(stream)))
    return scores_out


def sw_plan_query(qlen, lane_type=SW_LANE_AUTO):
    """The plan a profile of qlen residues would get (host only)."""
    vals = [_i32() for _ in range(4)]
    _check(lib().sw_plan_query(int(qlen), int(lane_type), *[ctypes.byref(v) for v in vals]))
    return dict(lanes=vals[0].value, seg_len=vals[1].value, chunks=vals[2].value, lane_type=vals[3].value)


def sw_mem_available():
    """Bytes of device memory a new call could use now (free memory plus
    the idle blocks of the device's stream-ordered pool)."""
    out = _i64(0)
    _check(lib().sw_mem_available(ctypes.byref(out)))
    return int(out.value)


def sw_stream_sync(stream=None, timeout_ms=60_000):
    return _check(lib().sw_stream_sync(_stream(stream), int(timeout_ms)))


def sw_last_error():
    return lib().sw_last_error().decode(errors="replace")


def sw_version():
    return lib().sw_version().decode()


def sw_probe_cell_rate(lane_type=SW_LANE_I32, iters=4096, stream=None):
    out = ctypes.c_double(0.0)
    _check(lib().sw_probe_cell_rate(int(lane_type), int(iters), ctypes.byref(out), _stream(stream)))
    return out.value


def sw_probe_cell_rate_pass(lane_type=SW_LANE_I32, corrected=0, iters=4096, stream=None):
    out = ctypes.c_double(0.0)
    _check(lib().sw_probe_cell_rate_pass(int(lane_type), int(corrected), int(iters), ctypes.byref(out),
                                         _stream(stream)))
    return out.value
