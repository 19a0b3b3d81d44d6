"""Autotuner for the striped kernels: for each query-length bin it times
every compiled layout (lane type x lanes per alignment x segment length) of
sw_align_db on a sample of the database and keeps the fastest.

The layouts are the paper's p (lanes per alignment) and segLen (positions per
lane); the lane type decides how many alignments one register carries.  The
result is a small table, cached as JSON per GPU model, that the batch runner
and the server use to build profiles with sw_profile_build_ex.
"""
import json
import os

import numpy as np

from . import sw

# query-length bins (upper bounds, inclusive)
BINS = (64, 128, 256, 512, 1024, 2048, 4096, 1 << 30)

CANDIDATES = {
    sw.SW_LANE_I16X2: ((8, 8), (8, 16), (16, 8), (16, 16), (32, 8), (32, 12), (32, 16), (16, 32), (32, 24),
                       (32, 32)),
    # one lane (one thread per alignment, no scan) up to warp-wide groups
    sw.SW_LANE_I32: ((1, 16), (1, 32), (4, 8), (4, 32), (8, 8), (8, 16), (16, 8), (16, 16), (32, 8), (32, 12),
                     (32, 16), (16, 32), (32, 32)),
    # split-query s16x2: virtual lanes (two per thread)
    sw.SW_LANE_I16X2Q: ((2, 16), (2, 32), (16, 8), (32, 8), (32, 16), (64, 8), (64, 16), (64, 20), (64, 24),
                        (64, 32)),
}


def bin_of(m):
    for b in BINS:
        if m <= b:
            return b
    return BINS[-1]


def default_cache_path():
    return os.path.join(os.path.expanduser("~"), ".cache", "sw_gb300", "autotune.json")


class Table:
    """Best layout per query-length bin: {bin: (lane, lanes, seg_len, gcups)}."""

    def __init__(self, entries=None, device=""):
        self.entries = dict(entries or {})
        self.device = device

    def plan(self, m):
        """(lane_type, lanes, seg_len) for a query of length m, or None."""
        e = self.entries.get(bin_of(m))
        return None if e is None else tuple(e[:3])

    def to_json(self):
        return {"device": self.device, "entries": {str(k): list(v) for k, v in self.entries.items()}}

    @classmethod
    def from_json(cls, d):
        return cls({int(k): tuple(v) for k, v in d["entries"].items()}, d.get("device", ""))

    def save(self, path=None):
        path = path or default_cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        data = {}
        if os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
        data[self.device] = self.to_json()
        with open(path, "w") as f:
            json.dump(data, f, indent=1)

    @classmethod
    def load(cls, device, path=None):
        path = path or default_cache_path()
        if not os.path.exists(path):
            return None
        with open(path) as f:
            data = json.load(f)
        return cls.from_json(data[device]) if device in data else None


def _time_layout(db, query, M, o, e, lane, L, S, out, reps, stream):
    import torch
    prof = sw.Profile(query, M, lane, stream=stream, lanes=L, seg_len=S)
    try:
        sw.sw_align_db(prof, db, o, e, out, stream=stream)  # warm-up
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            sw.sw_align_db(prof, db, o, e, out, stream=stream)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps
    finally:
        prof.free()


def tune(db, M, o, e, lengths=None, lanes=(sw.SW_LANE_I16X2, sw.SW_LANE_I16X2Q, sw.SW_LANE_I32), reps=2, seed=0,
         device_name=None, verbose=False):
    """Times every candidate layout for one query per length bin against the
    resident database `db` and returns the best per bin."""
    import torch
    rng = np.random.default_rng(seed)
    A = M.shape[0]
    stream = torch.cuda.current_stream()
    cells_db = int(db.offsets[-1].item())
    out = torch.empty(max(db.n, 1), dtype=torch.int32, device="cuda")
    lengths = lengths or [min(b, 6000) for b in BINS]
    best = {}
    for m in lengths:
        q = rng.integers(0, A, m).astype(np.uint8)
        cands = []
        for lane in lanes:
            for (L, S) in CANDIDATES[lane]:
                if L * S > 4 * max(m, 16):
                    continue  # mostly padding
                if (m + L * S - 1) // (L * S) > 8:
                    continue  # many chunks: each re-streams the database
                ms = _time_layout(db, q, M, o, e, lane, L, S, out, reps, stream)
                g = m * cells_db / (ms * 1e-3) / 1e9
                cands.append((g, lane, L, S))
                if verbose:
                    print("m=%d lane=%d L=%d S=%d: %.1f GCUPS" % (m, lane, L, S, g))
        g, lane, L, S = max(cands)
        best[bin_of(m)] = (lane, L, S, g)
    name = device_name or torch.cuda.get_device_name()
    return Table(best, name)
