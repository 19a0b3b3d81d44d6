"""Autotuner for the striped kernels: for each query-length bin it times
every compiled layout (lane type x lanes per alignment x segment length) of
sw_align_db against the database and keeps every layout's measured rate per
processed cell.  A query then gets the layout that maximises

    rate x m / (C x L x S) / (1 + 1.5 % x (C - 1)),   C = ceil(m / (L x S)),

for its own length m: the rate measured in its bin, the fraction of the
C chunks' L x S positions that are real, and a small cost per extra chunk
launch (each re-streams the database and hands boundary rows on).  So two
queries of the same bin can take different layouts when one of them fills a
layout's chunks and the other would mostly pad them.

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
    sw.SW_LANE_I16X2Q: ((2, 16), (2, 32), (16, 8), (16, 32), (32, 8), (32, 12), (32, 16), (32, 20), (32, 24), (32, 32),
                        (32, 40), (64, 8), (64, 16), (64, 20), (64, 24), (64, 28), (64, 32), (64, 40)),
}


CHUNK_COST = 0.015  # per extra chunk launch, as in the library's automatic plan


def chunks_of(m, L, S):
    return max(1, (int(m) + L * S - 1) // (L * S))


def admissible(m, L, S):
    """The layouts worth timing or choosing for a query of length m: not
    mostly padding, and at most 8 chunk launches."""
    return L * S <= 4 * max(int(m), 16) and chunks_of(m, L, S) <= 8


def expected_gcups(m, L, S, rate):
    """Cells of the query per second on a layout whose measured rate per
    processed cell is `rate`."""
    C = chunks_of(m, L, S)
    return rate * max(int(m), 1) / (C * L * S) / (1.0 + CHUNK_COST * (C - 1))


def bin_of(m):
    for b in BINS:
        if m <= b:
            return b
    return BINS[-1]


def default_cache_path():
    return os.path.join(os.path.expanduser("~"), ".cache", "sw_gb300", "autotune.json")


class Table:
    """Measured layouts per query-length bin:
    {bin: [(lane, lanes, seg_len, GCUPS per processed cell), ...]}."""

    def __init__(self, entries=None, device=""):
        self.entries = {int(k): [tuple(c) for c in v] for k, v in (entries or {}).items()}
        self.device = device

    def plan(self, m):
        """(lane_type, lanes, seg_len) for a query of length m: the bin's
        layout with the highest expected rate at this length, or None."""
        cands = self.entries.get(bin_of(m))
        if not cands:
            return None
        ok = [c for c in cands if admissible(m, c[1], c[2])] or cands
        best = max(ok, key=lambda c: expected_gcups(m, c[1], c[2], c[3]))
        return tuple(best[:3])

    def to_json(self):
        return {"device": self.device, "version": 2,
                "entries": {str(k): [list(c) for c in v] for k, v in self.entries.items()}}

    @classmethod
    def from_json(cls, d):
        if d.get("version", 1) < 2:
            # one (lane, lanes, seg_len, gcups) per bin: keep it as the
            # bin's only layout
            return cls({int(k): [tuple(v)] for k, v in d["entries"].items()}, d.get("device", ""))
        return cls({int(k): [tuple(c) for c in v] for k, v in d["entries"].items()}, d.get("device", ""))

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


def _time_layout_multi(db, queries, M, o, e, L, S, out, reps, stream):
    """ms per query of one batched launch (sw_align_multi) over `queries`,
    all of one length on one split layout: the way a ragged batch runs
    them, where the launch's tail is one query's, not every query's."""
    import torch
    profs = [sw.Profile(q, M, sw.SW_LANE_I16X2Q, stream=stream, lanes=L, seg_len=S) for q in queries]
    batch = None
    try:
        batch = sw.Multi(profs, db, stream=stream)
        sw.sw_align_multi(batch, o, e, out, stream=stream)  # warm-up
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            sw.sw_align_multi(batch, o, e, out, stream=stream)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps / len(queries)
    finally:
        if batch is not None:
            batch.free()
        for p in profs:
            p.free()


def tune(db, M, o, e, lengths=None, lanes=(sw.SW_LANE_I16X2, sw.SW_LANE_I16X2Q, sw.SW_LANE_I32), reps=2, seed=0,
         device_name=None, verbose=False, batched=0):
    """Times every admissible layout for one query per length bin against
    the resident database `db` and returns each layout's rate per processed
    cell, per bin.  batched = k > 0 times the split layouts of the batched
    launch (16 or more virtual lanes) as one sw_align_multi over k queries
    of the length instead, the rate a ragged batch sees (no per-query
    launch tail); use that table with BatchAligner's batched mode."""
    import torch
    rng = np.random.default_rng(seed)
    A = M.shape[0]
    stream = torch.cuda.current_stream()
    cells_db = int(db.offsets[-1].item())
    out = torch.empty(max(db.n, 1), dtype=torch.int32, device="cuda")
    lengths = lengths or [min(b, 6000) for b in BINS]
    best = {}
    if batched:
        out_k = torch.empty((batched, max(db.n, 1)), dtype=torch.int32, device="cuda")
    for m in lengths:
        q = rng.integers(0, A, m).astype(np.uint8)
        qs = [q] + [rng.integers(0, A, m).astype(np.uint8) for _ in range(max(0, batched - 1))]
        cands = []
        for lane in lanes:
            for (L, S) in CANDIDATES[lane]:
                if not admissible(m, L, S):
                    continue
                if batched and lane == sw.SW_LANE_I16X2Q and L >= 16:
                    ms = _time_layout_multi(db, qs, M, o, e, L, S, out_k, reps, stream)
                else:
                    ms = _time_layout(db, q, M, o, e, lane, L, S, out, reps, stream)
                C = chunks_of(m, L, S)
                # per processed cell, with the extra chunk launches of this
                # length taken out again (expected_gcups charges them per m)
                rate = C * L * S * cells_db / (ms * 1e-3) / 1e9 * (1.0 + CHUNK_COST * (C - 1))
                cands.append((lane, L, S, rate))
                if verbose:
                    print("m=%d lane=%d L=%d S=%d: %.1f GCUPS (%.1f per processed cell)"
                          % (m, lane, L, S, m * cells_db / (ms * 1e-3) / 1e9, rate))
        best[bin_of(m)] = cands
    name = device_name or torch.cuda.get_device_name()
    return Table(best, name)
