"""Many queries against one resident database (ragged batches).

Each query's profile is built with the layout the autotuner picked for its
length (or the built-in automatic one).  When every profile runs on the
split s16x2 lanes (the automatic lane type), the whole batch is one
sw_align_multi call -- one persistent launch per layout bin (single-chunk
queries walk query by query, longer ones (query, chunk) phase by phase),
plus one int32 launch that rescores the few pairs whose packed score
reached the s16 threshold -- captured once into a
CUDA graph and replayed.  Otherwise every query's sw_align_db call is
captured instead, spread over side streams.  Scores land in a
[n_queries, n_db] int32 device matrix.
"""
import numpy as np

from . import autotune, sw


class BatchAligner:
    """mode: "multi" (one batched launch per layout; the default), or
    "per_query" (one sw_align_db per query, spread round-robin over
    `streams` side streams that fork from and join back into the aligner's
    stream).  "multi" falls back to "per_query" when a profile cannot join
    the batched launch (another lane type, or gap costs beyond its packed
    lanes)."""

    def __init__(self, db, M, o, e, lane=sw.SW_LANE_AUTO, table=None, stream=None, streams=4, mode="multi",
                 items_per_group=0):
        import torch
        self.db = db
        self.M = np.ascontiguousarray(M, dtype=np.int8)
        self.o, self.e = int(o), int(e)
        self.lane = lane
        self.table = table
        self.stream = stream or torch.cuda.Stream()
        self.side = [torch.cuda.Stream() for _ in range(max(1, streams))]
        self.mode = mode
        self.items_per_group = int(items_per_group)  # > 0: fused-chunk tiles of that many sequences per lane group
        self.graph = None
        self.profiles = []
        self.order = None
        self.multi = None

    def _profile(self, q):
        plan = self.table.plan(len(q)) if self.table is not None else None
        if plan is not None:
            lane, L, S = plan
            if not (self.mode == "multi" and lane == sw.SW_LANE_I16X2Q and L < 16):
                return sw.Profile(q, self.M, lane, stream=self.stream, lanes=L, seg_len=S)
        return sw.Profile(q, self.M, self.lane, stream=self.stream)

    def prepare(self, queries, out):
        """Builds the profiles (length-binned order, longest bin first) and
        captures the alignment of every query into one CUDA graph."""
        import torch
        n = len(queries)
        assert out.shape == (n, self.db.n) and out.dtype == torch.int32 and out.is_cuda
        lens = np.array([len(q) for q in queries])
        self.order = sorted(range(n), key=lambda i: (-autotune.bin_of(int(lens[i])), -int(lens[i])))
        self.profiles = [None] * n
        for i in self.order:
            self.profiles[i] = self._profile(queries[i])
        self.stream.synchronize()  # profiles are built on self.stream
        self.out = out
        # one eager pass: sets kernel attributes, warms the memory pool and
        # (batched) checks the gap costs against the packed lanes
        if self.mode == "multi":
            try:
                self.multi = sw.Multi(self.profiles, self.db, stream=self.stream,
                                      items_per_group=self.items_per_group)
                with torch.cuda.stream(self.stream):
                    self._enqueue()
            except sw.SwError:
                if self.multi is not None:
                    self.multi.free()
                self.multi = None
                self.mode = "per_query"
        if self.multi is None:
            with torch.cuda.stream(self.stream):
                self._enqueue()
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream, capture_error_mode="thread_local"):
            self._enqueue()
        self.graph = g
        return self

    def _enqueue(self):
        import torch
        if self.multi is not None:
            sw.sw_align_multi(self.multi, self.o, self.e, self.out, stream=self.stream)
            return
        fork = torch.cuda.Event()
        fork.record(self.stream)
        for st in self.side:
            st.wait_event(fork)
        for n, i in enumerate(self.order):
            st = self.side[n % len(self.side)]
            sw.sw_align_db(self.profiles[i], self.db, self.o, self.e, self.out[i], stream=st)
        for st in self.side:
            j = torch.cuda.Event()
            j.record(st)
            self.stream.wait_event(j)

    def layouts(self):
        """The launch bins of the batched mode: distinct (virtual lanes,
        segment length, one chunk or several) of the batch's profiles; a
        replay issues one launch per bin plus at most three int32 launches."""
        return sorted({(p.plan()["lanes"], p.plan()["seg_len"], p.plan()["chunks"] == 1)
                       for p in self.profiles if p.qlen > 0})

    def run(self):
        """Replays the captured graph on the aligner's stream."""
        import torch
        with torch.cuda.stream(self.stream):
            self.graph.replay()
        return self.out

    def run_eager(self):
        import torch
        with torch.cuda.stream(self.stream):
            self._enqueue()
        return self.out

    def free(self):
        if self.multi is not None:
            self.multi.free()
            self.multi = None
        for p in self.profiles:
            if p is not None:
                p.free()
        self.profiles = []
        self.graph = None
