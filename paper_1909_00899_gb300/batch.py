"""Many queries against one resident database (ragged batches).

Queries are binned by length; each bin's profiles are built with the layout
the autotuner picked for it (or the built-in one), and the whole set of
sw_align_db calls -- every query, every chunk launch, the overflow flagging
and the int32 rescore -- is captured once into a CUDA graph and replayed.
Scores land in a [n_queries, n_db] int32 device matrix.
"""
import numpy as np

from . import autotune, sw


class BatchAligner:
    """streams: the queries are spread round-robin over this many streams
    that fork from and join back into the aligner's stream (inside the
    graph too), so one query's launch tail overlaps the next query's work."""

    def __init__(self, db, M, o, e, lane=sw.SW_LANE_AUTO, table=None, stream=None, streams=4):
        import torch
        self.db = db
        self.M = np.ascontiguousarray(M, dtype=np.int8)
        self.o, self.e = int(o), int(e)
        self.lane = lane
        self.table = table
        self.stream = stream or torch.cuda.Stream()
        self.side = [torch.cuda.Stream() for _ in range(max(1, streams))]
        self.graph = None
        self.profiles = []
        self.order = None

    def _profile(self, q):
        plan = self.table.plan(len(q)) if self.table is not None else None
        if plan is not None:
            lane, L, S = plan
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
        with torch.cuda.stream(self.stream):
            # one eager pass: sets kernel attributes and warms the memory pool
            self._enqueue()
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream, capture_error_mode="thread_local"):
            self._enqueue()
        self.graph = g
        return self

    def _enqueue(self):
        import torch
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
        for p in self.profiles:
            if p is not None:
                p.free()
        self.profiles = []
        self.graph = None
