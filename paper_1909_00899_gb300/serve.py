"""Serving loop: queries against a database kept resident on the device,
with continuous batching.

Requests arrive over time (for example a Poisson stream).  A request is
admitted as soon as it has arrived, a stream slot is free and the device
memory it needs (its score vector, its profile and, for queries longer than
one chunk, the boundary rows between chunks) fits both the memory budget
next to the requests already running and the memory the device has
available right now (sw_mem_available: free memory plus the idle blocks of
the stream-ordered pool the library allocates from), so other users of the
GPU shrink what the server takes on.  Admitted requests run concurrently on
separate CUDA streams (their kernels overlap on the device); completion is
detected by polling an event, after which the scores are copied to pinned
host memory and the request's memory returns to the budget.  Latency is
completion time minus arrival time on the host clock.

A request's scores do not depend on what runs beside it: every call owns its
scratch, its output and its profile.
"""
import collections
import time

import numpy as np

from . import sw


class Request:
    __slots__ = ("rid", "query", "arrival", "admitted", "done", "scores", "bytes", "slot", "event", "profile")

    def __init__(self, rid, query, arrival):
        self.rid = rid
        self.query = query
        self.arrival = arrival
        self.admitted = None
        self.done = None
        self.scores = None
        self.slot = None


class _Slot:
    """A stream with its own device and pinned host score buffers."""

    def __init__(self, n_db):
        import torch
        self.stream = torch.cuda.Stream()
        self.out_dev = torch.empty(max(n_db, 1), dtype=torch.int32, device="cuda")
        self.out_host = torch.empty(max(n_db, 1), dtype=torch.int32).pin_memory()


class Server:
    def __init__(self, db, M, o, e, lane=sw.SW_LANE_AUTO, table=None, slots=4, mem_budget=8 << 30):
        self.db = db
        self.M = np.ascontiguousarray(M, dtype=np.int8)
        self.o, self.e = int(o), int(e)
        self.lane = lane
        self.table = table
        self.budget = int(mem_budget)
        self.in_use = 0
        self.slots = [_Slot(db.n) for _ in range(slots)]
        self.free_slots = collections.deque(self.slots)
        self.total_residues = int(db.offsets[-1].item())
        self.rejected = 0
        self.waited_for_memory = 0  # admissions deferred because the device lacked the memory

    def request_bytes(self, m):
        """Device memory one request holds while it runs (its slot's score
        buffer is counted too, so the budget bounds the whole footprint)."""
        n = self.db.n
        nbytes = 4 * n + 64 * 1024          # scores, counters and small scratch
        nbytes += 4 * n                     # overflow list of packed lanes
        nbytes += 32 * (m + 512) * 4        # profiles (raw, both plans)
        if m > 256:
            nbytes += 8 * self.total_residues  # boundary rows between chunks
        return nbytes

    def _profile(self, q, stream):
        plan = self.table.plan(len(q)) if self.table is not None else None
        if plan is not None:
            lane, L, S = plan
            return sw.Profile(q, self.M, lane, stream=stream, lanes=L, seg_len=S)
        return sw.Profile(q, self.M, self.lane, stream=stream)

    def _admit(self, req, now):
        import torch
        slot = self.free_slots.popleft()
        req.slot = slot
        req.bytes = self.request_bytes(len(req.query))
        self.in_use += req.bytes
        req.admitted = now
        st = slot.stream
        req.profile = self._profile(req.query, st)
        sw.sw_align_db(req.profile, self.db, self.o, self.e, slot.out_dev, stream=st)
        req.profile.free_async(st)  # stream-ordered: after the alignment
        req.profile = None
        with torch.cuda.stream(st):
            slot.out_host.copy_(slot.out_dev, non_blocking=True)
            req.event = torch.cuda.Event()
            req.event.record(st)

    def _retire(self, req, now):
        req.done = now
        req.scores = req.slot.out_host.numpy()[: self.db.n].copy()
        self.in_use -= req.bytes
        self.free_slots.append(req.slot)
        req.slot = None
        req.event = None

    def run(self, queries, arrivals=None, timeout_s=3600.0):
        """Serves queries[i] arriving at arrivals[i] seconds after start (all
        at 0 when arrivals is None: the closed, saturated loop).  Returns the
        requests with their scores and times."""
        n = len(queries)
        arrivals = np.zeros(n) if arrivals is None else np.asarray(arrivals, dtype=np.float64)
        reqs = [Request(i, queries[i], float(arrivals[i])) for i in range(n)]
        pending = collections.deque(sorted(reqs, key=lambda r: r.arrival))
        running = []
        t0 = time.perf_counter()
        while pending or running:
            now = time.perf_counter() - t0
            if now > timeout_s:
                raise TimeoutError("serving loop exceeded %.0f s" % timeout_s)
            # admit everything that has arrived and fits
            while pending and pending[0].arrival <= now and self.free_slots:
                need = self.request_bytes(len(pending[0].query))
                if need > self.budget:
                    r = pending.popleft()  # can never fit: refuse
                    r.done = now
                    self.rejected += 1
                    continue
                if self.in_use + need > self.budget:
                    break
                if need > sw.sw_mem_available():
                    if not running:  # nothing of ours will free memory: refuse
                        r = pending.popleft()
                        r.done = now
                        self.rejected += 1
                        continue
                    self.waited_for_memory += 1
                    break
                r = pending.popleft()
                self._admit(r, now)
                running.append(r)
            # retire what finished
            still = []
            for r in running:
                if r.event.query():
                    self._retire(r, time.perf_counter() - t0)
                else:
                    still.append(r)
            running = still
            if running or (pending and pending[0].arrival > now):
                time.sleep(0.0002)
        self.wall = time.perf_counter() - t0
        return reqs


def latency_stats(reqs):
    lat = np.array([r.done - r.arrival for r in reqs if r.scores is not None])
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "n": 0}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "n": int(lat.size)}


def poisson_arrivals(rng, n, rate):
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
