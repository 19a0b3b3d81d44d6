#!/usr/bin/env python
"""Benchmark: scan-F striped Smith-Waterman/Gotoh on GB300.

Workload (one step): protein queries of lengths 128, 512, 2048 and 5000
against 100,000 database sequences with log-normal lengths (median 300,
sigma 0.76, clipped to [20, 35000], ~40M residues), seeded 20x20 matrix,
gap open 11, extend 1.  Every step builds the four query profiles and runs
sw_align_batch for each query; the lazy-F kernel runs the same step for the
comparison.  Metric: GCUPS = sum over alignments of m*n / seconds / 1e9.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  Under torchrun (N ranks) the database is N x
100,000 sequences drawn the same way, sharded by length bin so that every
rank holds 100,000 sequences with the same length profile (weak scaling);
each rank aligns the queries against its own shard with no collective while
aligning, the time is the max over ranks, and the score slices are gathered
once after the timed region for the oracle spot check.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

QLENS = (128, 512, 2048, 5000)
# DRAM bytes (read + write) of one launch of the dominant kernel, from one ncu
# capture of that launch; None while the kernel has changed since then.
NCU_TRAFFIC = {"bytes_per_launch": 51.398656e6 + 268.339968e6,
               "kernel": "sw_split_kernel<16, 40, true, false, false, false, true>",
               "launch": "m=5000 chunk 0 vs 100k sequences (ncu --set full)"}
METRIC = "GCUPS scan-F (bit-exact) vs lazy-F"
PROBE_ITERS = 1 << 19  # plain-pass probe: about 0.5 s on every SM
WORKLOAD = ("protein queries m in {128,512,2048,5000} vs 100k db seqs, log-normal lengths "
            "(median 300, sigma 0.76, clip [20,35000]), o=11 e=1")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lane", default="auto", choices=["auto", "i32", "i16x2", "i16x2q", "i8x4"])
    ap.add_argument("--n-db", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-lazyf", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU work of the oracle baseline sample")
    ap.add_argument("--qlens", default=",".join(map(str, QLENS)),
                    help="comma-separated query lengths (profiling cases)")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps and the probe only: no oracle check, lazy-F, e2e, other workloads or "
                         "CPU baseline")
    ap.add_argument("--workload", default="scale", choices=["scale", "pairs", "ragged", "serve", "width", "ends"],
                    help="scale: the default line; pairs/ragged/serve: the other workloads")
    ap.add_argument("--n-pairs", type=int, default=1_000_000)
    ap.add_argument("--n-queries", type=int, default=64, help="ragged: queries taken from the 10,000")
    ap.add_argument("--serve-db", type=int, default=1_000_000)
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--no-extras", action="store_true",
                    help="default line without the reads, ragged and serving sub-keys")
    ap.add_argument("--extras-queries", type=int, default=256,
                    help="ragged sub-key: queries taken from the 10,000")
    ap.add_argument("--extras-requests", type=int, default=120,
                    help="serving sub-key: requests per load")
    ap.add_argument("--streams", type=int, default=4,
                    help="CUDA streams the independent queries of a step are spread over")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def cpu_baseline_oracle(w, qlens, target_s, extras=True):
    """The oracle (scalar int32 Gotoh, all host cores) on a bounded sample of
    the same workload: every query against every k-th database sequence.
    extras: also one core, and the oracle's striped variants (informative)."""
    import numpy as np

    import oracle
    cores = len(os.sched_getaffinity(0))
    off = w["off"]
    n = len(off) - 1
    lens = np.diff(off)
    # calibrate on a small slice, then size the sample for ~target_s seconds
    probe_ids = np.arange(0, n, max(1, n // 200))
    t0 = time.perf_counter()
    cells = 0
    for q in w["queries"]:
        sub_db, sub_off = _subset(w["db"], off, probe_ids)
        oracle.gotoh_batch(q, sub_db, sub_off, w["M"], w["o"], w["e"], nthreads=cores)
        cells += len(q) * int(lens[probe_ids].sum())
    rate = cells / max(time.perf_counter() - t0, 1e-6)
    full_cells = sum(qlens) * int(lens.sum())
    frac = min(1.0, target_s * rate / full_cells)
    step = max(1, int(round(1.0 / frac)))
    ids = np.arange(0, n, step)
    sub_db, sub_off = _subset(w["db"], off, ids)
    t0 = time.perf_counter()
    cells = 0
    for q in w["queries"]:
        oracle.gotoh_batch(q, sub_db, sub_off, w["M"], w["o"], w["e"], nthreads=cores)
        cells += len(q) * int(lens[ids].sum())
    dt = time.perf_counter() - t0
    base = {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
            "sample": "all %d queries vs every %d-th db sequence (%d seqs, %.3g cells, %.1f s)"
                      % (len(w["queries"]), step, len(ids), cells, dt)}
    if not extras:
        return base
    # one core on a slice of the same sample
    ids1 = ids[:: max(1, cores)]
    sub1, off1 = _subset(w["db"], off, ids1)
    t1 = time.perf_counter()
    cells1 = 0
    for q in w["queries"]:
        oracle.gotoh_batch(q, sub1, off1, w["M"], w["o"], w["e"], nthreads=1)
        cells1 += len(q) * int(lens[ids1].sum())
    dt1 = time.perf_counter() - t1
    # the CPU striped variants (informative): Alg. 6 scan and Alg. 1 lazy-F
    # with p = 8 lanes, one thread, the second query against a few sequences
    striped = {}
    q = w["queries"][min(1, len(w["queries"]) - 1)]
    for name, fn in (("scan", oracle.striped_scan), ("lazyf", oracle.striped_lazyf)):
        t2, c2, k = time.perf_counter(), 0, 0
        while time.perf_counter() - t2 < 1.5 and k < n:
            i = ids[k % len(ids)]
            fn(q, w["db"][off[i]:off[i + 1]], w["M"], w["o"], w["e"], 8)
            c2 += len(q) * int(lens[i])
            k += 1
        striped[name] = c2 / (time.perf_counter() - t2) / 1e9
    return dict(base, **{
            "single_core": {"value": cells1 / dt1 / 1e9, "unit": "GCUPS", "cores": 1,
                            "sample": "every %d-th of those sequences" % max(1, cores)},
            "striped_p8_one_core": {"scan_gcups": striped["scan"], "lazyf_gcups": striped["lazyf"],
                                    "sample": "query m=%d vs the first sampled sequences, ~1.5 s each" % len(q)}})


def _subset(db, off, ids):
    import numpy as np
    parts = [db[off[i]:off[i + 1]] for i in ids]
    sub_off = np.zeros(len(ids) + 1, dtype=np.int64)
    np.cumsum([len(p) for p in parts], out=sub_off[1:])
    return np.concatenate(parts).astype(np.uint8), sub_off


def run_reference(args):
    """The reference arm: the oracle as it stands on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1909_00899_gb300 import synth
    w = synth.workload_protein_scale(n_db=args.n_db, qlens=QLENS)
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline_oracle(w, QLENS, per_step, extras=False)
        if k >= args.warmup:
            vals.append(cb)
    v = statistics.median([c["value"] for c in vals])
    workload = WORKLOAD
    if world > 1:  # the same description as the sharded GPU arm's
        workload += (", %d ranks: a database of %d sequences sharded by length bin, %d per rank"
                     % (world, args.n_db * world, args.n_db))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GCUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload, "l2": "n/a (host)"},
            "cpu_baseline": {"kind": "oracle", "cores": vals[-1]["cores"], "sample": vals[-1]["sample"],
                             "value": v, "unit": "GCUPS"},
            "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "scale":
        from paper_1909_00899_gb300 import build as libbuild
        libbuild.build()
        {"pairs": run_pairs, "ragged": run_ragged, "serve": run_serve, "width": run_width,
         "ends": run_ends}[args.workload](args)
        return
    import numpy as np
    import torch
    import torch.distributed

    from paper_1909_00899_gb300 import build as libbuild
    from paper_1909_00899_gb300 import dist, sw, synth

    global QLENS
    QLENS = tuple(int(x) for x in args.qlens.split(","))
    if args.quick:
        args.no_cpu_baseline = True
        args.no_lazyf = True
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
        if rank == 0:  # one build; the other ranks load what it made
            libbuild.build()
        torch.distributed.barrier()
    libbuild.build()
    lane = {"auto": sw.SW_LANE_AUTO, "i32": sw.SW_LANE_I32, "i16x2": sw.SW_LANE_I16X2,
            "i16x2q": sw.SW_LANE_I16X2Q, "i8x4": sw.SW_LANE_I8X4}[args.lane]

    # the global database: n_db sequences per rank; each rank keeps its
    # length-balanced shard (all of it on one GPU)
    wg = synth.workload_protein_scale(n_db=args.n_db * world, qlens=QLENS)
    shard_ids = None
    w = wg
    if world > 1:
        shard_ids = dist.shard_by_length(wg["off"], world)[rank]
        sdb, soff = dist.take(wg["db"], wg["off"], shard_ids)
        w = dict(wg, db=sdb, off=soff)
    M, o, e = w["M"], w["o"], w["e"]
    workload = WORKLOAD if (QLENS, args.n_db) == ((128, 512, 2048, 5000), 100_000) else (
        "protein queries m in {%s} vs %d db seqs, log-normal lengths (median 300, sigma 0.76, "
        "clip [20,35000]), o=11 e=1" % (",".join(map(str, QLENS)), args.n_db))
    if world > 1:
        workload += (", %d ranks: a database of %d sequences sharded by length bin, %d per rank"
                     % (world, args.n_db * world, args.n_db))
    n_db = len(w["off"]) - 1
    total_res = int(w["off"][-1])
    cells_step = sum(QLENS) * total_res  # this rank's cells per step
    cells_all = sum(QLENS) * int(wg["off"][-1])  # every rank's
    stream = torch.cuda.current_stream()
    db_d = torch.from_numpy(w["db"]).cuda()
    off_d = torch.from_numpy(w["off"]).cuda()
    outs = [torch.zeros(n_db, dtype=torch.int32, device="cuda") for _ in QLENS]
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    side = [torch.cuda.Stream() for _ in range(max(1, args.streams))]

    def lazy_lane(lazy):
        return {"s16x2": sw.SW_LANE_I16X2, "s16x2_split": sw.SW_LANE_I16X2Q}.get(lazy, sw.SW_LANE_I32)

    def step(lazy=False, scan_lane=None):
        """One pass of the path: every query's profile and its alignment
        against the whole db; the independent queries are spread over the
        side streams and joined back into the current stream.  lazy: False
        (scan-F), "int32", "s16x2" or "s16x2_split" (lazy-F on that lane
        type); scan_lane: the scan-F lane type instead of --lane."""
        fork = torch.cuda.Event()
        fork.record(stream)
        profs = []
        for i, q in enumerate(w["queries"]):
            st = side[i % len(side)]
            st.wait_event(fork)
            p = sw.Profile(q, M, lazy_lane(lazy) if lazy else (lane if scan_lane is None else scan_lane), stream=st)
            fn = sw.sw_align_lazyf_batch if lazy else sw.sw_align_batch
            fn(p, db_d, off_d, o, e, outs[i], stream=st)
            profs.append(p)
        for st in side:
            j = torch.cuda.Event()
            j.record(st)
            stream.wait_event(j)
        return profs

    step_ms = []  # this rank's per-step times of the last timed() call

    def timed(nsteps, lazy=False, scan_lane=None):
        for _ in range(args.warmup):
            step(lazy, scan_lane)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        total_ms = 0.0
        keep = []
        for _ in range(nsteps):
            flush.zero_()  # L2 flush between timed steps (the db is 40 MB < 129 MB L2)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            profs = step(lazy, scan_lane)
            b.record(stream)
            keep.append((profs, a, b))
        torch.cuda.synchronize()
        step_ms.clear()
        for _, a, b in keep:
            step_ms.append(a.elapsed_time(b))
            total_ms += step_ms[-1]
        if world > 1:
            total_ms = dist.max_over_ranks(total_ms, device="cuda")
        return total_ms

    def per_query(lazy=False, scan_lane=None):
        """Each query's alignment call alone on the current stream, timed
        with CUDA events on that stream (the dominant kernel's launches)."""
        ms = []
        for q, out in zip(w["queries"], outs):
            p = sw.Profile(q, M, lazy_lane(lazy) if lazy else (lane if scan_lane is None else scan_lane), stream=stream)
            torch.cuda.synchronize()
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            (sw.sw_align_lazyf_batch if lazy else sw.sw_align_batch)(p, db_d, off_d, o, e, out, stream=stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            p.free()
        return ms

    # correctness spot check against the oracle on a sample (not timed)
    check = None if args.quick else sample_check(wg, outs, step, rank, shard_ids)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    total_ms = timed(args.steps)
    clocks = sampler.stop()
    own_ms = sum(step_ms)  # this rank's own time (total_ms is the max over ranks)
    gcups = cells_all * args.steps / (total_ms * 1e-3) / 1e9
    median_ms = float(np.median(step_ms))
    if world > 1:
        median_ms = dist.max_over_ranks(median_ms, device="cuda")
    per_q = per_query()

    lazy = None
    scan_i32 = None
    if not args.no_lazyf:
        lsteps = max(1, min(args.steps, 2))
        by_lane = {}
        for lz in ("int32", "s16x2", "s16x2_split"):
            lms = timed(lsteps, lazy=lz)
            lper = per_query(lazy=lz)
            by_lane[lz] = {"value": cells_step * lsteps / (lms * 1e-3) / 1e9, "unit": "GCUPS",
                           "per_query_gcups": {str(m): m * total_res / (t * 1e-3) / 1e9
                                               for m, t in zip(QLENS, lper)}}
        # the comparison uses the faster lazy-F, lane type by lane type per query
        best = max(by_lane, key=lambda k: by_lane[k]["value"])
        lazy = dict(by_lane[best])
        lazy["lane"] = best
        lazy["per_query_gcups"] = {str(m): max(by_lane[k]["per_query_gcups"][str(m)] for k in by_lane)
                                   for m in QLENS}
        lazy["by_lane"] = by_lane
        # scan-F on int32 lanes too: the plain method, method against method
        # on the same lane type
        ims = timed(lsteps, scan_lane=sw.SW_LANE_I32)
        iper = per_query(scan_lane=sw.SW_LANE_I32)
        scan_i32 = {"value": cells_step * lsteps / (ims * 1e-3) / 1e9, "unit": "GCUPS",
                    "per_query_gcups": {str(m): m * total_res / (t * 1e-3) / 1e9 for m, t in zip(QLENS, iper)}}
        scan_i32["vs_lazyf_int32"] = scan_i32["value"] / by_lane["int32"]["value"]

    # end to end through the public API: host (pinned) inputs copied in,
    # scores copied out, inside the timed region
    e2e = None if args.quick else run_e2e(w, lane, args, stream, cells_step)
    if e2e is not None and world > 1:
        # every rank copied and aligned its own shard: the job's time is the
        # slowest rank's, its cells every rank's
        e2e_ms = dist.max_over_ranks(e2e["ms"], device="cuda")
        e2e["value"] = cells_all * e2e["steps"] / (e2e_ms * 1e-3) / 1e9
        e2e["h2d_bytes_per_step"] = int(dist.sum_over_ranks(e2e["h2d_bytes_per_step"], device="cuda"))
        e2e["d2h_bytes_per_step"] = int(dist.sum_over_ranks(e2e["d2h_bytes_per_step"], device="cuda"))
        e2e["ms"] = e2e_ms

    # roofline of the dominant kernel: the longest query's call is its
    # chunk launches (plus a profile build, the length order, the overflow
    # flag and the int32 rescore, together below 0.2 % of the launch time),
    # so its m*n over the call's event-timed duration is the kernel's cell
    # rate; the rate over every query's call is reported beside it
    plans = []
    launches_per_step = 0
    for m in QLENS:
        pf = sw.Profile(np.zeros(m, np.uint8), M, lane)
        pl = pf.plan()
        pf.free()
        pf32 = sw.Profile(np.zeros(m, np.uint8), M, sw.SW_LANE_I32)
        pl32 = pf32.plan()
        pf32.free()
        plans.append(pl)
        packed = pl["lane_type"] != sw.SW_LANE_I32
        # profile build (+ its int32 twin), 3 order kernels, one launch per
        # chunk, then for packed lanes the flag kernel and the int32 rescore;
        # a short one-chunk query also plans the windows of long sequences
        # (the library's rule: pieces of max(2 span, 2048) <= 8192 columns)
        span = m + (m * int(M.max()) - 1) // e
        windows = (pl["chunks"] == 1 and (not packed or pl32["chunks"] == 1) and e >= 1 and int(M.max()) >= 1
                   and pl["lanes"] * pl["seg_len"] <= 1024 and max(2 * span, 2048) <= 8192)
        launches_per_step += ((2 if packed else 1) + 3 + pl["chunks"] + ((1 + pl32["chunks"]) if packed else 0)
                              + (1 if windows else 0))
    i_dom = QLENS.index(max(QLENS))
    plan = plans[i_dom]
    cells_per_op = {1: 1, 2: 2, 3: 4, 4: 2}[plan["lane_type"]]
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clocks.get("sm_mhz") or 2070.0
    # integer ALU pipe: 16 lanes/clk per SM sub-partition, 4 per SM
    peak_alu = sms * 64 * mhz * 1e6 / (6.0 / cells_per_op) / 1e9
    all_gcups = sum(QLENS) * total_res / (sum(per_q) * 1e-3) / 1e9
    kernel_gcups = QLENS[i_dom] * total_res / (per_q[i_dom] * 1e-3) / 1e9
    d0 = int(M.min()) >= -o
    if plan["lane_type"] == sw.SW_LANE_I16X2Q:
        # template <threads, segment, D0, LAZY, ENDS, PIECES, AC>; the
        # always-corrected pass on the layouts the library runs it on
        ac = d0 and plan["lanes"] >= 16 and plan["seg_len"] not in (12, 20)
        kname = "sw_split_kernel<%d, %d, %s, false, false, false, %s>" % (
            plan["lanes"] // 2, plan["seg_len"], "true" if d0 else "false", "true" if ac else "false")
    else:
        kname = "sw_batch_kernel<lane %d, %d, %d, false, false>" % (plan["lane_type"], plan["lanes"],
                                                                    plan["seg_len"])
    # The roofline's peak: the measured cell rate of the plain pass (the
    # per-cell instruction sequence with no correction, scan, loads or
    # shuffles) on the dominant kernel's lane type across every SM, timed
    # long enough (about 0.5 s) to carry its own clock record.  The
    # correction and scan the method adds count against the kernel, not in
    # the denominator.  The unit-count figure is kept as peak_model.
    psampler = ClockSampler(torch.cuda.current_device())
    psampler.start()
    probe = sw.sw_probe_cell_rate(plan["lane_type"], PROBE_ITERS) / 1e9
    probe_clocks = psampler.stop()
    # informative: the corrected passes' own ceilings (the shorter corrected
    # pass, and the always-corrected pass the long-query kernels run)
    probe_corr = probe_ac = None
    if not args.quick and d0 and plan["lane_type"] != sw.SW_LANE_I8X4:
        probe_corr = sw.sw_probe_cell_rate_pass(plan["lane_type"], 1, PROBE_ITERS // 4) / 1e9
        if plan["lane_type"] == sw.SW_LANE_I16X2Q:
            probe_ac = sw.sw_probe_cell_rate_pass(plan["lane_type"], 2, PROBE_ITERS // 4) / 1e9

    line = {
        "metric": METRIC, "value": gcups, "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "ms_per_step_median": median_ms,
        "value_median_step": cells_all / (median_ms * 1e-3) / 1e9, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "s16x2+int32" if cells_per_op == 2 else
        ("int32" if cells_per_op == 1 else "s8x4+int32"), "data": "synthetic",
        "config": {"workload": workload, "n_db": n_db, "db_residues": total_res,
                   "cells_per_step": cells_step, "lane": args.lane, "plan_longest": plan,
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": ("database sharded by length bin over %d ranks (no collective while "
                                   "aligning; scores gathered once, untimed)" % world) if world > 1
                                  else "single GPU",
                   "db_residues_all_ranks": int(wg["off"][-1]), "cells_per_step_all_ranks": cells_all},
        "per_query_gcups": {str(m): m * total_res / (t * 1e-3) / 1e9 for m, t in zip(QLENS, per_q)},
        "plans": {str(m): p for m, p in zip(QLENS, plans)},
        "streams": args.streams,
        "lazyf": lazy,
        "scan_vs_lazyf": (cells_step * args.steps / (own_ms * 1e-3) / 1e9 / lazy["value"]) if lazy else None,
        "scan_int32": scan_i32,
        "scan_vs_lazyf_per_query": ({str(m): (m * total_res / (t * 1e-3) / 1e9) / lazy["per_query_gcups"][str(m)]
                                     for m, t in zip(QLENS, per_q)} if lazy else None),
        "roofline": {"bound": "alu", "achieved": kernel_gcups, "peak": probe, "unit": "GCUPS",
                     "frac": kernel_gcups / probe, "kernel": kname,
                     "launches_per_call": plan["chunks"], "ms_per_launch": per_q[i_dom] / max(1, plan["chunks"]),
                     "cells_per_launch": QLENS[i_dom] * total_res / max(1, plan["chunks"]),
                     "traffic": NCU_TRAFFIC["bytes_per_launch"] if NCU_TRAFFIC else None,
                     "traffic_basis": NCU_TRAFFIC,
                     "peak_basis": ("measured: sw_probe_cell_rate, the plain-pass cell sequence of lane type %d "
                                    "(h, H - o, X, E, F, running max; no correction, scan, loads or shuffles) on "
                                    "every SM, %d iterations, clocks in probe_clocks" % (plan["lane_type"],
                                                                                       PROBE_ITERS)),
                     "probe_clocks": probe_clocks,
                     "peak_model": peak_alu, "frac_of_model": kernel_gcups / peak_alu,
                     "peak_model_basis": ("unit counts, not a ceiling: %d SMs x 64 int lane-ops/clk (half-rate ALU "
                                          "pipe, 4 x 16 lanes) x %.0f MHz (median sampled) / %g instr per cell "
                                          "(6 per register, all on the ALU pipe; the kernels issue the additions "
                                          "on the FMA pipe, so the measured probe runs above it)"
                                          % (sms, mhz, 6.0 / cells_per_op)),
                     "achieved_basis": ("m*n of the m=%d call (its %d launches of the kernel; profile, order, "
                                        "flag and rescore launches < 0.2 %%) / its CUDA-event time on the "
                                        "launching stream" % (QLENS[i_dom], plan["chunks"])),
                     "achieved_all_queries": all_gcups, "frac_all_queries": all_gcups / probe,
                     "probe_corrected_gcups": probe_corr,
                     "frac_of_probe_corrected": (kernel_gcups / probe_corr) if probe_corr else None,
                     "probe_always_corrected_gcups": probe_ac,
                     "frac_of_probe_always_corrected": (kernel_gcups / probe_ac) if probe_ac else None},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "check": check,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle(w, QLENS, args.cpu_seconds)
    if world == 1 and not args.quick and not args.no_extras:
        # the other workloads, each with its own clock record and an oracle
        # spot check: reads vs windows with the lazy-F worst case, the
        # ragged batch, serving
        # (a failure in one is recorded under its key; the scale step's
        # numbers above stand and the line is still printed)
        del outs, db_d, off_d, flush
        torch.cuda.empty_cache()
        try:
            pl = pairs_summary(args, cpu=False)
            line["gap_adversary"] = pl.pop("gap_adversary")
            line["pairs"] = pl
        except Exception as ex:  # noqa: BLE001 -- reported in the line
            line["pairs"] = line["gap_adversary"] = {"error": "%s: %s" % (type(ex).__name__, ex)}
        for key, fn in (("ragged", lambda: ragged_summary(args, args.extras_queries)),
                        ("serving", lambda: serving_summary(args, args.extras_requests))):
            torch.cuda.empty_cache()
            try:
                line[key] = fn()
            except Exception as ex:  # noqa: BLE001 -- reported in the line
                line[key] = {"error": "%s: %s" % (type(ex).__name__, ex)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def sample_check(w, outs, step, rank, shard_ids=None):
    """Scores of a sample of sequences, per query, against the oracle.  w is
    the global database; with shards, every rank's score slices are first
    gathered into its order (the one collective of the data path)."""
    import numpy as np
    import torch

    import oracle
    from paper_1909_00899_gb300 import dist
    profs = step()
    torch.cuda.synchronize()
    del profs
    n = len(w["off"]) - 1
    if shard_ids is not None:
        full = dist.gather_scores(torch.stack(outs), shard_ids, n).cpu().numpy()
    else:
        full = torch.stack(outs).cpu().numpy()
    if rank != 0:
        return None
    rng = np.random.default_rng(7)
    ids = np.sort(rng.choice(n, size=min(n, 64), replace=False))
    sub_db, sub_off = _subset(w["db"], w["off"], ids)
    bad = 0
    for k, q in enumerate(w["queries"]):
        want = oracle.gotoh_batch(q, sub_db, sub_off, w["M"], w["o"], w["e"])
        bad += int((full[k][ids] != want).sum())
    if bad:
        raise SystemExit("bench: %d sampled scores differ from the oracle" % bad)
    return {"sampled": int(len(ids)) * len(w["queries"]), "mismatches": 0,
            "gathered_from_ranks": 1 if shard_ids is None else int(torch.distributed.get_world_size())}


def run_e2e(w, lane, args, stream, cells_step):
    """Same step through the public API from host buffers: the pinned db and
    offsets are copied in, every query is profiled from host memory and
    aligned, and its scores are copied back to pinned host memory, all inside
    the timed region."""
    import torch

    from paper_1909_00899_gb300 import sw
    db_h = torch.from_numpy(w["db"]).pin_memory()
    off_h = torch.from_numpy(w["off"]).pin_memory()
    n_db = len(w["off"]) - 1
    out_h = [torch.empty(n_db, dtype=torch.int32).pin_memory() for _ in QLENS]
    db_d = torch.empty_like(db_h, device="cuda")
    off_d = torch.empty_like(off_h, device="cuda")
    outs = [torch.empty(n_db, dtype=torch.int32, device="cuda") for _ in QLENS]
    side = [torch.cuda.Stream() for _ in range(max(1, args.streams))]

    def one():
        db_d.copy_(db_h, non_blocking=True)
        off_d.copy_(off_h, non_blocking=True)
        fork = torch.cuda.Event()
        fork.record(stream)
        profs = []
        for i, q in enumerate(w["queries"]):
            st = side[i % len(side)]
            st.wait_event(fork)
            p = sw.Profile(q, w["M"], lane, stream=st)
            sw.sw_align_batch(p, db_d, off_d, w["o"], w["e"], outs[i], stream=st)
            with torch.cuda.stream(st):
                out_h[i].copy_(outs[i], non_blocking=True)
            profs.append(p)
        for st in side:
            j = torch.cuda.Event()
            j.record(st)
            stream.wait_event(j)
        return profs

    for _ in range(max(1, args.warmup)):
        one()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 3))
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    keep = [one() for _ in range(steps)]
    b.record(stream)
    torch.cuda.synchronize()
    del keep
    ms = a.elapsed_time(b)
    h2d = db_h.numel() + off_h.numel() * 8 + sum(len(q) for q in w["queries"]) + 400 * 2 * len(QLENS)
    d2h = 4 * n_db * len(QLENS)
    return {"value": cells_step * steps / (ms * 1e-3) / 1e9, "unit": "GCUPS", "ms": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": steps}


# ---------------------------------------------------------------------------
# other workloads (each prints its own JSON line; the default line above is
# the scale workload)
# ---------------------------------------------------------------------------

def _events_ms(fn, stream, reps=1):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def run_pairs(args):
    """DNA reads against their own 2 kbp reference windows (1M pairs): one
    JSON line."""
    print(json.dumps(pairs_summary(args, cpu=not args.no_cpu_baseline)), flush=True)


def pairs_summary(args, cpu=True):
    """DNA reads against their own 2 kbp reference windows (1M pairs): scan-F
    on every lane type, end cells, lazy-F and its corrective factor per read
    class, and the synthetic lazy-F worst case (query X+Y+Z vs reference
    X+Z); sampled scores checked against the oracle.  The clocks are sampled
    over the whole GPU part."""
    import numpy as np
    import torch

    import oracle
    from paper_1909_00899_gb300 import sw, synth
    w = synth.workload_reads(n_pairs=args.n_pairs)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    n = len(w["q_off"]) - 1
    qlen = np.diff(w["q_off"])
    rlen = np.diff(w["r_off"])
    cells = float((qlen * rlen).sum())
    st = torch.cuda.current_stream()
    qd = torch.from_numpy(w["q"]).cuda()
    qo = torch.from_numpy(w["q_off"]).cuda()
    rd = torch.from_numpy(w["r"]).cuda()
    ro = torch.from_numpy(w["r_off"]).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    res = {}
    for name, lane in (("s16x2_split", sw.SW_LANE_I16X2Q), ("s16x2", sw.SW_LANE_I16X2), ("s8x4", sw.SW_LANE_I8X4),
                       ("int32", sw.SW_LANE_I32)):
        fn = lambda: sw.sw_align_pairs(qd, qo, rd, ro, w["M"], w["o"], w["e"], out, lane_type=lane, stream=st)
        for _ in range(args.warmup):
            fn()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            ms.append(_events_ms(fn, st))
        res[name] = {"gcups": cells / (np.mean(ms) * 1e-3) / 1e9, "ms": float(np.mean(ms))}
        if name == "s8x4":
            s = out.cpu().numpy()
            res[name]["flagged_fraction_per_class"] = {
                k: float((s[w["kinds"] == c] >= 127 - 1).mean()) for k, c in
                (("copy95", 0), ("deletion", 1), ("insertion", 2), ("copy99", 3))}
    # end cells (what mate rescue places a read by), automatic lane
    qe_t = torch.empty(n, dtype=torch.int32, device="cuda")
    re_t = torch.empty(n, dtype=torch.int32, device="cuda")
    fe = lambda: sw.sw_align_pairs_ends(qd, qo, rd, ro, w["M"], w["o"], w["e"], out, qe_t, re_t, stream=st)
    for _ in range(args.warmup):
        fe()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        ms.append(_events_ms(fe, st))
    ends = {"gcups": cells / (np.mean(ms) * 1e-3) / 1e9, "ms": float(np.mean(ms))}
    ids_e = np.sort(np.random.default_rng(4).choice(n, size=min(n, 2000), replace=False))
    sbe = _pairs_subset(w, ids_e)
    we = oracle.gotoh_end_pairs(sbe["q"], sbe["q_off"], sbe["r"], sbe["r_off"], w["M"], w["o"], w["e"])
    got_e = (out.cpu().numpy()[ids_e], qe_t.cpu().numpy()[ids_e], re_t.cpu().numpy()[ids_e])
    if not all(np.array_equal(a, b) for a, b in zip(got_e, we)):
        raise SystemExit("pairs: sampled end cells differ from the oracle")
    ends["check"] = {"sampled": int(ids_e.size), "mismatches": 0}
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    lz = lambda: sw.sw_align_lazyf_pairs(qd, qo, rd, ro, w["M"], w["o"], w["e"], out, lazy_steps=steps, stream=st)
    lz()
    steps.zero_()
    flush.zero_()
    lms = _events_ms(lz, st)
    lazy = {"gcups": cells / (lms * 1e-3) / 1e9, "ms": lms, "lane": "int32",
            "C_factor": float(steps.item()) * 32 / cells}
    # lazy-F on the split s16x2 layout too (the layout scan-F runs on); the
    # comparison takes the faster lazy-F
    lzq = lambda: sw.sw_align_lazyf_pairs(qd, qo, rd, ro, w["M"], w["o"], w["e"], out, stream=st,
                                          lane_type=sw.SW_LANE_I16X2Q)
    lzq()
    flush.zero_()
    lqms = _events_ms(lzq, st)
    lazy_split = {"gcups": cells / (lqms * 1e-3) / 1e9, "ms": lqms, "lane": "s16x2_split"}
    lazy_int32 = lazy
    if lqms < lms:
        lazy = dict(lazy_split, C_factor_int32=lazy_int32["C_factor"])
    # scan-F vs lazy-F and the lazy-F corrective factor C per read class
    per_class = {}
    for cname, c in (("copy95", 0), ("deletion", 1), ("insertion", 2), ("copy99", 3)):
        ids = np.flatnonzero(w["kinds"] == c)
        sub = _pairs_subset(w, ids)
        sq, sqo, sr, sro = (torch.from_numpy(x).cuda() for x in (sub["q"], sub["q_off"], sub["r"], sub["r_off"]))
        so = torch.empty(len(ids), dtype=torch.int32, device="cuda")
        scells = float((np.diff(sub["q_off"]) * np.diff(sub["r_off"])).sum())
        sf = lambda: sw.sw_align_pairs(sq, sqo, sr, sro, w["M"], w["o"], w["e"], so, stream=st)
        sf()
        sms = _events_ms(sf, st, 2)
        steps.zero_()
        lf = lambda: sw.sw_align_lazyf_pairs(sq, sqo, sr, sro, w["M"], w["o"], w["e"], so, lazy_steps=steps,
                                             stream=st)
        lf()
        c_fac = float(steps.item()) * 32 / scells
        lfm = _events_ms(lf, st, 2)
        lq = lambda: sw.sw_align_lazyf_pairs(sq, sqo, sr, sro, w["M"], w["o"], w["e"], so, stream=st,
                                             lane_type=sw.SW_LANE_I16X2Q)
        lq()
        lqm = _events_ms(lq, st, 2)
        per_class[cname] = {"pairs": int(len(ids)), "scan_gcups": scells / (sms * 1e-3) / 1e9,
                            "lazyf_gcups": scells / (min(lfm, lqm) * 1e-3) / 1e9,
                            "lazyf_gcups_by_lane": {"int32": scells / (lfm * 1e-3) / 1e9,
                                                    "s16x2_split": scells / (lqm * 1e-3) / 1e9},
                            "scan_vs_lazyf": min(lfm, lqm) / sms, "lazyf_C_factor_int32": c_fac}
    # the synthetic lazy-F worst case: query = X + Y + Z vs reference = X + Z
    adv = synth.workload_gap_adversary(n_pairs=min(200_000, n))
    aq, aqo, ar, aro = (torch.from_numpy(adv[k]).cuda() for k in ("q", "q_off", "r", "r_off"))
    na = len(adv["q_off"]) - 1
    ao = torch.empty(na, dtype=torch.int32, device="cuda")
    acells = float((np.diff(adv["q_off"]) * np.diff(adv["r_off"])).sum())
    af = lambda: sw.sw_align_pairs(aq, aqo, ar, aro, adv["M"], adv["o"], adv["e"], ao, stream=st)
    af()
    ams = _events_ms(af, st, 2)
    a_got = ao.cpu().numpy()
    steps.zero_()
    al = lambda: sw.sw_align_lazyf_pairs(aq, aqo, ar, aro, adv["M"], adv["o"], adv["e"], ao, lazy_steps=steps,
                                         stream=st)
    al()
    a_c = float(steps.item()) * 32 / acells
    alm = _events_ms(al, st, 2)
    aqz = lambda: sw.sw_align_lazyf_pairs(aq, aqo, ar, aro, adv["M"], adv["o"], adv["e"], ao, stream=st,
                                          lane_type=sw.SW_LANE_I16X2Q)
    aqz()
    aqm = _events_ms(aqz, st, 2)
    a_ids = np.sort(np.random.default_rng(6).choice(na, size=min(na, 1000), replace=False))
    a_sub = _pairs_subset(adv, a_ids)
    a_want = oracle.gotoh_pairs(a_sub["q"], a_sub["q_off"], a_sub["r"], a_sub["r_off"], adv["M"], adv["o"],
                                adv["e"])
    if not np.array_equal(a_got[a_ids], a_want):
        raise SystemExit("pairs: sampled gap-adversary scores differ from the oracle")
    per_class["gap_adversary"] = {"pairs": int(na), "scan_gcups": acells / (ams * 1e-3) / 1e9,
                                  "lazyf_gcups": acells / (min(alm, aqm) * 1e-3) / 1e9,
                                  "lazyf_gcups_by_lane": {"int32": acells / (alm * 1e-3) / 1e9,
                                                          "s16x2_split": acells / (aqm * 1e-3) / 1e9},
                                  "scan_vs_lazyf": min(alm, aqm) / ams, "lazyf_C_factor_int32": a_c,
                                  "recipe": "query X+Y+Z vs reference X+Z, |X|,|Z| 60..150, |Y| 40..200, "
                                            "DNA +1/-4, o=6 e=1",
                                  "check": {"sampled": int(a_ids.size), "mismatches": 0}}
    worst = max(per_class, key=lambda k: per_class[k]["scan_vs_lazyf"])
    # exactness on a sample, every lane type agreed already in the tests
    sw.sw_align_pairs(qd, qo, rd, ro, w["M"], w["o"], w["e"], out, stream=st)
    got = out.cpu().numpy()
    rng = np.random.default_rng(3)
    sample = np.sort(rng.choice(n, size=min(n, 4000), replace=False))
    sb = _pairs_subset(w, sample)
    want = oracle.gotoh_pairs(sb["q"], sb["q_off"], sb["r"], sb["r_off"], w["M"], w["o"], w["e"])
    if not np.array_equal(got[sample], want):
        raise SystemExit("pairs: sampled scores differ from the oracle")
    clocks = sampler.stop()
    best = max(res.values(), key=lambda r: r["gcups"])
    line = {"metric": "GCUPS reads vs windows (scan-F, bit-exact)", "value": best["gcups"], "unit": "GCUPS",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "data": "synthetic", "config": {"workload": "1M DNA reads (150 bp; 30% 95%-id, 10% 40-200 bp indel, "
                                                        "60% 99%-id) vs own 2 kbp windows, +1/-4, o=6 e=1",
                                            "n_pairs": n, "cells": cells},
            "by_lane": res, "with_end_cells": ends, "lazyf": lazy,
            "lazyf_by_lane": {"int32": lazy_int32, "s16x2_split": lazy_split},
            "scan_vs_lazyf": lazy["ms"] / best["ms"],
            "per_class": per_class, "largest_margin_class": worst,
            "gap_adversary": per_class["gap_adversary"], "clocks": clocks,
            "check": {"sampled": int(sample.size), "mismatches": 0}}
    if cpu:
        # about cpu_seconds of work at ~10 GCUPS on the host cores
        ids = np.arange(0, n, max(1, int(cells / (args.cpu_seconds * 1e10))))
        sb = _pairs_subset(w, ids)
        t0 = time.perf_counter()
        oracle.gotoh_pairs(sb["q"], sb["q_off"], sb["r"], sb["r_off"], w["M"], w["o"], w["e"])
        dt = time.perf_counter() - t0
        c = float((np.diff(sb["q_off"]) * np.diff(sb["r_off"])).sum())
        line["cpu_baseline"] = {"value": c / dt / 1e9, "unit": "GCUPS", "cores": len(os.sched_getaffinity(0)),
                                "kind": "oracle", "sample": "%d of %d pairs (%.3g cells, %.1f s)" % (len(ids), n, c, dt)}
    return line


def run_width(args):
    """Lazy-F against the vector width (the GPU analogue of Fig. 1): int32
    lanes, fixed query lengths, lanes per alignment L = 4, 8, 16, 32 (segment
    length m / L); the lazy-F corrective factor C (correction-loop j-steps
    per main-pass j-step) and GCUPS of lazy-F and scan-F on the same layout."""
    import numpy as np
    import torch

    from paper_1909_00899_gb300 import sw, synth
    torch.cuda.set_device(0)
    w = synth.workload_protein_scale(n_db=args.n_db, qlens=(128, 256, 512))
    M = w["M"]
    db_d = torch.from_numpy(w["db"]).cuda()
    off_d = torch.from_numpy(w["off"]).cuda()
    h = sw.Database(db_d, off_d)
    st = torch.cuda.current_stream()
    out = torch.empty(h.n, dtype=torch.int32, device="cuda")
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    total = int(w["off"][-1])
    rows = []
    for q, layouts in ((w["queries"][0], ((4, 32), (8, 16), (16, 8))),
                       (w["queries"][1], ((8, 32), (16, 16), (32, 8))),
                       (w["queries"][2], ((16, 32), (32, 16)))):
        cells = len(q) * total
        for L, S in layouts:
            prof = sw.Profile(q, M, sw.SW_LANE_I32, lanes=L, seg_len=S)
            # both methods timed through the same call shape (long sequences
            # split into windows alike); C from the statistics call, which
            # keeps every sequence whole
            scan = lambda: sw.sw_align_db(prof, h, w["o"], w["e"], out, stream=st)
            lazy = lambda: sw.sw_align_lazyf_db(prof, h, w["o"], w["e"], out, stream=st)
            stats = lambda: sw.sw_align_lazyf_db_stats(prof, h, w["o"], w["e"], out, lazy_steps=steps, stream=st)
            scan()
            sms = _events_ms(scan, st, 2)
            steps.zero_()
            stats()
            torch.cuda.synchronize()
            c_fac = float(steps.item()) * 32 / cells
            lazy()
            lms = _events_ms(lazy, st, 2)
            rows.append({"m": len(q), "lanes": L, "seg_len": S, "lazyf_C": c_fac,
                         "scan_gcups": cells / (sms * 1e-3) / 1e9, "lazyf_gcups": cells / (lms * 1e-3) / 1e9,
                         "scan_vs_lazyf": lms / sms})
            prof.free()
    line = {"metric": "lazy-F corrective factor and GCUPS vs lanes per alignment (int32)",
            "value": max(r["scan_vs_lazyf"] for r in rows), "unit": "x (scan-F over lazy-F, best width)",
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "protein queries m=128, 256, 512 vs %d log-normal sequences (%d residues), o=11 e=1"
                                   % (h.n, total)},
            "rows": rows}
    print(json.dumps(line), flush=True)



def run_ends(args):
    """Cost of end cells: scores only (automatic layout and int32) against
    scores with end cells (int32), one query at a time against the scale
    database."""
    import numpy as np
    import torch

    from paper_1909_00899_gb300 import sw, synth
    torch.cuda.set_device(0)
    w = synth.workload_protein_scale(n_db=args.n_db, qlens=(512, 2048))
    M = w["M"]
    db_d = torch.from_numpy(w["db"]).cuda()
    off_d = torch.from_numpy(w["off"]).cuda()
    n = len(w["off"]) - 1
    total = int(w["off"][-1])
    st = torch.cuda.current_stream()
    sc = torch.empty(n, dtype=torch.int32, device="cuda")
    qe = torch.empty(n, dtype=torch.int32, device="cuda")
    re_ = torch.empty(n, dtype=torch.int32, device="cuda")
    rows = []
    for q in w["queries"]:
        cells = len(q) * total
        pa = sw.Profile(q, M)
        p32 = sw.Profile(q, M, sw.SW_LANE_I32)
        fa = lambda: sw.sw_align_batch(pa, db_d, off_d, w["o"], w["e"], sc, stream=st)
        fae = lambda: sw.sw_align_batch_ends(pa, db_d, off_d, w["o"], w["e"], sc, qe, re_, stream=st)
        f32 = lambda: sw.sw_align_batch(p32, db_d, off_d, w["o"], w["e"], sc, stream=st)
        fe = lambda: sw.sw_align_batch_ends(p32, db_d, off_d, w["o"], w["e"], sc, qe, re_, stream=st)
        row = {"m": len(q)}
        for name, f in (("auto", fa), ("auto_ends", fae), ("int32", f32), ("int32_ends", fe)):
            f()
            row[name + "_gcups"] = cells / (_events_ms(f, st, 2) * 1e-3) / 1e9
        rows.append(row)
        pa.free()
        p32.free()
    line = {"metric": "GCUPS with end cells vs scores only", "value": rows[-1]["auto_ends_gcups"],
            "unit": "GCUPS", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "protein queries m=512, 2048 vs %d log-normal sequences, o=11 e=1" % n},
            "rows": rows}
    print(json.dumps(line), flush=True)


def _pairs_subset(w, ids):
    import numpy as np
    q = [w["q"][w["q_off"][i]:w["q_off"][i + 1]] for i in ids]
    r = [w["r"][w["r_off"][i]:w["r_off"][i + 1]] for i in ids]
    qo = np.zeros(len(ids) + 1, np.int64)
    ro = np.zeros(len(ids) + 1, np.int64)
    np.cumsum([len(x) for x in q], out=qo[1:])
    np.cumsum([len(x) for x in r], out=ro[1:])
    return {"q": np.concatenate(q).astype(np.uint8), "q_off": qo,
            "r": np.concatenate(r).astype(np.uint8), "r_off": ro}


def run_ragged(args):
    print(json.dumps(ragged_summary(args, args.n_queries)), flush=True)


def ragged_summary(args, n_queries):
    """Ragged batch: a deterministic, length-stratified subset of 10,000
    protein queries (log-uniform 32..4096) against 200k log-normal sequences,
    every query's alignment captured in one CUDA graph with the autotuned
    layout per length bin."""
    import numpy as np
    import torch

    import oracle
    from paper_1909_00899_gb300 import autotune, sw, synth
    from paper_1909_00899_gb300.batch import BatchAligner
    rng = synth.rng_for(3)
    M = synth.protein_matrix(rng)
    qlens_all = synth.lengths_loguniform(rng, 10_000, 32, 4096)
    db, off = synth.random_db(rng, 200_000, 20, "lognormal", median=300, sigma=0.76, lo=20, hi=35000)
    order = np.argsort(qlens_all, kind="stable")
    pick = order[np.linspace(0, len(order) - 1, n_queries).astype(int)]
    queries = [synth.residues(np.random.default_rng([5, int(i)]), int(qlens_all[i]), 20) for i in pick]
    db_d = torch.from_numpy(db).cuda()
    off_d = torch.from_numpy(off).cuda()
    h = sw.Database(db_d, off_d)
    # autotune against the database itself over the split layouts the
    # batched launch runs, each timed as one batched launch of 4 queries of
    # the bin's length (the batch's own setting: no per-query launch tail)
    table = autotune.tune(h, M, 11, 1, lengths=[48, 100, 200, 400, 800, 1600, 3200], reps=1,
                          lanes=(sw.SW_LANE_I16X2Q,), batched=4)
    out = torch.empty((len(queries), h.n), dtype=torch.int32, device="cuda")
    ba = BatchAligner(h, M, 11, 1, table=table, streams=args.streams).prepare(queries, out)
    st = ba.stream
    layouts = ba.layouts()
    for _ in range(args.warmup):
        ba.run()
    ms = []
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        ba.run()
        b.record(st)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    clocks = sampler.stop()
    total_res = int(off[-1])
    cells = float(sum(len(q) for q in queries)) * total_res
    got = out.cpu().numpy()
    ids = np.random.default_rng(4).choice(h.n, size=300, replace=False)
    sdb, soff = _subset(db, off, ids)
    for k in range(0, len(queries), max(1, len(queries) // 8)):
        want = oracle.gotoh_batch(queries[k], sdb, soff, M, 11, 1)
        if not np.array_equal(got[k][ids], want):
            raise SystemExit("ragged: sampled scores differ from the oracle")
    # launches of one replay: one per layout and, when some pairs could pass
    # the packed lanes' range, one int32 launch per int32 layout
    thresh = 32767 - (4096 + 128 - 11) - int(M.max())
    skip_len = -(-thresh // int(M.max()))
    n_i32 = len({(32, 8) if m <= 256 else (32, 16) if m <= 512 else (32, 32) for m in map(len, queries)
                 if m >= skip_len}) if int(np.diff(off).max()) >= skip_len else 0
    line = {"metric": "GCUPS ragged batch (graph replay, bit-exact)", "value": cells / (np.mean(ms) * 1e-3) / 1e9,
            "unit": "GCUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "data": "synthetic",
            "config": {"workload": "%d of 10,000 protein queries (log-uniform 32..4096, length-stratified) vs "
                                   "200k log-normal sequences (%d residues), o=11 e=1" % (len(queries), total_res),
                       "cells_per_step": cells, "full_config_cells": float(qlens_all.sum()) * total_res},
            "ms_per_step": float(np.mean(ms)),
            "projected_full_config_s": float(qlens_all.sum()) * total_res / (cells / (np.mean(ms) * 1e-3)),
            "autotune": table.to_json(), "clocks": clocks, "check": {"queries_checked": 8, "db_sample": 300},
            "mode": "batched" if ba.multi is not None else "per_query",
            "launches_per_replay": (len(layouts) + n_i32) if ba.multi is not None else None,
            "launch_bins": [{"lanes": x[0], "seg_len": x[1],
                             "kernel": "phase" if x[2] else "fused-chunk" if ba.items_per_group else "chunk-walk"}
                            for x in layouts]}
    ba.free()
    return line


def run_serve(args):
    print(json.dumps(serving_summary(args, args.serve_requests)), flush=True)


def serving_summary(args, n_requests):
    """Serving: Poisson stream of protein queries (log-uniform 50..10,000)
    against a resident database of 1M log-normal sequences (~350M residues),
    admitted by a memory budget; p50/p99 latency at 50% and 90% of the
    closed-loop peak rate."""
    import numpy as np
    import torch

    import oracle
    from paper_1909_00899_gb300 import serve, sw, synth
    rng = synth.rng_for(4)
    M = synth.protein_matrix(rng)
    db, off = synth.random_db(rng, args.serve_db, 20, "lognormal", median=300, sigma=0.555, lo=20, hi=35000)
    db_d = torch.from_numpy(db).cuda()
    off_d = torch.from_numpy(off).cuda()
    h = sw.Database(db_d, off_d)
    total_res = int(off[-1])

    def queries(n, salt):
        r = np.random.default_rng([6, salt])
        lens = synth.lengths_loguniform(r, n, 50, 10_000)
        return [synth.residues(r, int(m), 20) for m in lens]

    budget = 48 << 30
    srv = serve.Server(h, M, 11, 1, slots=4, mem_budget=budget)
    srv.run(queries(4, 0))  # warm-up
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    qs = queries(n_requests, 1)
    t0 = time.perf_counter()
    reqs = srv.run(qs)
    peak_qps = len(qs) / (time.perf_counter() - t0)
    peak_gcups = sum(len(q) for q in qs) * total_res / srv.wall / 1e9
    loads = {}
    for frac in (0.5, 0.9):
        qs2 = queries(n_requests, int(frac * 10))
        arr = serve.poisson_arrivals(np.random.default_rng([7, int(frac * 10)]), len(qs2), frac * peak_qps)
        srv2 = serve.Server(h, M, 11, 1, slots=4, mem_budget=budget)
        r2 = srv2.run(qs2, arr)
        st = serve.latency_stats(r2)
        st["offered_qps"] = frac * peak_qps
        st["achieved_gcups"] = sum(len(q) for q in qs2) * total_res / srv2.wall / 1e9
        loads["%d%%" % int(frac * 100)] = st
        if frac == 0.9:
            ids = np.random.default_rng(8).choice(h.n, size=200, replace=False)
            sdb, soff = _subset(db, off, ids)
            for k in range(0, len(qs2), 20):  # 5% of the requests
                want = oracle.gotoh_batch(qs2[k], sdb, soff, M, 11, 1)
                if not np.array_equal(r2[k].scores[ids], want):
                    raise SystemExit("serve: sampled scores differ from the oracle")
    clocks = sampler.stop()
    line = {"metric": "serving latency p50/p99 and throughput (bit-exact)", "value": peak_gcups, "unit": "GCUPS",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "protein queries log-uniform 50..10000 vs %d resident log-normal sequences "
                                   "(median 300, sigma 0.555, %d residues), o=11 e=1, 4 slots, %d GB budget"
                                   % (h.n, total_res, budget >> 30),
                       "requests_per_load": n_requests},
            "peak_qps": peak_qps, "loads": loads, "clocks": clocks,
            "check": {"requests_checked": "5%", "db_sample": 200}}
    return line


if __name__ == "__main__":
    main()
