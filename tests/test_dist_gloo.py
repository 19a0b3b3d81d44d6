"""World-size-2 gloo tests of the multi-process path (CPU, no GPU): the
job's time is the slowest rank's, work counts add up, shards cover every
unit exactly once, and a database sharded by length bin and scored per rank
(the oracle standing in for each rank's GPU call) gathers back into exactly
the single-process scores."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1909_00899_gb300 import dist as sdist
    t = sdist.max_over_ranks(10.0 + 5.0 * rank)
    c = sdist.sum_over_ranks(100.0 * (rank + 1))
    dist.barrier()
    out[rank] = (t, c)
    dist.destroy_process_group()


def test_two_rank_reductions():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (15.0, 300.0)


def _shard_worker(rank, world, port, out):
    import numpy as np
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1909_00899_gb300 import dist as sdist
    from paper_1909_00899_gb300 import synth
    w = synth.workload_protein_small(n_db=301)  # every rank draws the same global database
    rng = np.random.default_rng(5)
    queries = [w["query"], synth.residues(rng, 70, 20), synth.residues(rng, 400, 20)]
    ids = sdist.shard_by_length(w["off"], world)[rank]
    sdb, soff = sdist.take(w["db"], w["off"], ids)
    # this rank's scores of its own shard, one row per query
    local = torch.from_numpy(np.stack([oracle.gotoh_batch(q, sdb, soff, w["M"], w["o"], w["e"])
                                       for q in queries]).astype(np.int32))
    full = sdist.gather_scores(local, ids, len(w["off"]) - 1)
    out[rank] = (len(ids), full.numpy().tolist())
    dist.destroy_process_group()


def test_sharded_database_gathers_to_single_process_scores():
    import numpy as np

    import oracle
    from paper_1909_00899_gb300 import synth
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    w = synth.workload_protein_small(n_db=301)
    rng = np.random.default_rng(5)
    queries = [w["query"], synth.residues(rng, 70, 20), synth.residues(rng, 400, 20)]
    want = np.stack([oracle.gotoh_batch(q, w["db"], w["off"], w["M"], w["o"], w["e"]) for q in queries])
    assert res[0][0] + res[1][0] == 301 and min(res[0][0], res[1][0]) > 100
    for r in range(world):
        np.testing.assert_array_equal(np.array(res[r][1]), want)


def test_length_shards_balanced_and_complete():
    """Host logic of the sharding: every sequence on exactly one rank, the
    residues of each length bin split evenly, the bins equal to the device
    order's quarter-octave key."""
    import numpy as np

    from paper_1909_00899_gb300 import dist as sdist
    from paper_1909_00899_gb300 import synth

    def key(n):  # 1 + 4 floor(log2 n) + the two bits below the leading one
        if n <= 0:
            return 0
        lg = n.bit_length() - 1
        return 1 + 4 * lg + (((n >> (lg - 2)) & 3) if lg >= 2 else 0)

    vals = np.array(list(range(0, 3000)) + [(1 << k) + d for k in range(2, 40) for d in (-1, 0, 1)], np.int64)
    assert [int(x) for x in sdist.length_bins(vals)] == [key(int(v)) for v in vals]
    rng = np.random.default_rng(11)
    db, off = synth.random_db(rng, 20000, 20, "lognormal", median=300, sigma=0.76, lo=20, hi=35000)
    lens = np.diff(off)
    bins = sdist.length_bins(lens)
    for world in (1, 2, 3, 8):
        shards = sdist.shard_by_length(off, world)
        assert np.array_equal(np.sort(np.concatenate(shards)), np.arange(len(lens)))
        tot = [int(lens[s].sum()) for s in shards]
        assert max(tot) <= min(tot) * 1.03
        for b in np.unique(bins):  # per bin: at most one longest sequence apart
            per = [int(lens[s][bins[s] == b].sum()) for s in shards]
            assert max(per) - min(per) <= int(lens[bins == b].max())
        sdb, soff = sdist.take(db, off, shards[-1])
        for k in (0, len(shards[-1]) // 2, len(shards[-1]) - 1):
            i = shards[-1][k]
            assert np.array_equal(sdb[soff[k]:soff[k + 1]], db[off[i]:off[i + 1]])


def test_shards_cover_units_once():
    from paper_1909_00899_gb300.dist import shard
    for n in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                a, b = shard(n, r, world)
                seen.extend(range(a, b))
            assert seen == list(range(n))


def test_single_process_identity():
    from paper_1909_00899_gb300 import dist as sdist
    assert sdist.max_over_ranks(3.5) == 3.5
    assert sdist.env()[1] >= 1
