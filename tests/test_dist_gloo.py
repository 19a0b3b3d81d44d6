"""World-size-2 gloo test of the multi-process helpers (CPU, no GPU): the
job's time is the slowest rank's, work counts add up, shards cover every
unit exactly once."""
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
