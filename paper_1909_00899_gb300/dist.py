"""Multi-process helpers for running the alignment path as one process per
GPU.  Every alignment is independent (the carry scan stays inside a warp),
so the database is sharded across ranks and ranks exchange nothing while
aligning: each rank keeps its shard resident and scores it, the slowest
rank decides the job's time, and the only collective on the data path is
the final gather of the score slices into the database's order."""
import os

import numpy as np


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _initialised():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def max_over_ranks(value, device=None):
    """The largest value over all ranks (the job's time is the slowest
    rank's); identity when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not _initialised():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    import torch
    import torch.distributed as dist
    if not _initialised():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(n, rank, world):
    """Contiguous [start, stop) share of n independent units for one rank."""
    per, rem = divmod(int(n), int(world))
    start = rank * per + min(rank, rem)
    return start, start + per + (1 if rank < rem else 0)


def length_bins(lengths):
    """Quarter-octave length bin of each sequence (0 for empty; else
    1 + 4 floor(log2 n) + the two bits below the leading one), the bins the
    device-side work order groups sequences by."""
    n = np.asarray(lengths, dtype=np.int64)
    out = np.zeros(n.shape, dtype=np.int64)
    pos = n > 0
    v = n[pos]
    lg = np.floor(np.log2(v)).astype(np.int64)
    # exact floor(log2) for large values (float rounding at powers of two)
    lg = np.where((np.int64(1) << lg) > v, lg - 1, lg)
    lg = np.where((np.int64(1) << (lg + 1)) <= v, lg + 1, lg)
    frac = np.where(lg >= 2, (v >> np.maximum(lg - 2, 0)) & 3, 0)
    out[pos] = 1 + 4 * lg + frac
    return out


def shard_by_length(offsets, world):
    """Database shards for `world` ranks, balanced per length bin: within
    each bin the sequences, longest first (then by id), are dealt to the
    ranks in snake order (0, 1, ..., w-1, w-1, ..., 0, 0, 1, ...), the ranks
    ordered at the start of each bin by the residues they hold so far
    (fewest first).  Every rank then gets about the same residues of every
    length, so both its work for any query and the length of its longest
    items match the others'.  Returns one sorted int64 array of global
    sequence ids per rank; together they cover every sequence exactly once."""
    off = np.asarray(offsets, dtype=np.int64)
    lens = np.diff(off)
    world = int(world)
    if world <= 1:
        return [np.arange(len(lens), dtype=np.int64)]
    bins = length_bins(lens)
    owner = np.empty(len(lens), dtype=np.int64)
    total = np.zeros(world, dtype=np.int64)
    for b in np.unique(bins)[::-1]:  # longest bins first
        ids = np.flatnonzero(bins == b)
        ids = ids[np.lexsort((ids, -lens[ids]))]
        order = np.lexsort((np.arange(world), total))  # fewest residues first
        k = np.arange(len(ids))
        rnd, pos = k // world, k % world
        slot = np.where(rnd % 2 == 0, pos, world - 1 - pos)
        owner[ids] = order[slot]
        np.add.at(total, owner[ids], lens[ids])
    return [np.flatnonzero(owner == r).astype(np.int64) for r in range(world)]


def take(db, offsets, ids):
    """The residues and offsets of the sequences `ids` (a rank's shard), in
    that order, as a database of its own (host numpy arrays)."""
    off = np.asarray(offsets, dtype=np.int64)
    ids = np.asarray(ids, dtype=np.int64)
    lens = off[ids + 1] - off[ids]
    sub_off = np.zeros(len(ids) + 1, dtype=np.int64)
    np.cumsum(lens, out=sub_off[1:])
    if len(ids) == 0:
        return np.zeros(0, dtype=np.uint8), sub_off
    idx = np.repeat(off[ids] - sub_off[:-1], lens) + np.arange(int(sub_off[-1]), dtype=np.int64)
    return np.asarray(db)[idx].astype(np.uint8), sub_off


def gather_scores(local, ids, n_global, device=None):
    """Every rank's score slices put back into the global database order:
    local is this rank's scores (torch tensor, [..., len(ids)]), ids the
    global sequence ids of its shard.  One all_gather of the padded slices
    and their ids; every rank returns the full [..., n_global] tensor (on
    `device`, default local's).  Identity placement on a single process."""
    import torch
    import torch.distributed as dist
    device = device or local.device
    ids_t = torch.as_tensor(np.asarray(ids, dtype=np.int64), device=device)
    lead = tuple(local.shape[:-1])
    out = torch.full(lead + (int(n_global),), -1, dtype=local.dtype, device=device)
    if not _initialised():
        out[..., ids_t] = local.to(device)
        return out
    world = dist.get_world_size()
    cnt = torch.tensor([ids_t.numel()], dtype=torch.int64, device=device)
    cnts = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(cnts, cnt)
    width = int(max(int(c.item()) for c in cnts))
    pad_s = torch.full(lead + (width,), -1, dtype=local.dtype, device=device)
    pad_s[..., :ids_t.numel()] = local.to(device)
    pad_i = torch.full((width,), -1, dtype=torch.int64, device=device)
    pad_i[:ids_t.numel()] = ids_t
    all_s = [torch.empty_like(pad_s) for _ in range(world)]
    all_i = [torch.empty_like(pad_i) for _ in range(world)]
    dist.all_gather(all_s, pad_s)
    dist.all_gather(all_i, pad_i)
    for s, i, c in zip(all_s, all_i, cnts):
        k = int(c.item())
        out[..., i[:k]] = s[..., :k]
    return out
