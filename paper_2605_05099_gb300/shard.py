"""Sharding across GPUs, one process per GPU.

Fills shard by stream: rank r of a multi-process run fills spawn key r of
the seed (a single process keeps the caller's stream).  Batches shard by
request: rank r takes requests r, r + world, ...  No data moves between
ranks; the only collective is the timing reduction (max of the ranks'
times, sum of their work), done by whoever measures.
"""
NO_STREAM = (1 << 64) - 1


def rank_spawn_key(rank, world, stream=NO_STREAM):
    """Spawn key of rank `rank`'s stream: the caller's for one process."""
    return stream if world == 1 else rank


def shard_requests(reqs, rank, world):
    """Requests served by rank `rank` (round robin, so sizes balance)."""
    return list(reqs[rank::world])


def reduce_timing(ms, work, device=None):
    """(max over ranks of ms, sum over ranks of work) through
    torch.distributed; plain values without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(work)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())
