"""The multi-process path on CPU (gloo, world size 2): each rank's fill
stream is spawn key = rank, seeded by the library's host code exactly as the
oracle seeds it; the ranks' streams differ; batch requests split with no
overlap and nothing missing; the timing reduction takes the max time and
the summed work.  No GPU and no data-path collective."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import paper_2605_05099_gb300 as rp
        from paper_2605_05099_gb300 import inputs, shard
        key = shard.rank_spawn_key(rank, world)
        assert key == rank
        words = rp.rp_seed_state("xoshiro256pp", 2024, key)
        assert words == oracle.state_words(oracle.gen("xoshiro256pp", 2024, key))[:4]
        got = [None] * world
        dist.all_gather_object(got, words)
        reqs = inputs.batch_workload(n_req=37, lo=10, hi=1e4, seed=1)
        mine = [r["stream"] for r in shard.shard_requests(reqs, rank, world)]
        all_mine = [None] * world
        dist.all_gather_object(all_mine, mine)
        ms, work = shard.reduce_timing(10.0 + rank, 100.0 * (rank + 1))
        q.put((rank, got, all_mine, ms, work))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, all_mine, ms, work in res:
        assert got[0] != got[1]
        flat = sorted(s for part in all_mine for s in part)
        assert flat == list(range(37))
        assert not set(all_mine[0]) & set(all_mine[1])
        assert ms == 11.0 and work == 300.0


def test_single_process_keeps_stream():
    from paper_2605_05099_gb300 import shard
    assert shard.rank_spawn_key(0, 1) == shard.NO_STREAM
    assert shard.rank_spawn_key(0, 1, 7) == 7
    assert shard.reduce_timing(3.0, 5.0) == (3.0, 5.0)
