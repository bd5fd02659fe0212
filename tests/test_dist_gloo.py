"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the max-over-ranks timing
reduction, the barrier, and the split of independent pings across ranks."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        m = bench.reduce_max(1.5 + rank)
        bench.barrier()
        costs = bench.batch_costs(512)
        parts = bench.shard_pings(costs, w)
        out.put((rank, r, w, lr, m, parts[rank], parts, costs))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_and_shard():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda x: x[0])
    mine = []
    for rank, r, w, lr, m, part, parts, costs in res:
        assert (r, w, lr) == (rank, 2, rank)
        assert m == pytest.approx(2.5)
        assert parts == res[0][6]                   # both ranks computed the same split
        mine.append(part)
    # every ping of the 512-ping batch is gridded exactly once, by one rank
    assert sorted(mine[0] + mine[1]) == list(range(512))
    costs = res[0][7]
    loads = [sum(costs[i] for i in p) for p in mine]
    assert max(loads) - sum(costs) / 2 <= max(costs)


def test_shard_pings_balance():
    """Coverage and balance of the work split for several world sizes, including more ranks
    than pings: the largest rank load is within one ping of the ideal share (and of the lower
    bound max(mean load, largest ping))."""
    import random

    import bench
    rnd = random.Random(3)
    for n in (0, 1, 7, 64, 512):
        costs = [rnd.randint(20_000, 400_000) + rnd.choice([512, 1024, 2048]) ** 2
                 for _ in range(n)]
        for world in (1, 2, 3, 8):
            parts = bench.shard_pings(costs, world)
            assert len(parts) == world
            assert sorted(i for p in parts for i in p) == list(range(n))
            if n:
                loads = [sum(costs[i] for i in p) for p in parts]
                lower = max(sum(costs) / world, max(costs))
                assert max(loads) <= lower + max(costs)
                assert max(loads) <= sum(costs) / world + max(costs)
