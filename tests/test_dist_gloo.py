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
        spans = [bench.shard(513, k, w) for k in range(w)]
        out.put((rank, r, w, lr, m, spans[rank], spans))
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
    res.sort()
    for rank, r, w, lr, m, mine, spans in res:
        assert (r, w, lr) == (rank, 2, rank)
        assert m == pytest.approx(2.5)
        assert spans[0][0] == 0 and spans[-1][1] == 513
        assert spans[0][1] == spans[1][0]
        assert abs((spans[0][1] - spans[0][0]) - (spans[1][1] - spans[1][0])) <= 1


def test_shard_covers_all_units():
    import bench
    for n in (0, 1, 7, 512):
        for world in (1, 2, 3, 8):
            spans = [bench.shard(n, r, world) for r in range(world)]
            covered = [i for a, b in spans for i in range(a, b)]
            assert covered == list(range(n))
