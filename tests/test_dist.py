"""Host logic of the multi-GPU path on CPU with two gloo ranks: disjoint run
ids and shards that cover every unit once, and the max-over-ranks timing."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2503_10302_gb300 import dist as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    R, steps = 256, 3
    ids = [D.run_ids(s, rank, world, R) for s in range(steps)]
    b, e = D.shard(1001, rank, world)
    t = D.max_over_ranks(10.0 + rank, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, (ids, (b, e), t))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_partition_and_timing():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    R = 256
    runs = set()
    for ids, _, _ in res:
        for first in ids:
            block = set(range(first, first + R))
            assert not (runs & block)
            runs |= block
    assert runs == set(range(2 * 3 * R))
    (b0, e0), (b1, e1) = res[0][1], res[1][1]
    assert b0 == 0 and e0 == b1 and e1 == 1001 and abs((e0 - b0) - (e1 - b1)) <= 1
    assert res[0][2] == res[1][2] == 11.0
