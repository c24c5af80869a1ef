"""Multi-rank path of bench.py on CPU (gloo, world_size 2): queries are sharded
without any data-path exchange, and the per-rank measurements are combined
as max time / summed work."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    items = list(range(23))
    mine = bench.shard(items, rank, world)
    # per-rank "measurements": time grows with rank, work = number of items
    local = [10.0 + rank, float(len(mine)), float(sum(mine))]
    allv = bench.combine(local, world)
    q.put((rank, mine, allv.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_combine():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    shards = [set(o[1]) for o in out]
    assert shards[0].isdisjoint(shards[1])
    assert shards[0] | shards[1] == set(range(23))
    for _, _, allv in out:
        a = np.array(allv)
        assert a.shape == (2, 3)
        assert a[:, 0].max() == 11.0
        assert a[:, 1].sum() == 23
        assert a[:, 2].sum() == sum(range(23))


def test_single_rank_combine():
    import bench
    a = bench.combine([1.0, 2.0], 1)
    assert a.shape == (1, 2) and a[0, 1] == 2.0
    assert bench.shard(list(range(5)), 0, 1) == list(range(5))
