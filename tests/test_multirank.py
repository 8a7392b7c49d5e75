"""The N > 1 host logic of bench.py on CPU with the gloo backend (world size 2):
weak-scaling aggregation (max time over ranks, summed work) and the round-robin
sharding of independent instances."""
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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate(10.0 + rank, 100.0 * (rank + 1), dist, "cpu")
    mine = bench.shard(7, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out.put((rank, ms, units, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_aggregation_two_ranks():
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
    for rank, ms, units, gathered in res:
        assert ms == 11.0                 # the slowest rank
        assert units == 300.0             # all ranks' work
        flat = sorted(i for g in gathered for i in g)
        assert flat == list(range(7))     # every instance exactly once
        assert gathered[0] == [0, 2, 4, 6] and gathered[1] == [1, 3, 5]
