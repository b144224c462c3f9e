"""The multi-rank path of bench.py on CPU with two gloo ranks: the batched workload's instances are sharded over
the ranks (each exactly once, no collective on the data path), the timed region is the maximum over ranks and the
work is summed over ranks."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = bench.shard(64, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, units)
    t = bench.reduce_over_ranks(0.5 + rank, world, "cpu", "max")
    w = bench.reduce_over_ranks(len(units) * 1000, world, "cpu", "sum")
    q.put((rank, gathered, t, w))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharded_units_and_rank_reductions(world):
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, t, w in results:
        flat = sorted(u for part in gathered for u in part)
        assert flat == list(range(64))                      # every instance exactly once
        assert all(len(part) == 64 // world for part in gathered)
        assert t == 0.5 + (world - 1)                        # the slowest rank's time
        assert w == 64 * 1000                                # all ranks' work


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.reduce_over_ranks(3.5, 1, None, "max") == 3.5
