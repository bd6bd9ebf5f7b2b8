"""The N>1 path on CPU: slice shards and the end-of-run reductions, with two
gloo ranks (127.0.0.1).  No GPU is needed: the data path has no collective."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def test_slice_shards_partition_the_stack():
    from paper_1306_1392_b300.shard import slice_shard
    for n in (0, 1, 7, 64, 1023, 1024):
        for world in (1, 2, 3, 8):
            ranges = [slice_shard(n, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slice_shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1306_1392_b300.shard import reduce_throughput, slice_shard
        z0, z1 = slice_shard(1024, world, rank)
        ms, units = reduce_throughput(100.0 + 10 * rank, float(z1 - z0))
        q.put((rank, z0, z1, ms, units))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [(r[1], r[2]) for r in res] == [(0, 512), (512, 1024)]
    assert all(r[3] == 110.0 and r[4] == 1024.0 for r in res)      # max time, summed slices


def test_reduce_without_process_group_is_identity():
    from paper_1306_1392_b300.shard import reduce_throughput
    assert reduce_throughput(5.0, 3.0) == (5.0, 3.0)
