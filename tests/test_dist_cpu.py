"""Multi-rank host logic of bench.py on CPU: gloo, world size 2.

Each rank maps its own keyframes of one trajectory (weak scaling, no
data-path collective); the only cross-rank step is the max of the timings.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    frames = bench.shard_frames(world, rank)
    t = bench.rank_max(10.0 + 5.0 * rank, world, "cpu")
    dist.destroy_process_group()
    q.put((rank, frames, t))


def test_shards_are_disjoint_and_rank_max_is_the_slowest():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, f0, t0), (_, f1, t1) = res
    assert set(f0).isdisjoint(f1) and len(f0) == len(f1) == bench.FRAMES_PER_RANK
    assert sorted(f0 + f1) == list(range(world * bench.FRAMES_PER_RANK))
    assert t0 == t1 == 15.0
    value, t = bench.combine_rank_times([t0, t1], [100, 100])
    assert t == 15.0 and value == pytest.approx(200 / 0.015)
