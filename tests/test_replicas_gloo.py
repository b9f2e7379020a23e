"""The N > 1 path of bench.py on the CPU with two gloo ranks: replicas take
disjoint frames (no data-path collective) and the job time is the maximum
over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    frames = bench.rank_frames(rank, world, 300, 150)
    elapsed = bench.reduce_max(10.0 + rank, dist, None)
    gathered = [None] * world
    dist.all_gather_object(gathered, frames)
    if rank == 0:
        out.put((gathered, elapsed))
    dist.destroy_process_group()


def test_two_replicas_split_frames_and_take_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, elapsed = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = gathered
    assert set(a).isdisjoint(b) and set(a) | set(b) == set(range(300))
    assert elapsed == 11.0


def test_single_rank_defaults():
    import bench
    assert bench.rank_frames(0, 1, 300, 5) == [0, 1, 2, 3, 4]
    assert bench.reduce_max(3.5, None) == 3.5
