"""bench.py's multi-GPU aggregation on CPU: world_size-2 gloo ranks, each
with its own time, reduce to the slowest rank's time and the whole job's
throughput (replicas only: no data moves between ranks)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [2.0, 3.5][rank]
    frames = 4
    t = bench.max_over_ranks(seconds, dist, "cpu")
    q.put((rank, t, bench.job_rate(frames, t, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 3.5                     # the slowest rank's time
        assert rate == pytest.approx(8 / 3.5)   # all ranks' frames over it


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.job_rate(3, 1.5, 1) == 2.0
