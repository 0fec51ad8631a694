"""The N-replica host logic of the benchmark (one process per GPU, each
rendering its own keyframe, no data-path exchange) on two CPU processes
with the gloo backend: the slowest rank's time sets the job's throughput."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 100.0 + 25.0 * rank  # rank 1 is the slow one
        total = bench.max_over_ranks(my_ms, world)
        dist.barrier()
        value = bench.job_throughput(307200, 10, world, total)
        q.put((rank, total, value, bench.keyframe_of_rank(rank)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [125.0, 125.0]
    # both ranks report the whole job: 2 x 307,200 px x 10 steps in 125 ms
    assert out[0][2] == out[1][2] == pytest.approx(2 * 307200 * 10 / 1e6 / 0.125)
    assert [o[3] for o in out] == [0, 1]


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(100, 4, 1, 2.0) == pytest.approx(100 * 4 / 1e6 / 2e-3)
    assert [bench.keyframe_of_rank(r) for r in (0, 7, 8, 13)] == [0, 7, 0, 5]
