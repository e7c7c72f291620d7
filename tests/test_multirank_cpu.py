"""The benchmark's multi-rank host logic on CPU: two gloo ranks on 127.0.0.1.

Every rank compresses its own replica (data seed + rank, weak scaling); the
job's time is the slowest rank's (all-reduce MAX) and the job's throughput
counts every rank's nodes. No GPU and no data-path collective are involved.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank                        # rank 1 is the slow one
        job_ms = bench.max_over_ranks(ms, world, "cpu")
        value = bench.job_throughput(508, 10, world, job_ms)
        bench.select_workload("c2")
        pts = bench.workload_points(rank)[:4]            # each rank its own data seed
        out.put((rank, job_ms, value, pts))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_replica():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, job_ms, value, pts = out.get(timeout=120)
        res[r] = (job_ms, value, pts)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 150.0
    assert abs(res[0][1] - 508 * 10 * 2 / 0.150) < 1e-6
    assert not np.array_equal(res[0][2], res[1][2])


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert abs(bench.job_throughput(508, 10, 1, 200.0) - 25400.0) < 1e-9
