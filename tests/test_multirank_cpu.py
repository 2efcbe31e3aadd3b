"""The multi-rank bench path on CPU: two gloo ranks, each timing its own
independent problem (no data-path collective); the job time is the max over
ranks and the value the work of all ranks over that time."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [0.5, 2.0][rank]  # rank 1 is the slowest
    t = bench.aggregate_over_ranks(dist, torch, seconds, "cpu")
    out[rank] = (t, bench.job_value(world, 1000, 4, t))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.0, 2 * 1000 * 4 / 2.0)


def test_single_rank_is_identity():
    import torch

    import bench

    assert bench.aggregate_over_ranks(None, torch, 1.25, "cpu") == 1.25
    assert bench.job_value(1, 10, 3, 2.0) == 15.0
