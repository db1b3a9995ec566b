"""The benchmark's N > 1 host logic on CPU: two ranks over gloo.

Each rank runs a replica of the workload ("replicas only": one grid is not
split across GPUs in this build), so the only cross-rank step is the
max-over-ranks time; the whole-job value is world x cells / that time.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_setup()
        assert (w, r) == (world, rank)
        ms_local = 2.0 + rank          # rank 1 is the slow one
        value, ms_max = bench.job_throughput(1000, ms_local, world)
        out[rank] = (value, ms_max)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_job_throughput_takes_slowest_rank(world):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert sorted(out.keys()) == list(range(world))
    for rank in range(world):
        value, ms_max = out[rank]
        assert ms_max == 2.0 + (world - 1)
        assert value == pytest.approx(1000 * world / (ms_max * 1e-3))
