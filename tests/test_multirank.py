"""The multi-GPU host logic of bench.py on CPU: two gloo ranks (world_size 2).

Every rank searches its own replica (weak scaling, no collective on the data
path); the only collectives are the timing barrier and the max-over-ranks
reduction of the timed milliseconds, which these tests exercise with gloo."""
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


def _worker(rank, world, port, local_ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        assert bench._dist_env() == (world, rank, rank)
        dist.barrier()
        t = bench.job_time_ms(local_ms[rank], dist, "cpu")
        out[rank] = t
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("local_ms", [(10.0, 25.0), (40.0, 5.0)])
def test_job_time_is_max_over_two_gloo_ranks(local_ms):
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_worker, args=(world, _free_port(), local_ms, out), nprocs=world, start_method="spawn",
                       join=True)
    assert out[0] == out[1] == max(local_ms)


def test_job_value_is_weak_scaling_throughput():
    # two ranks of 256 queries x 20 steps in the slowest rank's 1,000 ms
    assert bench.job_value(2, 256, 20, 1000.0) == pytest.approx(2 * 256 * 20)
    assert bench.job_value(1, 256, 20, 500.0) == pytest.approx(256 * 20 * 2)
    # one process: the local time is the job time
    assert bench.job_time_ms(12.5) == 12.5
