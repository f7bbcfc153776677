"""The multi-GPU host logic on CPU: two gloo ranks (world_size 2).

bench.py: every rank searches its own replica (weak scaling, no collective on the
data path); the only collectives are the timing barrier and the max-over-ranks
reduction of the timed milliseconds.  Candidate sharding
(paper_2101_07731_gb300/sharded.py): every rank searches its own shard and the exact
merge of the per-shard answers is the one data-path exchange."""
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


# ------------------------------------------------------------------ candidate sharding

def _merge_worker(rank, world, port, shards, out):
    import numpy as np
    import oracle as O
    from paper_2101_07731_gb300.sharded import merge_nn_shards
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        Q, Cn, W = shards["Q"], shards["C"], shards["W"]
        lo, hi = shards["bounds"][rank]
        # this rank's shard searched exactly (the oracle stands in for the GPU search)
        li, ld = O.nn_brute(Q, Cn[lo:hi], W)
        gi, gd = merge_nn_shards(torch.from_numpy(np.asarray(li, np.int64)),
                                 torch.from_numpy(np.asarray(ld, np.float64)), lo)
        out[rank] = (gi.numpy().tolist(), gd.numpy().tolist())
    finally:
        dist.destroy_process_group()


def test_candidate_sharded_nn_merge_is_exact_over_two_gloo_ranks():
    import numpy as np
    import oracle as O
    import synth
    spec = synth.SeriesSpec("random_walk", 24, 2, 61)
    Q = synth.generate(spec, synth.ROLE_QUERY, 6)
    Cn = synth.generate(spec, synth.ROLE_CAND, 40)
    # ties across shards: candidate 27 (rank 1) duplicates candidate 3 (rank 0), and
    # query 0 is candidate 27 itself, so both shards find distance 0
    Cn[27] = Cn[3]
    Q[0] = Cn[27]
    W = 3
    shards = {"Q": Q, "C": Cn, "W": W, "bounds": [(0, 17), (17, 40)]}
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_merge_worker, args=(2, _free_port(), shards, out), nprocs=2, start_method="spawn", join=True)
    ridx, rdist = O.nn_brute(Q, Cn, W)
    for rank in (0, 1):
        gi, gd = out[rank]
        assert gi == [int(v) for v in ridx]
        assert gd == [float(v) for v in rdist]
    assert out[0][0][0] == 3  # the tie goes to the smaller global index
