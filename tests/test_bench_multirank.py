"""The benchmark's multi-rank logic on CPU with two gloo ranks: every rank learns the slowest
rank's time, the whole-job rate counts the units of all ranks over that time, and the
replicas solve different seeded volumes (no data-path collective: replicas only)."""

import os
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        t_local = 1.0 + rank          # rank 1 is the slow one
        t_max = bench.max_over_ranks(t_local, "cpu")
        rate = bench.whole_job_rate(100.0, world, t_max)
        vol = bench.replica_volume("vol32_iso9_n3_k3", rank)
        out[rank] = (t_max, rate, float(np.sum(vol.m)), bench.dist_env())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = 29500 + (os.getpid() % 2000)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0                  # max over ranks, on both ranks
    assert res[0][1] == res[1][1] == 2 * 100.0 / 2.0      # all ranks' units / slowest time
    assert res[0][2] != res[1][2]                         # seed = rank: distinct replicas
    assert res[0][3] == (0, 0, 2) and res[1][3] == (1, 1, 2)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(0.25, "cpu") == 0.25
    assert bench.whole_job_rate(3932160 * 30, 1, 0.004) == 3932160 * 30 / 0.004
