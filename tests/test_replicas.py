"""bench.py's N > 1 path runs independent replicas: the step time is the
slowest rank's and the value counts every rank's units.  Checked with two
gloo ranks on the CPU."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank              # rank 1 is the slowest
        slow = bench.max_over_ranks(mine, dist, device="cpu")
        out[rank] = (slow, bench.job_throughput(world, 150, slow * 1e-3))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_with_two_gloo_ranks():
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slow, value = res[0]
    assert slow == 15.0
    assert value == pytest.approx(2 * 150 / 0.015)


def test_single_process_passes_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_throughput(1, 150, 0.5) == 300.0
