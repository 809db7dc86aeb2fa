"""The multi-GPU path of the benchmark is "replicas only": each rank runs
its own system, and the whole-job rate is all ranks' units over the slowest
rank's time.  Checked with two gloo ranks on the CPU."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 180.0][rank]
    mx = bench.max_over_ranks(local_ms, world)
    rate = bench.whole_job_rate(1.0e9, world, mx)
    out[rank] = (mx, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    mx, rate = res[0]
    assert mx == 180.0
    assert rate == pytest.approx(2 * 1.0e9 / 0.180)


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(100.0, 1, 1000.0) == 100.0
