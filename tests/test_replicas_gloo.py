"""The multi-GPU form runs independent replicas (the step has no exchange across
GPUs here): the job time is the slowest rank's, and the throughput counts every
replica's zones.  The rank reduction of bench.py, on two gloo ranks on the CPU."""
import os
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")
    out[rank] = (t, bench.replica_throughput(1000, 4, t, ws))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_rank, args=(2, 29533, out), nprocs=2, join=True, start_method="spawn")
    assert out[0][0] == 15.0 and out[1][0] == 15.0
    assert abs(out[0][1] - 2 * 1000 * 4 / 15e-3) < 1e-6
