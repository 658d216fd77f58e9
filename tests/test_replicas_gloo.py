"""The multi-process path of bench.py is "replicas only" (independent problems,
no data-path collective): each rank seeds its own problem by its rank, and the
reported time is the maximum over ranks. This checks that host logic with two
gloo processes on the CPU (the GPU runs use NCCL, one rank per GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    import numpy as np
    p = W.grid_problem_784(bench.replica_seed(rank))
    local_time = 1.0 + rank  # a stand-in per-rank time: rank 1 is the slower one
    out[rank] = (bench.max_over_ranks(local_time, world), float(np.asarray(p["r"]).sum()),
                 float(p["r"][0]))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_max_over_ranks_and_distinct_seeds():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 2.0          # both ranks report the slowest rank's time
    assert abs(out[0][1] - 1.0) < 1e-12 and abs(out[1][1] - 1.0) < 1e-12
    assert out[0][2] != out[1][2]                 # different problems per rank


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
