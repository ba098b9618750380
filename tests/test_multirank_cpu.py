"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): each rank gets
its own batch of samples of the same sizes (weak scaling), and the timing reduction
takes the slowest rank's time and the sum of the particle-steps."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    params, counts = bench.rank_workload("batched_mixed", rank, world, samples=16)
    ms, ps = bench.reduce_over_ranks(10.0 * (rank + 1), 1000 * (rank + 1), world, "cpu")
    out[rank] = (params.tolist(), counts.tolist(), ms, ps)
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_inputs_and_reduction():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    p0, c0, ms0, ps0 = out[0]
    p1, c1, ms1, ps1 = out[1]
    assert c0 == c1                                   # same per-rank work
    assert not np.allclose(p0, p1)                    # independent samples
    assert ms0 == ms1 == 20.0 and ps0 == ps1 == 3000.0
    # rank 0 of a multi-rank run keeps the single-GPU sizes; ranges stay inside +-50 % of nominal
    p = np.asarray(p1)
    assert np.all(p > 0) and np.all(p[:, 0] <= 0.075 + 1e-12) and np.all(p[:, 1] <= 0.75 + 1e-12)


def test_single_rank_needs_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.reduce_over_ranks(5.0, 7, 1, "cpu") == (5.0, 7.0)
