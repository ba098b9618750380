"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): the ranks split one
study of world x the workload's samples into contiguous ranges balanced by sum N_s^2 (weak
scaling), and the timing reduction takes the slowest rank's time and the sum of the
particle-steps."""
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
    params, counts, ranges = bench.rank_workload("batched_mixed", rank, world, samples=16)
    ms, ps = bench.reduce_over_ranks(10.0 * (rank + 1), 1000 * (rank + 1), world, "cpu")
    out[rank] = (params.tolist(), counts.tolist(), ms, ps, ranges)
    dist.barrier()
    dist.destroy_process_group()


def test_study_sharded_by_rank_and_timing_reduction():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    import sys
    sys.path.insert(0, ROOT)
    import workloads
    p0, c0, ms0, ps0, r0 = out[0]
    p1, c1, ms1, ps1, r1 = out[1]
    assert r0 == r1 and r0[0][0] == 0 and r0[0][1] == r0[1][0] and r0[1][1] == 32
    # the two ranges are the study of 32 samples drawn by the workload's recipe, each once
    w = workloads.WORKLOADS["batched_mixed"]
    assert np.array_equal(np.asarray(c0 + c1), workloads.sample_counts(32, *w["count"], w["param_seed"]))
    assert np.array_equal(np.asarray(p0 + p1), workloads.sample_params(32, w["param_seed"]))
    # balanced pair work: within one sample's cost of half the total
    cost = [sum(int(c) ** 2 for c in cc) for cc in (c0, c1)]
    assert max(cost) <= sum(cost) / 2 + max(int(c) ** 2 for c in c0 + c1)
    assert ms0 == ms1 == 20.0 and ps0 == ps1 == 3000.0
    # inputs stay inside +-50 % of nominal
    p = np.asarray(p0 + p1)
    assert np.all(p > 0) and np.all(p[:, 0] <= 0.075 + 1e-12) and np.all(p[:, 1] <= 0.75 + 1e-12)


def test_single_rank_needs_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import workloads
    assert not dist.is_initialized()
    assert bench.reduce_over_ranks(5.0, 7, 1, "cpu") == (5.0, 7.0)
    # one rank runs the single-GPU workload itself
    params, counts, ranges = bench.rank_workload("batched_mixed", 0, 1, samples=16)
    p, c = workloads.workload_inputs("batched_mixed", 16)
    assert np.array_equal(params, p) and np.array_equal(counts, c) and ranges == [(0, 16)]
