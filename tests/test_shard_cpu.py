"""Sharding one study over ranks (gloo, world sizes 2 and 3, CPU): the sample-range partition
and the gather of per-sample tallies that V_dep and the MFMC estimators consume whole."""
import itertools
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


def test_partition_covers_every_sample_once_and_is_optimal():
    from paper_2205_04979_gb300 import shard
    import workloads
    _, counts = workloads.workload_inputs("batched_mixed")
    for world in (1, 2, 3, 4, 8):
        r = shard.partition(counts, world)
        assert len(r) == world and r[0][0] == 0 and r[-1][1] == len(counts)
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))          # contiguous, no gap or overlap
        cost = shard.range_costs(counts, r)
        assert sum(cost) == int(np.sum(np.asarray(counts, np.int64) ** 2))
        # balanced: within one sample's cost of the perfect split
        assert max(cost) <= sum(cost) / world + int(np.max(np.asarray(counts, np.int64) ** 2))
    # brute force on a small case: no contiguous split has a smaller largest cost
    rng = np.random.default_rng(3)
    c = rng.integers(1, 50, 9)
    for world in (2, 3, 4):
        best = min(max(shard.range_costs(c, list(zip((0,) + cuts, cuts + (9,)))))
                   for cuts in itertools.combinations(range(1, 9), world - 1))
        assert max(shard.range_costs(c, shard.partition(c, world))) == best
    # more ranks than samples: trailing empty ranges
    assert shard.partition([5, 5], 4) == [(0, 1), (1, 2), (2, 2), (2, 2)]


def _tallies(samples, C=5):
    """Deterministic stand-in tallies per sample (what each rank's step would accumulate)."""
    s = np.asarray(samples, np.int64)[:, None]
    k = np.arange(C, dtype=np.int64)[None, :]
    return (s * 7 + k * 3) % 11, 1000 + s * 13 + k


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    from paper_2205_04979_gb300 import shard
    import oracle
    import workloads
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    _, counts = workloads.workload_inputs("batched_mixed", 64)
    ranges = shard.partition(counts, world)
    lo, hi = ranges[rank]
    nd, na = _tallies(range(lo, hi))
    full_nd = shard.gather_rows(torch.from_numpy(nd), ranges, rank)
    full_na = shard.gather_rows(torch.from_numpy(na), ranges, rank)
    # pick-freeze outputs of this rank's groups: [groups][d + 2][C] doubles
    y = np.sin(np.arange(lo, hi)[:, None, None] * 0.37 + np.arange(5)[None, :, None] + np.arange(2)[None, None, :])
    full_y = shard.gather_rows(torch.from_numpy(y), ranges, rank)
    vdep = oracle.vdep(full_nd.numpy(), full_na.numpy(), 0.05)
    out[rank] = (ranges, full_nd.numpy().tolist(), full_na.numpy().tolist(), full_y.numpy().tolist(), vdep.tolist())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gathered_tallies_equal_the_single_rank_tables(world):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from oracle import mfmc
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    nd, na = _tallies(range(64))
    y = np.sin(np.arange(64)[:, None, None] * 0.37 + np.arange(5)[None, :, None] + np.arange(2)[None, None, :])
    for r in range(world):
        ranges, gnd, gna, gy, gv = out[r]
        assert np.array_equal(np.asarray(gnd), nd) and np.array_equal(np.asarray(gna), na)
        assert np.array_equal(np.asarray(gy), y)                      # bit-exact, sample order
        assert np.array_equal(np.asarray(gv), oracle.vdep(nd, na, 0.05))
    # the estimators on the gathered table are the single-rank estimators
    s_all = mfmc.mfmc_sobol([y], [64], [1.0])
    s_gat = mfmc.mfmc_sobol([np.asarray(out[world - 1][3])], [64], [1.0])
    for a, b in zip(s_all, s_gat):
        assert np.array_equal(a, b)
