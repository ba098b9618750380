"""Sharding one Monte Carlo study over ranks, one GPU each.

The samples of a study are independent until the estimators: each rank steps a contiguous
range of samples with no per-step exchange, and the per-(sample, class) tallies and the
pick-freeze outputs are gathered once at the end, so that V_dep+ (Sec. 2.1) and the
MFMC / Sobol' estimators (Sec. 3) see the whole sample set, as if one GPU had run it.

The pair sum makes a sample of N_s particles cost about N_s^2, so the ranges balance
sum N_s^2: ``partition`` returns the contiguous split that minimises the largest range cost
(binary search on that bottleneck with a greedy feasibility check; integer costs, exact).
"""
import numpy as np


def range_costs(counts, ranges):
    c = np.asarray(counts, np.int64) ** 2
    return [int(c[lo:hi].sum()) for lo, hi in ranges]


def _greedy(cost, cap, world):
    """Contiguous ranges of at most `cap` cost each, left to right; None if more than `world` are needed."""
    ranges, lo, acc = [], 0, 0
    for s, c in enumerate(cost):
        if acc + c > cap and s > lo:
            ranges.append((lo, s))
            lo, acc = s, 0
            if len(ranges) == world:
                return None
        acc += c
    ranges.append((lo, len(cost)))
    return ranges


def partition(counts, world):
    """[(lo, hi)] * world: contiguous sample ranges covering 0..S once, minimising max sum N_s^2.

    Ranks beyond the number of non-empty ranges get empty ranges at the end.
    """
    if world < 1:
        raise ValueError("world >= 1")
    cost = np.asarray(counts, np.int64) ** 2
    S = len(cost)
    if S == 0:
        return [(0, 0)] * world
    lo_cap, hi_cap = int(cost.max()), int(cost.sum())
    while lo_cap < hi_cap:                      # smallest cap with a feasible greedy split
        mid = (lo_cap + hi_cap) // 2
        if _greedy(cost, mid, world) is None:
            lo_cap = mid + 1
        else:
            hi_cap = mid
    ranges = _greedy(cost, lo_cap, world)
    ranges += [(S, S)] * (world - len(ranges))
    return ranges


def gather_rows(local, ranges, rank, group=None):
    """Every rank receives the full table: rows of all ranks' ranges concatenated in sample order.

    local: torch tensor [hi - lo, ...] of this rank's range (CPU for gloo, CUDA for NCCL).
    One all_gather of tensors padded to the longest range.
    """
    import torch
    import torch.distributed as dist
    world = len(ranges)
    lo, hi = ranges[rank]
    assert local.shape[0] == hi - lo, "local rows must match the rank's range"
    longest = max(h - l for l, h in ranges)
    pad = torch.zeros((longest,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: hi - lo] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][: h - l] for r, (l, h) in enumerate(ranges)], 0)
