"""Env sharding over GPUs: one process per GPU, each owning a contiguous range
of the global env set.

The environments of the batched simulation (Sec. IV, Fig. 1: thousands of
independent robots) exchange nothing during a step, so a step needs no
collective.  Ranks split the envs into contiguous ranges balanced by the
per-env work W*H*B (cells x beams), create their batch with
``env_base = lo`` so each env keeps its global noise stream, and meet only
outside the timed region: a barrier and a max over ranks of the timed
duration.
"""
import numpy as np


def env_cost(map_w, map_h, n_beams, map_d=None):
    """Per-env work estimate: cells x beams (x depth for voxel volumes)."""
    c = np.asarray(map_w, np.int64) * np.asarray(map_h, np.int64) * np.asarray(n_beams, np.int64)
    if map_d is not None:
        c = c * np.asarray(map_d, np.int64)
    return c


def _parts_needed(cost, cap):
    parts, acc = 1, 0
    for c in cost:
        if acc + c > cap:
            parts, acc = parts + 1, int(c)
        else:
            acc += int(c)
    return parts


def partition(cost, world):
    """Bounds [world + 1] of `world` contiguous, non-empty env ranges whose
    largest summed cost is the smallest possible (binary search on that
    bottleneck, greedy cuts from the left)."""
    cost = np.asarray(cost, dtype=np.int64)
    E = int(cost.size)
    if world < 1:
        raise ValueError("world size must be >= 1")
    if E < world:
        raise ValueError("fewer envs (%d) than ranks (%d)" % (E, world))
    if np.any(cost < 0):
        raise ValueError("negative env cost")
    lo, hi = int(cost.max()), int(cost.sum())
    while lo < hi:
        mid = (lo + hi) // 2
        if _parts_needed(cost, mid) <= world:
            hi = mid
        else:
            lo = mid + 1
    cap = lo
    bounds, acc, n_cur = [0], 0, 0
    for e in range(E):
        c = int(cost[e])
        # cut when the range is full, or when the envs left only just cover
        # the ranges still to fill (one env each)
        if n_cur > 0 and (acc + c > cap or E - e == world - len(bounds)):
            bounds.append(e)
            acc, n_cur = 0, 0
        acc += c
        n_cur += 1
    bounds.append(E)
    assert len(bounds) == world + 1
    return np.asarray(bounds, dtype=np.int64)


def env_range(cost, world, rank):
    """(lo, hi) of this rank's envs."""
    b = partition(cost, world)
    return int(b[rank]), int(b[rank + 1])


def max_over_ranks(x, device=None):
    """Max of a host float over the ranks of the default process group
    (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, device=None):
    """Sum of a host number over the ranks of the default process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return type(x)(t.item())
