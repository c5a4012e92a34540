"""Env sharding (one process per GPU) tested on CPU with gloo ranks.

* `partition` gives contiguous, non-empty ranges covering every env once,
  with the smallest possible largest range cost (brute force on small
  inputs);
* two gloo ranks each step their own contiguous share of an uneven env set
  with the oracle (the compute stand-in on CPU) under their global env ids;
  gathered on rank 0 the ranges, rewards and maps equal those of one process
  stepping the whole set, bit for bit;
* the max over ranks of the timed duration is the largest rank's value.
"""
import itertools
import os
import socket

import numpy as np
import pytest

from paper_2603_25834_gb300 import shard, synth

E_SET, STEPS = 9, 4
KW = dict(sides=(24, 40, 56), beams=(16, 24, 40), K=2)
PARAMS = dict(r_max=2.5, sigma=0.02)


def brute_best(cost, world):
    E = len(cost)
    best = None
    for cuts in itertools.combinations(range(1, E), world - 1):
        b = (0,) + cuts + (E,)
        m = max(sum(cost[b[i]:b[i + 1]]) for i in range(world))
        best = m if best is None else min(best, m)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_partition_is_contiguous_complete_and_optimal(seed):
    rng = np.random.default_rng(seed)
    E = int(rng.integers(1, 10))
    world = int(rng.integers(1, E + 1))
    cost = rng.integers(0, 50, size=E)
    b = shard.partition(cost, world)
    assert b[0] == 0 and b[-1] == E and len(b) == world + 1
    assert np.all(np.diff(b) >= 1)
    m = max(int(cost[b[i]:b[i + 1]].sum()) for i in range(world))
    assert m == brute_best(list(cost), world)


def test_partition_rejects_bad_input():
    with pytest.raises(ValueError):
        shard.partition([1, 2], 3)
    with pytest.raises(ValueError):
        shard.partition([1, 2], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shapes():
    side, nb = synth.uneven_shapes(E_SET, KW["sides"], KW["beams"])
    return shard.env_cost(side, side, nb)


def _run_oracle(envs):
    import oracle
    inp = synth.uneven(E_SET, envs=envs, **KW)
    b = oracle.OracleBatch2D(inp, env_ids=np.asarray(list(envs)), **PARAMS)
    acts = synth.random_actions(STEPS, E_SET, 5)[:, list(envs)]
    z, rew = [], []
    for s in range(STEPS):
        o = b.step(acts[s])
        z.append([o["z"][i, :int(inp.n_beams[i])].copy() for i in range(inp.n_envs)])
        rew.append(o["reward_comp"].copy())
    maps = [b.env_belief(i).copy() for i in range(inp.n_envs)]
    return z, rew, maps


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = shard.env_range(_shapes(), world, rank)
        res = (lo, hi) + _run_oracle(range(lo, hi))
        got = [None] * world
        dist.all_gather_object(got, res)
        mx = shard.max_over_ranks(10.0 + rank)
        if rank == 0:
            q.put((got, mx))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_one_process(orc):
    import multiprocessing as mp
    import torch.multiprocessing as tmp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    tmp.spawn(_rank_main, args=(2, _free_port(), q), nprocs=2, join=True)
    got, mx = q.get()
    assert mx == 11.0
    assert [g[0] for g in got] == [0, got[0][1]] and got[1][1] == E_SET
    assert got[0][1] == got[1][0]
    z1, rew1, maps1 = _run_oracle(range(E_SET))
    for lo, hi, z, rew, maps in got:
        for s in range(STEPS):
            for i, e in enumerate(range(lo, hi)):
                assert np.array_equal(z[s][i], z1[s][e]), (s, e)
            assert np.array_equal(rew[s], rew1[s][lo:hi])
        for i, e in enumerate(range(lo, hi)):
            assert np.array_equal(maps[i], maps1[e])
