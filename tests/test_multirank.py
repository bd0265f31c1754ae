"""The multi-process path on CPU: world_size-2 gloo ranks shard the
instances, run their chains (the oracle stands in for each rank's GPU), and
reduce only counters and timings.  The sharded job must equal the one-process
job exactly, because every chain keeps its global Philox stream id."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2210_10513_gb300 import shard


def _problems():
    from paper_2210_10513_gb300 import synth
    ns = [24, 40, 17, 33, 50]
    return [dict(n=n, q=synth.dense_int(n, -9, 9, 10 + i, np.int32), betas=[0.3, 0.6]) for i, n in enumerate(ns)]


CFG = dict(variant="unbiased", k=5, L0=50, seed=17)
CPR = 2
RECORDS = 400


def _run_shard(start, stop, base):
    from oracle import oracle as O
    probs = _problems()[start:stop]
    res = O.run_independent([O.Problem(q=p["q"]) for p in probs], [p["betas"] for p in probs], CFG, CPR, None,
                            RECORDS, id_base=base)
    return {"flips": sum(r["state"].flips for r in res.values()),
            "sum_m": sum(r["state"].sum_m for r in res.values()),
            "energy": sum(r["state"].E for r in res.values()),
            "chains": len(res)}


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = _problems()
    costs = [p["n"] ** 2 * len(p["betas"]) for p in probs]
    start, stop = shard.shard_instances(costs, world, rank)
    base = shard.chain_base([len(p["betas"]) for p in probs], CPR, start)
    local = _run_shard(start, stop, base)
    total = shard.reduce_sum(local, dist)
    tmax = shard.reduce_max(float(rank + 1), dist)
    dist.barrier()
    if rank == 0:
        np.save(os.path.join(out_dir, "total.npy"), np.array([total["flips"], total["sum_m"], total["energy"],
                                                               total["chains"], tmax]))
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_shard_bounds_place_each_edge_nearest_its_target():
    # costs [1, 10] on two ranks: the edge after the first instance is nearer
    # the half-way cost (5.5) than the end, so neither rank is empty
    assert [shard.shard_instances([1, 10], 2, r) for r in range(2)] == [(0, 1), (1, 2)]
    assert [shard.shard_instances([10, 1], 2, r) for r in range(2)] == [(0, 1), (1, 2)]
    assert [shard.shard_instances([3, 3, 3, 3], 2, r) for r in range(2)] == [(0, 2), (2, 4)]


def test_shard_bounds_cover_everything():
    costs = [5, 1, 1, 9, 2, 2, 7]
    for world in (1, 2, 3, 4, 7, 9):
        spans = [shard.shard_instances(costs, world, r) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == len(costs)
        for a, b in zip(spans, spans[1:]):
            assert a[1] == b[0] and a[0] <= a[1]
    assert shard.chain_base([2, 3, 1], 4, 2) == 4 * 2 + 4 * 3


@pytest.mark.timeout(600)
def test_two_rank_gloo_job_equals_single_process(tmp_path):
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=540)
        assert p.exitcode == 0
    got = np.load(os.path.join(tmp_path, "total.npy"))
    full = _run_shard(0, len(_problems()), 0)
    assert got[0] == full["flips"] and got[1] == full["sum_m"] and got[3] == full["chains"]
    assert abs(got[2] - full["energy"]) < 1e-9 * max(1.0, abs(full["energy"]))
    assert got[4] == 2.0  # max over ranks


def test_shard_costs_balanced():
    """Each rank's share of the summed cost is within one instance's cost of
    the even share, and every instance belongs to exactly one rank."""
    rng = np.random.default_rng(3)
    for trial in range(200):
        n = int(rng.integers(1, 60))
        costs = (rng.integers(128, 2049, size=n) ** 2).tolist()
        world = int(rng.integers(1, 9))
        spans = [shard.shard_instances(costs, world, r) for r in range(world)]
        owned = np.zeros(n, int)
        for a, b in spans:
            owned[a:b] += 1
            if n >= world:
                assert b > a, (trial, spans)  # no rank left without an instance
        assert (owned == 1).all()
        total, cmax = float(sum(costs)), float(max(costs))
        for a, b in spans:
            assert sum(costs[a:b]) <= total / world + cmax + 1e-9, (trial, spans)
    assert shard.group_base(3, 5) == 15
