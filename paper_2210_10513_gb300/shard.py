"""Sharding across GPUs (one process per GPU).

Chains and exchange groups are independent, so a multi-GPU job splits the
instances into contiguous shards, one per rank, and needs no collective on
the data path; each rank's context takes the global id of its first chain and
group (pns_config.chain_base / group_base) so that it draws exactly the
Philox streams the whole job would.  Only counters and timings are reduced,
on the host side of torch.distributed.
"""


def shard_instances(costs, world, rank):
    """Contiguous [start, stop) of instances for `rank`, balancing the summed
    cost (e.g. n^2 bytes of Q per instance times its chains).  Boundary b
    (b = 1 .. world - 1) sits at the instance edge nearest the cost target
    b * total / world, kept strictly increasing so that no rank is empty while
    there are at least `world` instances; the last rank ends at the last
    instance."""
    n = len(costs)
    if world <= 1:
        return 0, n
    prefix = [0.0]
    for c in costs:
        prefix.append(prefix[-1] + float(c))
    total = prefix[-1]
    bounds = [0]
    for b in range(1, world):
        target = total * b / world
        # the edge i (0 < i < n) whose prefix cost is nearest the target
        best = None
        for i in range(1, n):
            if best is None or abs(prefix[i] - target) < abs(prefix[best] - target):
                best = i
        best = best if best is not None else n
        lo = bounds[-1] + 1 if n >= world else bounds[-1]  # at least one instance per rank
        hi = n - (world - b) if n >= world else n           # and room for the ranks after it
        bounds.append(min(max(best, lo), max(lo, hi)))
    bounds.append(n)
    return bounds[rank], bounds[rank + 1]


def chain_base(n_replicas, chains_per_replica, start):
    """Global id of the first chain of instance `start`."""
    return sum(chains_per_replica * r for r in n_replicas[:start])


def group_base(chains_per_replica, start):
    """Global id of the first exchange group of instance `start`."""
    return chains_per_replica * start


def reduce_sum(values, dist=None):
    """Sum a dict of scalars over ranks (float64 on the host backend)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return dict(values)
    import torch
    keys = sorted(values)
    t = torch.tensor([float(values[k]) for k in keys], dtype=torch.float64)
    dist.all_reduce(t)
    return {k: float(v) for k, v in zip(keys, t.tolist())}


def reduce_max(x, dist=None):
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
