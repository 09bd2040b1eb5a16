"""The batched form across several GPUs: instance sharding.

Independent instances exchange nothing while they run, so the batch splits
by instance with no collective on the data path: rank r of N owns the
instances i with i mod N == r (round-robin, so every shape class is spread
over the ranks in proportion), advances them as its own batch on its own
GPU, and the ranks meet once at the end to all-gather a few scalars per
instance (accepted and rejected steps, final time, status).
"""
import math

STAT_FIELDS = ("accepted", "rejected", "t", "status")


def instance_shard(n, rank, world):
    """Indices of the instances rank `rank` of `world` owns."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(range(rank, n, world))


def gather_instance_stats(ids, stats, n, world, device="cpu"):
    """All-gather of the per-instance stats of every rank (torch.distributed
    initialised): `ids` are this rank's instance indices and `stats` their
    dicts (STAT_FIELDS).  Returns the list of n dicts in instance order, the
    same on every rank.  With world == 1 the local stats are returned in
    instance order."""
    if world == 1:
        out = [None] * n
        for i, s in zip(ids, stats):
            out[i] = {k: s[k] for k in STAT_FIELDS}
        return out
    import torch
    import torch.distributed as dist
    slots = math.ceil(n / world)
    local = torch.full((slots, 1 + len(STAT_FIELDS)), -1.0, dtype=torch.float64, device=device)
    for j, (i, s) in enumerate(zip(ids, stats)):
        local[j, 0] = float(i)
        for f, k in enumerate(STAT_FIELDS):
            local[j, 1 + f] = float(s[k])
    parts = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(parts, local)
    out = [None] * n
    for part in parts:
        for row in part.cpu().tolist():
            if row[0] < 0:
                continue
            i = int(row[0])
            out[i] = {k: row[1 + f] for f, k in enumerate(STAT_FIELDS)}
            out[i]["accepted"] = int(out[i]["accepted"])
            out[i]["rejected"] = int(out[i]["rejected"])
            out[i]["status"] = int(out[i]["status"])
    missing = [i for i, s in enumerate(out) if s is None]
    if missing:
        raise RuntimeError(f"instances without stats after the gather: {missing[:8]}")
    return out
