"""Multi-process helpers (one process per GPU).

The hot path has no data-path collective: a single grid runs as one replica
per GPU, and batched patches are independent problems sharded across ranks.
These helpers only synchronise timing: a barrier and the maximum of a
per-rank time, plus the cost-balanced assignment of patches to ranks.
"""
import os


def world():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, device=None):
    """Maximum of a float over all ranks (value itself when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def shard_patches(dims, nranks):
    """Assign patches to ranks, largest first to the least loaded rank
    (greedy LPT on interior points).  Returns a list of patch-index lists,
    each sorted; every patch appears exactly once."""
    cost = [int(a) * int(b) * int(c) for a, b, c in dims]
    order = sorted(range(len(dims)), key=lambda p: (-cost[p], p))
    load = [0] * nranks
    out = [[] for _ in range(nranks)]
    for p in order:
        r = min(range(nranks), key=lambda q: (load[q], q))
        out[r].append(p)
        load[r] += cost[p]
    return [sorted(x) for x in out]
