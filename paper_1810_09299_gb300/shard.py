"""Sharding of independent cases across ranks (one process per GPU).

The batched workload is a set of independent simulations, so ranks share no
data: each rank advances its own cases and only the benchmark's bookkeeping
(the slowest rank's time, the total node count) crosses ranks.  There is no
collective on the data path.
"""
from __future__ import annotations

from typing import List, Sequence


def assign_cases(sizes: Sequence[int], world: int, rank: int) -> List[int]:
    """Indices of the cases rank `rank` owns: greedy longest-processing-time
    assignment by node count (deterministic; ties go to the lowest rank)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    load = [0] * world
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += sizes[i]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def job_throughput(local_nodes: int, steps: int, local_ms: float, dist=None, device=None):
    """Whole-job MLUPS: total nodes of all ranks x steps / slowest rank's time.
    Returns (mlups, max_ms, total_nodes).  Without an initialised process group
    this is the single-rank value."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return local_nodes * steps / (local_ms * 1e-3) / 1e6, local_ms, local_nodes
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    n = torch.tensor([float(local_nodes)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    ms, nodes = float(t.item()), int(n.item())
    return nodes * steps / (ms * 1e-3) / 1e6, ms, nodes
