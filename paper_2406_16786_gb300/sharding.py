"""Sharding of independent domains across ranks (one GPU per rank).

The batched workload (many independent channels) partitions without any data exchange: each
rank steps its own domains, and the ranks meet only to time the job and to gather the
domains' counters at the end.  Domains are assigned by longest processing time first, with
the particle count as the work estimate.  Host logic only; the collectives run on whatever
process group the caller initialised (gloo on CPU in the tests, NCCL under torchrun).
"""
from __future__ import annotations

from typing import Dict, List, Sequence


def assign_lpt(work: Sequence[float], nranks: int) -> List[List[int]]:
    """Longest processing time first: domains in decreasing work, each to the least-loaded
    rank (the lowest rank on ties).  Returns the domain indices of every rank, ascending."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    load = [0.0] * nranks
    out: List[List[int]] = [[] for _ in range(nranks)]
    for q in sorted(range(len(work)), key=lambda i: (-float(work[i]), i)):
        r = min(range(nranks), key=lambda k: (load[k], k))
        out[r].append(q)
        load[r] += float(work[q])
    return [sorted(x) for x in out]


def gather_counters(local: Dict[int, dict], group=None) -> Dict[int, dict]:
    """Every rank's {domain index: counters} merged on all ranks (all_gather_object)."""
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return dict(local)
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, dict(local), group=group)
    merged: Dict[int, dict] = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise ValueError("domain %d reported by two ranks" % k)
            merged[k] = v
    return merged


def max_over_ranks(value: float, group=None) -> float:
    """The largest value over the ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
