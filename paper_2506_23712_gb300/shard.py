"""Member sharding across processes (one GPU each).

Ensemble members are independent until the lambda mixture (Sec. IV: the
members differ only in their injection rate and are mixed afterwards), so a
multi-GPU run partitions the members, advances each shard with its own
context, and gathers the per-member statistics (a few tens of KB each) to one
process, which mixes them with ``ens_mixture_host``.  No collective runs
during time stepping.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def partition_members(grid_sizes: Sequence[int], world: int) -> List[List[int]]:
    """Longest-processing-time greedy partition of member indices over
    `world` ranks, balancing the per-step work (proportional to N^3).
    Deterministic: ties go to the lowest rank / lowest member index."""
    order = sorted(range(len(grid_sizes)), key=lambda i: (-int(grid_sizes[i]) ** 3, i))
    loads = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += int(grid_sizes[i]) ** 3
    return [sorted(p) for p in parts]


def gather_stats(member_ids: Sequence[int], counts: np.ndarray, moments: np.ndarray, n_total: int,
                 dst: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Gather every rank's per-member counts and moments to rank `dst`, in
    global member order (torch.distributed, any backend).  Other ranks get
    (None, None)."""
    import torch.distributed as dist
    payload = (list(map(int, member_ids)), np.asarray(counts, dtype=np.uint64), np.asarray(moments, dtype=np.float64))
    rank = dist.get_rank()
    objs = [None] * dist.get_world_size() if rank == dst else None
    dist.gather_object(payload, objs, dst=dst)
    if rank != dst:
        return None, None
    L, M = payload[1].shape[1], payload[2].shape[1]
    all_counts = np.zeros((n_total, L), dtype=np.uint64)
    all_moments = np.zeros((n_total, M), dtype=np.float64)
    seen = np.zeros(n_total, dtype=bool)
    for ids, c, m in objs:
        for k, i in enumerate(ids):
            if seen[i]:
                raise ValueError("member %d reported by two ranks" % i)
            seen[i] = True
            all_counts[i] = c[k]
            all_moments[i] = m[k]
    if not seen.all():
        raise ValueError("members missing from the gather: %s" % np.flatnonzero(~seen).tolist())
    return all_counts, all_moments
