"""Parameter sweeps across GPUs: the capillaries of a sweep are independent
problems, so they are split over the ranks (one process per GPU) with no
exchange during the run; each rank steps its share as one batch and the
observables trajectories are gathered once at the end.

``assign`` balances the ranks' lattice sizes (longest-processing-time-first
on nx * ny, then each rank's share kept in sweep order); ``run_sharded``
runs a rank's share through ``runner`` and gathers every trajectory on all
ranks through torch.distributed (any backend: NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import heapq
from typing import Callable, List, Sequence

import numpy as np


def assign(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Indices of the items each of `world` ranks takes, balancing the summed
    sizes: items in decreasing size go to the least loaded rank (ties to the
    lower rank); each rank's list is then sorted."""
    if world < 1:
        raise ValueError("world >= 1")
    heap = [(0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [sorted(v) for v in out]


def run_sharded(caps: Sequence, runner: Callable[[Sequence], np.ndarray], rank: int, world: int,
                group=None) -> np.ndarray:
    """Runs this rank's share of `caps` with runner(share) -> array
    [len(share), ...] and returns the whole sweep's array [len(caps), ...] on
    every rank (one all_gather of the shares at the end)."""
    import torch.distributed as dist

    parts = assign([c.nx * c.ny for c in caps], world)
    mine = parts[rank]
    local = runner([caps[i] for i in mine]) if mine else None
    gathered = [None] * world
    if world > 1:
        dist.all_gather_object(gathered, (mine, local), group=group)
    else:
        gathered = [(mine, local)]
    shape = next(np.asarray(v).shape[1:] for idx, v in gathered if idx)
    full = np.zeros((len(caps),) + shape)
    for idx, v in gathered:
        for j, i in enumerate(idx):
            full[i] = v[j]
    return full
