"""Sharding a batch of loops across ranks (one process per GPU).

The loops of a batch are independent problems, so a multi-GPU descent needs no collective on
its data path: every rank descends its own subset and the results are gathered once at the
end.  Loops are assigned longest-processing-time first (cost = Ns * Nx per tau-step), which
keeps the ranks' step times within one loop's cost of each other.
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np


def partition(ns: Sequence[int], nx: int, world: int) -> List[List[int]]:
    """Loop indices for each rank: longest loops first, each to the least loaded rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(ns)), key=lambda b: (-ns[b], b))
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda i: (load[i], i))
        parts[r].append(b)
        load[r] += int(ns[b]) * int(nx)
    for p in parts:
        p.sort()
    return parts


def local_batch(u_packed: np.ndarray, ns: Sequence[int], nx: int, T: Sequence[float],
                idx: Sequence[int]):
    """The packed grid field and periods of the loops `idx` (in that order)."""
    offs = np.concatenate([[0], np.cumsum([n * nx for n in ns])])
    u = np.concatenate([u_packed[offs[b]:offs[b + 1]] for b in idx]) if idx else np.zeros(0)
    return u, np.asarray([T[b] for b in idx], dtype=np.float64), [ns[b] for b in idx]


def scatter_back(results: Dict[int, dict], ns: Sequence[int], nx: int):
    """Reassemble per-loop results {b: {"u": grid [Ns_b*Nx], "T": float, ...}} in batch order."""
    B = len(ns)
    missing = [b for b in range(B) if b not in results]
    if missing:
        raise ValueError(f"loops without a result: {missing}")
    u = np.concatenate([np.asarray(results[b]["u"]).ravel() for b in range(B)])
    T = np.asarray([results[b]["T"] for b in range(B)], dtype=np.float64)
    return u, T


def gather(results: Dict[int, dict], group=None) -> Dict[int, dict]:
    """All ranks' per-loop results on every rank (one all_gather_object at the end)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    bag = [None] * world
    dist.all_gather_object(bag, results, group=group)
    out: Dict[int, dict] = {}
    for part in bag:
        for b, v in part.items():
            if b in out:
                raise ValueError(f"loop {b} descended on two ranks")
            out[b] = v
    return out
