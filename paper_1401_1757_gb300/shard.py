"""Partitioning of policy x scenario chains across ranks (one process per GPU).

Chains are independent (the paper's own decomposition is by policy, Section
5.1.1), so ranks exchange no data on the compute path.  Two splits:

* ``scenario_shard``: contiguous scenario ranges; every rank values the whole
  portfolio under its own scenarios, so per-scenario totals are complete on
  the owning rank and nothing is reduced.
* ``policy_shard``: policies dealt to ranks balanced by projection length
  (sum of steps, longest first); per-scenario totals are then partial sums
  that the caller adds up once at the end.
"""
from __future__ import annotations

import heapq

import numpy as np


def scenario_shard(n_scen: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of the scenarios owned by ``rank`` (sizes differ by at most one)."""
    if not (0 <= rank < world):
        raise ValueError("rank outside [0, world)")
    base, extra = divmod(n_scen, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def policy_shard(steps, world: int) -> list[np.ndarray]:
    """Policy indices per rank, greedy longest-first onto the least-loaded rank."""
    steps = np.asarray(steps, dtype=np.int64)
    order = np.argsort(-steps, kind="stable")
    heap = [(0, r) for r in range(world)]
    owned = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        owned[r].append(int(i))
        heapq.heappush(heap, (load + int(steps[i]), r))
    return [np.sort(np.asarray(o, dtype=np.int64)) for o in owned]
