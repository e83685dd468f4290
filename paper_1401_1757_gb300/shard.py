"""Partitioning of policy x scenario chains across ranks (one process per GPU).

Chains are independent (the paper's own decomposition is by policy, Section
5.1.1; Section 6 proposes many GPUs the same way).  Two splits:

* ``policy_shard`` / ``PolicyPartition``: policies dealt to ranks balanced by
  projection length (sum of steps, longest first); every rank values its
  policies under the same scenario set, and the one exchange is a sum of the
  per-scenario FP64 portfolio totals over the ranks (``reduce_totals``).
* ``scenario_shard``: contiguous scenario ranges; every rank values the whole
  portfolio under its own scenarios, so per-scenario totals are complete on
  the owning rank and nothing is reduced.  The same split serves the outer
  paths of a nested valuation: each rank passes its range's first index as
  ``outer_first`` (the paths' random streams are keyed by the global index),
  and every node statistic is complete on the rank that owns the path.
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


def projection_steps(pol: dict, n_ages: int = 1440, horizon: int = 0) -> np.ndarray:
    """Steps S_p of each record as the library counts them for the products
    0-3 (single-life annuity to the table's end, the reversionary annuity to
    the younger life's, assurances their term), capped by ``horizon``."""
    prod, a1, a2, term = pol["product"], pol["age1_m"], pol["age2_m"], pol["term_m"]
    S = np.where(prod == 0, np.maximum(0, n_ages - a1),
                 np.where(prod == 1, np.maximum(0, n_ages - np.minimum(a1, a2)), term))
    S = np.where((prod <= 1) & (term > 0), np.minimum(S, term), S)
    if horizon > 0:
        S = np.minimum(S, horizon)
    return S.astype(np.int64)


class PolicyPartition:
    """One rank's share of a portfolio, balanced by the sum of projection
    steps, and the exchange step that follows the valuation: the per-scenario
    portfolio totals of the ranks are partial sums, added by one FP64 sum
    over the ranks (``torch.distributed.all_reduce``, NCCL on GPUs or gloo on
    host tensors)."""

    def __init__(self, steps, world: int, rank: int):
        if not (0 <= rank < world):
            raise ValueError("rank outside [0, world)")
        self.world, self.rank = world, rank
        self.idx = policy_shard(steps, world)[rank]

    def take(self, pol: dict) -> dict:
        """The records this rank values."""
        return {k: np.ascontiguousarray(v[self.idx]) for k, v in pol.items()}

    def reduce_totals(self, totals, dist=None):
        """Sum the per-scenario FP64 totals (a torch tensor) over the ranks in place."""
        if self.world > 1:
            import torch
            if totals.dtype != torch.float64:
                raise ValueError("the totals are summed in FP64")
            dist.all_reduce(totals)
        return totals
