"""Host-side logic of the multi-GPU path: independent units per rank, no collective on the data path.

k-points and systems share nothing (§5.3 notes the trivial parallelism in k), so N GPUs run
independent work: each rank takes a share of the (system, k-point) units, chosen by a greedy
longest-processing-time assignment on an estimated cost, and the only communication is the
timing barrier and two scalar reductions (the slowest rank's time, the work all ranks did).

The process group is the caller's (NCCL on GPUs; the functions take any torch.distributed group,
so the logic is tested with gloo on CPU).
"""
from __future__ import annotations

import heapq
from typing import List, Optional, Sequence


def unit_cost(npw: int, nband: int, degree: int) -> float:
    """Estimated cost of one ChebFi iteration of a unit: the block applications of the filter plus
    H on the filtered block (npw * nb * (degree + 1)) and the Rayleigh-Ritz eigensolve (nb^3)."""
    nb = nband + max(4, (nband + 9) // 10)
    return float(npw) * nb * (degree + 1) + float(nb) ** 3


def npw_estimate(volume: float, ecut: float) -> float:
    """Plane waves in the sphere 1/2 |k+G|^2 <= Ecut, to leading order: the sphere's volume
    (4 pi / 3)(2 Ecut)^(3/2) over the reciprocal cell's (2 pi)^3 / Omega."""
    return volume * (2.0 * ecut) ** 1.5 / (6.0 * 3.141592653589793 ** 2)


def lpt_partition(costs: Sequence[float], nranks: int) -> List[List[int]]:
    """Greedy longest-processing-time assignment: units in decreasing cost order, each to the rank
    with the least total so far (ties to the lower rank).  Returns the unit indices of every rank,
    each list in increasing index order.  Deterministic, so every rank computes the same answer
    without communicating."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(nranks)]
    heapq.heapify(heap)
    share: List[List[int]] = [[] for _ in range(nranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        share[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(s) for s in share]


def max_over_ranks(x: float, dist=None, device: Optional[str] = None) -> float:
    """The largest x over the ranks of the default group (x itself without a group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist=None, device: Optional[str] = None) -> float:
    """The sum of x over the ranks of the default group (x itself without a group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_done: float, seconds: float, dist=None, device: Optional[str] = None) -> float:
    """Whole-job throughput: the units every rank processed divided by the slowest rank's time."""
    total = sum_over_ranks(units_done, dist, device)
    slowest = max_over_ranks(seconds, dist, device)
    return total / slowest if slowest > 0 else 0.0


def gather_results(mine: dict, dist=None) -> dict:
    """Union of every rank's per-unit results ({unit index: result}) on every rank (the rank's own
    dict without a group).  The units are disjoint by construction (lpt_partition), so a unit seen
    twice is an error."""
    if dist is None:
        return dict(mine)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, dict(mine))
    out = {}
    for part in parts:
        for u, r in part.items():
            if u in out:
                raise ValueError(f"unit {u} was processed by two ranks")
            out[u] = r
    return out
