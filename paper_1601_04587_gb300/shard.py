"""Sharding of independent domain solves across ranks (one process per GPU).

Every unit of the hot path — a domain propagator, a level-1 variant of a
region, a serving request — is an independent Dirichlet problem: there is
no halo exchange between domains, so ranks share nothing while they solve.
Units are assigned by estimated cost (longest first, to the least-loaded
rank, ties by index: deterministic), each rank solves its own, and the
per-unit results (small: correlators or trace vectors) are gathered once and
merged in unit order, so the merged result does not depend on the number of
ranks.
"""
from __future__ import annotations


def solve_cost(n_sites: int, ncol: int = 12, iterations: float = 1.0) -> float:
    """Cost model of a unit: site-columns times expected iterations."""
    return float(n_sites) * float(ncol) * float(iterations)


def partition(costs, world: int):
    """Greedy longest-processing-time assignment: list of unit indices per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    loads = [0.0] * world
    assign = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        assign[r].append(i)
        loads[r] += float(costs[i])
    return [sorted(a) for a in assign]


def run_sharded_batch(units, costs, compute_batch, dist=None):
    """`compute_batch(list_of_units)` -> their results (same order), called once on this
    rank's share (one batched solve per rank); returns the results of all units in
    unit order, gathered from every rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(compute_batch(list(units)))
    world, rank = dist.get_world_size(), dist.get_rank()
    mine = partition(costs, world)[rank]
    res = list(compute_batch([units[i] for i in mine])) if mine else []
    if len(res) != len(mine):
        raise ValueError("compute_batch returned a result count different from its units")
    local = dict(zip(mine, res))
    gathered = [None] * world
    dist.all_gather_object(gathered, local)
    merged = {}
    for part in gathered:
        merged.update(part)
    return [merged[i] for i in range(len(units))]


def run_sharded(units, costs, compute, dist=None):
    """Compute `compute(unit)` for this rank's share and return the results of
    all units in unit order (gathered from every rank)."""
    return run_sharded_batch(units, costs, lambda us: [compute(u) for u in us], dist)
