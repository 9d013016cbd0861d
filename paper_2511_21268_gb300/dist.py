"""Sharding of independent systems across ranks (one process per GPU).

A batch of independent systems (the 48 uneven 2-D instances of the batched
workload, or any list of SPD systems) has no coupling between systems, so it
shards with no collective on the data path: each rank builds one
block-diagonal batch hierarchy (amg_setup_batch) of its share and solves it;
only the results (and timings) are gathered at the end.

Assignment: systems sorted by stored entries (descending, index ascending on
ties), each given to the rank with the fewest stored entries so far (lowest
rank on ties) -- a deterministic greedy balance of the per-rank matrix
traffic, which is what the batch solve's time follows.
"""
from __future__ import annotations


def assign_by_nnz(nnz: list[int], world: int) -> list[list[int]]:
    """Indices of the systems each rank solves (ascending within a rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for k in sorted(range(len(nnz)), key=lambda k: (-int(nnz[k]), k)):
        r = min(range(world), key=lambda r: (load[r], r))
        out[r].append(k)
        load[r] += int(nnz[k])
    return [sorted(ix) for ix in out]


def solve_sharded(systems, rhs, solve_shard, rank: int, world: int, dist=None):
    """Solve the share of `systems` that belongs to `rank` and gather every
    system's result on every rank.

    systems: list of (rowptr, col, val) per system; rhs: list of F.
    solve_shard(systems_part, rhs_part) -> list of per-system results (any
    picklable objects, e.g. dicts with u / iters / relres), called once with
    this rank's share (possibly empty).  dist: torch.distributed (initialised)
    or None for world = 1.  Returns the results of all systems in the
    original order.
    """
    parts = assign_by_nnz([len(s[2]) for s in systems], world)
    mine = parts[rank]
    local = solve_shard([systems[k] for k in mine], [rhs[k] for k in mine]) if mine else []
    if len(local) != len(mine):
        raise RuntimeError("solve_shard returned a result count different from its share")
    if world == 1:
        gathered = [list(zip(mine, local))]
    else:
        gathered = [None] * world
        dist.all_gather_object(gathered, list(zip(mine, local)))
    out = [None] * len(systems)
    for part in gathered:
        for k, res in part:
            out[k] = res
    if any(r is None for r in out):
        raise RuntimeError("a system was solved by no rank")
    return out
