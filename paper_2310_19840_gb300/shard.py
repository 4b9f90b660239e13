"""Splitting one batch of realisations over several GPUs (host logic only).

The members of a batch are independent problems (each random-sea realisation
is integrated on its own), so a batch shards across GPUs with no exchange
inside a step: every rank advances a subset of the members with its own
library context, and only the per-member invariants are gathered at the end.

The cost of a member is taken as the work of its transforms, n log2 n for
n = nx * ny points.  ``partition`` assigns members greedily, largest first,
each to the rank with the smallest load so far (the longest-processing-time
rule), which keeps every rank's load within one member's cost of every
other's.  ``gather_invariants`` sums a per-member table of (mass, energy) over
the ranks with one all-reduce of FP64 values, each rank having filled in only
the rows of its own members.
"""
from __future__ import annotations

import math


def member_cost(nx: int, ny: int) -> float:
    """Transform work of one member of nx x ny points: n log2 n."""
    n = nx * ny
    return n * math.log2(n) if n > 1 else 1.0


def partition(shapes, world: int):
    """Member indices per rank for members of the given (nx, ny) shapes.

    Largest cost first (ties in member order), each into the currently
    lightest rank (ties to the lowest rank); the lists come back sorted."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = [member_cost(nx, ny) for nx, ny in shapes]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(m) for m in out]


def rank_loads(shapes, parts):
    """Total cost per rank of a partition."""
    return [sum(member_cost(*shapes[i]) for i in p) for p in parts]


def gather_invariants(n_members: int, local: dict, world: int, device=None):
    """(mass, energy) of every member as an (n_members, 2) float64 array, from
    each rank's {member: (mass, energy)} of its own members (one all-reduce)."""
    import numpy as np
    import torch
    t = torch.zeros((n_members, 2), dtype=torch.float64, device=device)
    for i, (m, e) in local.items():
        t[i, 0] = m
        t[i, 1] = e
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return np.asarray(t.cpu().numpy())
