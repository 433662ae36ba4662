"""Sharding a batch of spatial cells over ranks (one process per GPU).

Cells of the space-homogeneous operator are independent, so ranks share no data: each rank
evaluates its own cells and nothing is exchanged on the data path.  Two layouts are used:

* weak scaling: every rank owns a batch of its own (the benchmark's default);
* strong scaling: one global batch is split by ``partition``, which balances the work, counted
  as N^d log2(N^d) per cell (the transforms dominate), with the longest-processing-time-first
  rule: cells in decreasing cost, each to the rank with the least work so far.  The heaviest
  rank then carries at most 4/3 of the optimum (Graham's bound).

``allreduce_diagnostics`` sums per-rank totals of the FP64 diagnostics (mass, momentum, energy,
entropy, entropy production) when a global figure is wanted; it is not on the data path.
"""
from __future__ import annotations

import math

import numpy as np


def cell_cost(N: int, d: int = 3) -> float:
    """Relative work of one cell: N^d log2(N^d)."""
    m = float(N) ** d
    return m * math.log2(m)


def partition(Ns, world: int, d: int = 3):
    """Split cell indices 0..len(Ns)-1 over ``world`` ranks; returns one sorted index array per rank.

    Deterministic: every rank computes the same split from the same sizes, so no exchange is
    needed to agree on it.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    Ns = np.asarray(Ns)
    costs = np.array([cell_cost(int(n), d) for n in Ns])
    order = sorted(range(len(Ns)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    owned = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owned[r].append(i)
        load[r] += costs[i]
    return [np.array(sorted(o), dtype=np.int64) for o in owned]


def loads(Ns, parts, d: int = 3):
    """Work per rank of a partition."""
    return [float(sum(cell_cost(int(Ns[i]), d) for i in p)) for p in parts]


def allreduce_diagnostics(diag):
    """Global sums over ranks of the per-cell diagnostics ``diag`` [cells, EF_DIAG_STRIDE] (FP64):
    mass, momentum, energy, entropy and entropy production are summed over the rank's cells, then
    over ranks; the minimum of F (column 7) and of the output (column 9) and the maximum loss
    frequency (column 8) are reduced with min / max.  Without an initialised process group it
    reduces the local cells only."""
    import torch

    d = diag if isinstance(diag, torch.Tensor) else torch.as_tensor(diag, dtype=torch.float64)
    sums = d[:, :7].sum(dim=0)
    mins = torch.stack([d[:, 7].min(), d[:, 9].min()])
    maxs = d[:, 8].max().reshape(1)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(sums, op=dist.ReduceOp.SUM)
        dist.all_reduce(mins, op=dist.ReduceOp.MIN)
        dist.all_reduce(maxs, op=dist.ReduceOp.MAX)
    out = torch.zeros(d.shape[1], dtype=d.dtype, device=d.device)
    out[:7] = sums
    out[7] = mins[0]
    out[8] = maxs[0]
    out[9] = mins[1]
    return out
