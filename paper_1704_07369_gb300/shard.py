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

The spatially inhomogeneous coupling (cells as the points of a periodic 1D spatial grid, upwind
transport between neighbours) is the one place where ranks do exchange data: each rank owns a
contiguous block of cells (``spatial_blocks``) stored with one halo cell at each end, and before
every transport step ``halo_exchange`` sends its first cell to the left neighbour rank and its
last cell to the right one (periodic over ranks).  ``lie_steps_sharded`` drives the split steps.
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


def spatial_blocks(ncells: int, world: int):
    """Contiguous blocks of a periodic 1D spatial grid of ``ncells`` cells over ``world`` ranks, in
    rank order: a list of (first cell, cell count), counts differing by at most one."""
    if world < 1 or ncells < world:
        raise ValueError("need 1 <= world <= ncells")
    base, extra = divmod(ncells, world)
    out, start = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((start, n))
        start += n
    return out


def halo_exchange(F_ext, group=None):
    """Fill the halo cells of a rank's block ``F_ext`` ([n + 2, ...]: F_ext[1..n] the rank's cells in
    spatial order, F_ext[0] and F_ext[n + 1] the halos) with the neighbouring ranks' boundary cells:
    the left halo gets the left rank's last cell, the right halo the right rank's first cell,
    periodically over ranks.  One rank (or no process group) wraps onto itself.  Point-to-point
    messages, two sends and two receives per rank; on the GPU they go through NCCL, on the host
    through gloo."""
    import torch.distributed as dist
    n = F_ext.shape[0] - 2
    if n < 1:
        raise ValueError("a block needs at least one cell besides its two halos")
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    if world == 1:
        F_ext[0].copy_(F_ext[n])
        F_ext[n + 1].copy_(F_ext[1])
        return
    rank = dist.get_rank(group)
    left, right = (rank - 1) % world, (rank + 1) % world
    if group is not None:
        left, right = dist.get_global_rank(group, left), dist.get_global_rank(group, right)
    # send order (to the left, to the right) and receive order (from the right, from the left)
    # pair up message by message even when left == right (two ranks)
    reqs = [dist.isend(F_ext[1].contiguous(), left, group=group, tag=0),
            dist.isend(F_ext[n].contiguous(), right, group=group, tag=1)]
    rbuf, lbuf = F_ext[n + 1], F_ext[0]
    reqs.append(dist.irecv(rbuf, right, group=group, tag=0))
    reqs.append(dist.irecv(lbuf, left, group=group, tag=1))
    for q in reqs:
        q.wait()


def lie_steps_sharded(F_ext, scratch_ext, nsteps: int, transport, collide, group=None):
    """Lie splitting over a rank's block with halos.  ``F_ext`` and ``scratch_ext`` are [n + 2, ...];
    each step exchanges the halos of the current buffer, ``transport(cur, other)`` writes all
    n + 2 cells of the other buffer (the two halo outputs are never used), ``collide(view)``
    updates the interior other[1 .. n] in place, and the buffers swap.  Returns the buffer that
    holds the state."""
    a, b = F_ext, scratch_ext
    for _ in range(int(nsteps)):
        halo_exchange(a, group)
        transport(a, b)
        collide(b[1:-1])
        a, b = b, a
    return a
