"""Host-side multi-GPU plumbing: shard plans and cross-rank aggregation.

Q_i depends only on the rays leaving cell i (the domain parallelisation of the
paper's Section 3; Section 5 gives every GPU the whole temperature field and
each its own subdomain of emitting cells).  A shard is therefore an emitting
box; no exchange happens during a solve.  torch.distributed is plumbing here:
one barrier and two scalar reductions for timing.
"""
from __future__ import annotations


def shard_boxes(nx: int, ny: int, nz: int, world: int):
    """Contiguous z-slab boxes (i0, i1, j0, j1, k0, k1), one per rank, covering
    the grid exactly once; slabs differ in thickness by at most one cell (a rank
    may get an empty box when world > nz)."""
    boxes = []
    for r in range(world):
        k0 = (nz * r) // world
        k1 = (nz * (r + 1)) // world
        boxes.append((0, nx, 0, ny, k0, k1))
    return boxes


def aggregate(local_units: float, local_seconds: float, device=None):
    """(sum of units over ranks, max of seconds over ranks) -- the whole-job
    throughput is the first divided by the second."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_units), float(local_seconds)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())
