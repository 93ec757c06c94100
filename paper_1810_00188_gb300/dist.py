"""Host-side multi-GPU plumbing: shard plans, the field broadcast, the gather of
the per-shard results and cross-rank aggregation.

Q_i depends only on the rays leaving cell i (the domain parallelisation of the
paper's Section 3; Section 5 gives every GPU the whole temperature field and
each its own subdomain of emitting cells).  A shard is therefore an emitting
box; no exchange happens during a solve.  The collectives are the two the paper's
Section 5 layout implies: one broadcast of the {T, x} field before the solve and
one gather of the Q and sigma slabs after it.  Independent snapshots (batches)
split across ranks with no collective at all.  torch.distributed is plumbing
here (NCCL on GPUs, gloo on CPU).
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


def split_snapshots(cells, world: int):
    """Snapshots of a batch (their cell counts, the work of each at equal rays per
    cell) assigned to ranks: largest first, each to the least-loaded rank (ties to
    the lowest rank).  Returns one list of snapshot indices per rank, each in
    decreasing order of work; every snapshot appears exactly once.  The largest
    load exceeds the mean by less than the largest snapshot."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i))
    loads = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += int(cells[i])
    return parts


def _dist():
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return None
    return dist


def broadcast_fields(T, x=None, src: int = 0):
    """Every rank leaves with rank src's T (and x) field.  T and x are torch
    tensors of the same shape and dtype on every rank (their contents matter on
    src only); they are overwritten in place and returned.  T and x of one dtype
    travel as one buffer (one collective)."""
    import torch
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return T, x
    if x is None or x.dtype != T.dtype:
        dist.broadcast(T, src=src)
        if x is not None:
            dist.broadcast(x, src=src)
        return T, x
    buf = torch.cat([T.reshape(-1), x.reshape(-1)])
    dist.broadcast(buf, src=src)
    n = T.numel()
    T.copy_(buf[:n].view_as(T))
    x.copy_(buf[n:].view_as(x))
    return T, x


def gather_slabs(parts, boxes, shape, dst: int = 0):
    """The z-slab results of every rank assembled on rank dst.

    parts: this rank's tensors (e.g. Q and sigma), each [k1-k0, ny, nx] for its
    box in `boxes` (shard_boxes of the full grid).  Slabs may differ in thickness,
    so each travels padded to the thickest; one gather per tensor.  Returns the
    full [nz, ny, nx] tensors on dst and None elsewhere."""
    import torch
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return [p.reshape(shape) for p in parts]
    world, rank = dist.get_world_size(), dist.get_rank()
    kmax = max(b[5] - b[4] for b in boxes)
    nz, ny, nx = shape
    out = []
    for p in parts:
        pad = torch.zeros((kmax, ny, nx), dtype=p.dtype, device=p.device)
        pad[:p.shape[0]] = p
        lst = [torch.empty_like(pad) for _ in range(world)] if rank == dst else None
        dist.gather(pad, lst, dst=dst)
        if rank == dst:
            full = torch.empty((nz, ny, nx), dtype=p.dtype, device=p.device)
            for r, b in enumerate(boxes):
                full[b[4]:b[5]] = lst[r][:b[5] - b[4]]
            out.append(full)
    return out if rank == dst else None


def solve_sharded(solve_box, T, x, shape, src: int = 0):
    """A strong-scaling solve of one field over all ranks (Section 5's layout).

    The field is broadcast from rank src, every rank solves its z-slab with
    solve_box(T, x, box) -> (q, sigma) tensors of the box's shape, and the slabs
    are gathered on rank src.  Returns (q, sigma) of the whole grid on src and
    None elsewhere.  Because every cell's estimate depends only on its own rays,
    the result equals a single-rank solve bit for bit."""
    dist = _dist()
    world = 1 if dist is None else dist.get_world_size()
    rank = 0 if dist is None else dist.get_rank()
    nz, ny, nx = shape
    T, x = broadcast_fields(T, x, src=src)
    boxes = shard_boxes(nx, ny, nz, world)
    q, s = solve_box(T, x, boxes[rank])
    return gather_slabs([q, s], boxes, shape, dst=src)


def aggregate(local_units: float, local_seconds: float, device=None):
    """(sum of units over ranks, max of seconds over ranks) -- the whole-job
    throughput is the first divided by the second."""
    import torch
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return float(local_units), float(local_seconds)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())
