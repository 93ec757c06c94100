"""The N>1 host path on CPU: two gloo ranks (no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1810_00188_gb300.dist import shard_boxes


def test_shard_boxes_cover_the_grid_once():
    for nz, world in ((64, 1), (64, 2), (64, 8), (7, 3), (3, 8)):
        boxes = shard_boxes(16, 8, nz, world)
        assert len(boxes) == world
        owner = np.zeros(nz, dtype=int)
        for b in boxes:
            assert b[:4] == (0, 16, 0, 8) and b[4] <= b[5]
            owner[b[4]:b[5]] += 1
        assert np.all(owner == 1)
        sizes = [b[5] - b[4] for b in boxes]
        assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle
    from paper_1810_00188_gb300 import dist as pdist
    from paper_1810_00188_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # aggregation: units summed, time maxed over ranks
        units, secs = pdist.aggregate(10.0 * (rank + 1), 1.0 + rank)
        # each rank solves its shard of the same field; gather the shards
        grid, kd, T, x = inputs.nongrey_channel(6, 6, 5, seed=3)
        box = pdist.shard_boxes(grid.nx, grid.ny, grid.nz, world)[rank]
        res = oracle.solve(grid, kd, T, x, rays=16, seed=2, box=box, nthreads=1)
        parts = [None] * world
        dist.all_gather_object(parts, res["q"])
        if rank == 0:
            out.put((units, secs, np.concatenate(parts, axis=0)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_shard():
    import oracle
    from paper_1810_00188_gb300 import inputs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    units, secs, q_sharded = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert units == 30.0 and secs == 2.0
    grid, kd, T, x = inputs.nongrey_channel(6, 6, 5, seed=3)
    full = oracle.solve(grid, kd, T, x, rays=16, seed=2, nthreads=1)
    assert np.array_equal(q_sharded, full["q"])
