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


def test_split_snapshots_covers_once_and_balances():
    from paper_1810_00188_gb300.dist import split_snapshots
    rng = np.random.default_rng(4)
    sizes = [32**3, 48 * 64 * 48, 96**3, 128**3]
    for world in (1, 2, 3, 8):
        cells = [sizes[i] for i in rng.integers(0, 4, 32)]
        parts = split_snapshots(cells, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(32))
        loads = [sum(cells[i] for i in p) for p in parts]
        assert max(loads) - sum(cells) / world < max(cells)
        for p in parts:
            assert all(cells[a] >= cells[b] for a, b in zip(p, p[1:]))
    assert split_snapshots([], 2) == [[], []]
    assert split_snapshots([5], 3) == [[0], [], []]


def _sharded_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1810_00188_gb300 import dist as pdist
    from paper_1810_00188_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grid, kd, T, x = inputs.nongrey_channel(6, 6, 5, seed=3, x_mode="field")
        # only rank 0 holds the field; the others receive it
        Tt = torch.tensor(T) if rank == 0 else torch.zeros(grid.shape, dtype=torch.float64)
        xt = torch.tensor(x) if rank == 0 else torch.zeros(grid.shape, dtype=torch.float64)

        def solve_box(Tb, xb, box):
            r = oracle.solve(grid, kd, Tb.numpy(), xb.numpy(), rays=16, seed=2, box=box, nthreads=1)
            return torch.tensor(r["q"]), torch.tensor(r["sigma"])

        res = pdist.solve_sharded(solve_box, Tt, xt, grid.shape)
        if rank == 0:
            out.put((res[0].numpy(), res[1].numpy()))
        else:
            assert res is None
            assert np.array_equal(Tt.numpy(), T) and np.array_equal(xt.numpy(), x)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_three_gloo_ranks_broadcast_solve_and_gather_uneven_slabs():
    import oracle
    from paper_1810_00188_gb300 import inputs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 3, port, q)) for r in range(3)]
    for p in procs:
        p.start()
    qs, ss = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    grid, kd, T, x = inputs.nongrey_channel(6, 6, 5, seed=3, x_mode="field")
    full = oracle.solve(grid, kd, T, x, rays=16, seed=2, nthreads=1)
    # slabs of 1, 2 and 2 z-planes, padded in transit; the union is the full solve
    assert np.array_equal(qs, full["q"]) and np.array_equal(ss, full["sigma"])


def test_bench_starts_one_rank_per_gpu_when_asked():
    """`bench.py --gpus 2` outside a launcher starts two ranks itself (torch's
    launcher, 127.0.0.1); on the reference arm rank 0 alone runs the oracle and
    prints the one JSON line with n_gpus = 2, and the other rank exits 0.  A
    launcher whose world size differs from --gpus is refused."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0", "--n", "6", "--rays", "4"],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["config"]["parallelism"].startswith("weak") and "(2)" in line["config"]["parallelism"]
    bad = dict(env, WORLD_SIZE="3", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0", "--n", "6", "--rays", "4"],
                       capture_output=True, text=True, env=bad, timeout=600)
    assert r.returncode != 0 and "launcher started 3 ranks" in r.stderr
