"""Batched snapshots in one graph launch, and the autotuner.

Each batch item must equal the regular FP32 solve of the same context with the
same snapshot and ray offset, bit for bit (results do not depend on the launch
shape), on two consecutive runs with different ray offsets.
"""
import numpy as np
import pytest

from paper_1810_00188_gb300 import autotune, inputs, mcrt

pytestmark = pytest.mark.gpu


def _snapshots():
    kd = inputs.make_kdist(0)
    shapes = [(12, 16, 10), (20, 24, 8), (7, 9, 5)]
    snaps = []
    for k, (nx, ny, nz) in enumerate(shapes):
        grid = inputs.Grid(nx, ny, nz, 4.0, 2.0, 2.0, eps_wall=(0.8, 1.0), T_wall=(500.0, 1000.0))
        T, x = inputs.channel_fields(grid, 40 + k, x_mode="field")
        snaps.append((grid, T, x))
    return kd, snaps


def test_batch_matches_single_solves_bitwise_on_two_runs():
    import torch
    kd, snaps = _snapshots()
    solvers, outs, items = [], [], []
    for k, (grid, T, x) in enumerate(snaps):
        S = mcrt.Solver(grid, kd)
        S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
        q = torch.full(grid.shape, float("nan"), dtype=torch.float64, device="cuda")
        s = torch.full_like(q, float("nan"))
        solvers.append(S)
        outs.append((q, s))
        items.append((S.ctx, q.data_ptr(), s.data_ptr(), 10 + k))
    rays = 300
    params = mcrt.Solver.params(rays=rays, seed=7, precision=mcrt.MCRT_FP32)
    stream = torch.cuda.current_stream().cuda_stream
    for weights, streams, offsets in (([1.0, 2.0, 0.5], 3, (0, 5000)), (None, 2, (700,)), (None, 1, (0,))):
        b = mcrt.mcrt_batch_create(items, params, weights=weights, streams=streams)
        try:
            _check_runs(b, snaps, solvers, outs, rays, stream, offsets)
        finally:
            mcrt.mcrt_batch_destroy(b)
    for S in solvers:
        S.close()


def _check_runs(b, snaps, solvers, outs, rays, stream, offsets):
    if True:
        for offset in offsets:
            mcrt.mcrt_batch_run(b, offset, stream)
            st = mcrt.mcrt_batch_get_stats(b)
            assert st["rays"] == sum(g.ncells for g, _, _ in snaps) * rays
            # one trace launch, the long-ray march and one reduction for all snapshots
            assert st["launches"] == 3
            for k, (S, (q, s)) in enumerate(zip(solvers, outs)):
                qr, sr = S.solve(rays=rays, seed=7, snapshot=10 + k, ray_offset=offset,
                                 precision=mcrt.MCRT_FP32)
                assert np.array_equal(q.cpu().numpy(), qr), (offset, k)
                assert np.array_equal(s.cpu().numpy(), sr), (offset, k)


def _run_and_compare(items_spec, params_kw, rays, offsets=(0, 3000)):
    """Batch of (grid, kd, T, x, cell proposal or None) items against single
    solves of the same contexts, bitwise, on consecutive runs."""
    import torch
    solvers, outs, items = [], [], []
    for k, (grid, kd, T, x, prop) in enumerate(items_spec):
        S = mcrt.Solver(grid, kd)
        S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
        if prop is not None:
            S.set_cell_proposal_probs(prop)
        q = torch.full(grid.shape, float("nan"), dtype=torch.float64, device="cuda")
        s = torch.full_like(q, float("nan"))
        solvers.append(S)
        outs.append((q, s))
        items.append((S.ctx, q.data_ptr(), s.data_ptr(), 20 + k))
    params = mcrt.Solver.params(rays=rays, seed=9, precision=mcrt.MCRT_FP32, **params_kw)
    stream = torch.cuda.current_stream().cuda_stream
    b = mcrt.mcrt_batch_create(items, params, streams=2)
    try:
        for offset in offsets:
            mcrt.mcrt_batch_run(b, offset, stream)
            st = mcrt.mcrt_batch_get_stats(b)
            assert st["rays"] == sum(sp[0].ncells for sp in items_spec) * rays
            for k, (S, (q, s)) in enumerate(zip(solvers, outs)):
                qr, sr = S.solve(rays=rays, seed=9, snapshot=20 + k, ray_offset=offset,
                                 precision=mcrt.MCRT_FP32, **params_kw)
                assert np.array_equal(q.cpu().numpy(), qr), (offset, k)
                assert np.array_equal(s.cpu().numpy(), sr), (offset, k)
        launches = st["launches"]
    finally:
        mcrt.mcrt_batch_destroy(b)
    for S in solvers:
        S.close()
    return launches


def test_single_launch_batch_multigrid_stretched_and_cell_proposal():
    """Snapshots sharing the k-distribution run as one trace launch, the
    long-ray march and one reduction (3 launches; the multigrid march hands no
    ray off: 2), also with a stretched snapshot and with per-cell proposals."""
    import torch
    kd = inputs.make_kdist(0)
    spec = []
    for k, (nx, ny, nz) in enumerate([(24, 24, 12), (12, 16, 8), (16, 24, 16)]):
        grid = inputs.Grid(nx, ny, nz, 4.0, 2.0, 2.0, eps_wall=(0.8, 1.0), T_wall=(500.0, 1000.0),
                           reflect=k % 2)
        if k == 2:
            grid.yf = inputs.channel_faces(ny, 2.0, 1.5)
        T, x = inputs.channel_fields(grid, 60 + k, x_mode="field")
        spec.append((grid, kd, T, x, None))
    assert _run_and_compare(spec, {}, 150) == 3
    assert _run_and_compare(spec, dict(mg_levels=2, mg_steps=3), 150) == 2
    K = kd.n_bands * kd.n_g
    g = torch.Generator(device="cpu").manual_seed(3)
    spec_c = []
    for grid, kd_, T, x, _ in spec:
        qp = torch.rand((grid.ncells, K + 2), generator=g) ** 4 + 1e-3
        qp[:, :K] /= qp[:, :K].sum(dim=1, keepdim=True)
        qp[:, K] = 0.2 + 0.6 * torch.rand(grid.ncells, generator=g)
        spec_c.append((grid, kd_, T, x, qp.float().cuda()))
    assert _run_and_compare(spec_c, dict(proposal=mcrt.MCRT_PROPOSAL_CELL), 120) == 3


def test_mixed_kdist_batch_uses_per_snapshot_launches():
    kds = [inputs.make_kdist(0), inputs.make_kdist(1)]
    spec = []
    for k, (nx, ny, nz) in enumerate([(12, 16, 10), (20, 24, 8)]):
        grid = inputs.Grid(nx, ny, nz, 4.0, 2.0, 2.0, eps_wall=(0.8, 1.0), T_wall=(500.0, 1000.0))
        T, x = inputs.channel_fields(grid, 70 + k, x_mode="field")
        spec.append((grid, kds[k], T, x, None))
    assert _run_and_compare(spec, {}, 130) >= 4


def test_batch_rejects_bad_items():
    import torch
    kd, snaps = _snapshots()
    grid, T, x = snaps[0]
    S = mcrt.Solver(grid, kd)
    q = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    params = mcrt.Solver.params(rays=8, precision=mcrt.MCRT_FP32)
    with pytest.raises(mcrt.McrtError) as e:  # no fields yet
        mcrt.mcrt_batch_create([(S.ctx, q.data_ptr(), None, 0)], params)
    assert e.value.status == mcrt.MCRT_E_STATE
    S.set_fields(T, x)
    with pytest.raises(mcrt.McrtError):  # same context twice
        mcrt.mcrt_batch_create([(S.ctx, q.data_ptr(), None, 0), (S.ctx, q.data_ptr(), None, 1)], params)
    with pytest.raises(mcrt.McrtError):  # FP64 is not batched
        mcrt.mcrt_batch_create([(S.ctx, q.data_ptr(), None, 0)],
                               mcrt.Solver.params(rays=8, precision=mcrt.MCRT_FP64))
    S.close()


def test_autotuner_picks_a_shape_without_changing_results():
    import torch
    grid, kd, T, x = inputs.nongrey_channel(24, 24, 24, seed=2)
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    q = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    s = torch.zeros_like(q)
    params = S.params(rays=200, seed=3, precision=mcrt.MCRT_FP32)
    S.solve_into(params, q, s)
    before = q.cpu().numpy().copy()
    best, table = autotune.tune_solver(S, params, q, s, reps=2)
    assert best in table and all(v > 0 for v in table.values())
    assert S.tuning()["min_blocks_per_sm"] == best[0] and S.tuning()["steps_per_round"] == best[1]
    S.solve_into(params, q, s)
    assert np.array_equal(q.cpu().numpy(), before)
    S.close()
