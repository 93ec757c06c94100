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
    # the per-item form, asked for by items[0]'s tuning: the same bits
    solvers[0].set_tuning(batch_per_snapshot=1)
    assert solvers[0].tuning()["batch_per_snapshot"] == 1
    for streams in (2, 1):
        b = mcrt.mcrt_batch_create(items, params, streams=streams)
        try:
            _check_runs(b, snaps, solvers, outs, rays, stream, (900,), per_item=True)
        finally:
            mcrt.mcrt_batch_destroy(b)
    solvers[0].set_tuning()
    for S in solvers:
        S.close()


def _check_runs(b, snaps, solvers, outs, rays, stream, offsets, per_item=False):
    for offset in offsets:
        mcrt.mcrt_batch_run(b, offset, stream)
        st = mcrt.mcrt_batch_get_stats(b)
        assert st["rays"] == sum(g.ncells for g, _, _ in snaps) * rays
        if per_item:  # a trace launch and a reduction (at least) per snapshot
            assert st["launches"] >= 2 * len(snaps)
        else:  # one trace launch, the long-ray march and one reduction for all snapshots
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


def test_batch_many_rays_per_cell_tally_segments_bitwise():
    """4100 rays per cell: three tally segments per cell.  The batch tallies add
    a cell's segments in one warp (the single launch's reduction, and the
    per-snapshot launches' plain-load tally), the single solves sum each segment
    with a warp of its own and add the segments in a second kernel: the same
    bits."""
    kds = [inputs.make_kdist(0), inputs.make_kdist(1)]
    spec, spec_mixed = [], []
    for k, (nx, ny, nz) in enumerate([(8, 8, 6), (6, 10, 4)]):
        grid = inputs.Grid(nx, ny, nz, 4.0, 2.0, 2.0, eps_wall=(0.8, 1.0), T_wall=(500.0, 1000.0))
        T, x = inputs.channel_fields(grid, 80 + k, x_mode="field")
        spec.append((grid, kds[0], T, x, None))
        spec_mixed.append((grid, kds[k], T, x, None))
    assert _run_and_compare(spec, {}, 4100, offsets=(0,)) == 3
    assert _run_and_compare(spec_mixed, {}, 4100, offsets=(0,)) >= 4


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
    best, table = autotune.tune_solver(S, params, q, s, reps=2, scratch_mib=(1, 64), claim_rays=(64, 65536))
    assert best in table and all(v > 0 for v in table.values())
    assert any(k[2] == 1 for k in table)  # the scratch cap was tried (1 MiB: many chunks)
    assert any(k[3] == 64 for k in table)  # and the claimed runs
    assert S.tuning()["min_blocks_per_sm"] == best[0] and S.tuning()["steps_per_round"] == best[1]
    S.solve_into(params, q, s)
    assert np.array_equal(q.cpu().numpy(), before)
    S.close()


# ---- every snapshot of a batch against the oracle, cell by cell -----------------

def _oracle_batch_check(spec, params_kw, rays, offsets, streams=2, seed=9, snap0=30):
    """Runs the batch of (grid, kd, T, x, counts or None) items and compares every
    snapshot with the FP64 oracle on the same draws (snapshot word snap0 + k, the
    run's ray offset): |Q - Q_oracle| <= 1e-4 S_i, the FP32 tolerance of the
    single-solve parity tests.  Per-cell proposals are host-built integer counts
    given to both sides.  Returns the launches of the last run."""
    import torch

    import oracle
    solvers, outs, items = [], [], []
    for k, (grid, kd, T, x, prop) in enumerate(spec):
        S = mcrt.Solver(grid, kd)
        S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
        if prop is not None:
            S.set_cell_proposal(*prop)
        q = torch.full(grid.shape, float("nan"), dtype=torch.float64, device="cuda")
        s = torch.full_like(q, float("nan"))
        solvers.append(S)
        outs.append((q, s))
        items.append((S.ctx, q.data_ptr(), s.data_ptr(), snap0 + k))
    params = mcrt.Solver.params(rays=rays, seed=seed, precision=mcrt.MCRT_FP32, **params_kw)
    stream = torch.cuda.current_stream().cuda_stream
    b = mcrt.mcrt_batch_create(items, params, streams=streams)
    try:
        for offset in offsets:
            mcrt.mcrt_batch_run(b, offset, stream)
            st = mcrt.mcrt_batch_get_stats(b)
            assert st["rays"] == sum(sp[0].ncells for sp in spec) * rays
            for k, ((grid, kd, T, x, prop), (q, s)) in enumerate(zip(spec, outs)):
                kw = {}
                if prop is not None:
                    nc, nb, ng = grid.ncells, kd.n_bands, kd.n_g
                    kw["proposal"] = (prop[0], prop[1].reshape(nc, nb * ng), prop[2])
                orc = oracle.solve(grid, kd, T, x, rays=rays, seed=seed, snapshot=snap0 + k,
                                   ray_offset=offset, tol=params.tol, max_steps=params.max_steps,
                                   mg_levels=params_kw.get("mg_levels", 1),
                                   mg_steps=params_kw.get("mg_steps", 5), **kw)
                qn = q.cpu().numpy()
                err = np.abs(qn - orc["q"]) / np.maximum(orc["scale"], 1e-300)
                assert np.all(np.isfinite(qn)), (offset, k)
                assert err.max() <= 1e-4, (offset, k, float(err.max()))
                sn = s.cpu().numpy()
                big = orc["sigma"] > 1e-3 * orc["scale"]
                np.testing.assert_allclose(sn[big], orc["sigma"][big], rtol=2e-2)
        launches = st["launches"]
    finally:
        mcrt.mcrt_batch_destroy(b)
    for S in solvers:
        S.close()
    return launches


def _uneven_snapshots(kd, shapes, seed0, stretched=(), reflect=()):
    spec = []
    for k, (nx, ny, nz) in enumerate(shapes):
        grid = inputs.Grid(nx, ny, nz, 4.0, 2.0, 2.0, eps_wall=(0.8, 1.0), T_wall=(500.0, 1000.0),
                           reflect=1 if k in reflect else 0)
        if k in stretched:
            grid.yf = inputs.channel_faces(ny, 2.0, 1.5)
        T, x = inputs.channel_fields(grid, seed0 + k, x_mode="field")
        spec.append((grid, kd, T, x, None))
    return spec


def test_single_launch_batch_against_oracle():
    """Four snapshots of uneven sizes sharing the k-distribution (one persistent
    trace launch): a ragged 7x9x5 grid, a stretched wall-normal grid, grey
    specular walls and a larger channel; two runs at different ray offsets."""
    kd = inputs.make_kdist(0)
    spec = _uneven_snapshots(kd, [(7, 9, 5), (12, 16, 8), (16, 12, 10), (20, 24, 8)], 80,
                             stretched=(1,), reflect=(2,))
    assert _oracle_batch_check(spec, {}, 64, (0, 4096)) == 3


def test_single_launch_batch_multigrid_against_oracle():
    """The multigrid march (2 grids, 3 segments per grid) of a batch, including a
    stretched snapshot, against the oracle's multigrid march."""
    kd = inputs.make_kdist(0)
    spec = _uneven_snapshots(kd, [(12, 16, 8), (24, 24, 12), (16, 24, 16)], 90, stretched=(0,),
                             reflect=(1,))
    assert _oracle_batch_check(spec, dict(mg_levels=2, mg_steps=3), 48, (0, 777)) == 2


def test_single_launch_batch_cell_proposals_against_oracle():
    """Per-cell integer proposals (host counts of 2^32, hemisphere splits across
    (0, 1)) on every snapshot of a batch, against the oracle with the same counts."""
    kd = inputs.make_kdist(0)
    spec = _uneven_snapshots(kd, [(9, 10, 6), (12, 16, 8), (7, 9, 5)], 95, stretched=(1,))
    rng = np.random.default_rng(12)
    nb, ng = kd.n_bands, kd.n_g
    spec_c = []
    for grid, kd_, T, x, _ in spec:
        nc = grid.ncells
        def cum(rows, k):
            c = rng.integers(1, 2**26, size=(rows, k)).astype(np.int64)
            c[:, -1] += 2**32 - c.sum(axis=1)
            return np.cumsum(c, axis=1).astype(np.uint64)
        prop = (cum(nc, nb), cum(nc * nb, ng).reshape(nc, nb, ng),
                rng.integers(1, 2**23, size=nc).astype(np.uint32))
        spec_c.append((grid, kd_, T, x, prop))
    assert _oracle_batch_check(spec_c, dict(proposal=mcrt.MCRT_PROPOSAL_CELL), 40, (0, 123)) == 3


def test_mixed_kdist_graph_batch_against_oracle():
    """Snapshots with different k-distributions run as per-snapshot launches in
    concurrent graph branches; every snapshot against the oracle."""
    spec = []
    for k, (nx, ny, nz) in enumerate([(12, 16, 10), (7, 9, 5), (20, 24, 8)]):
        kd = inputs.make_kdist(k)
        grid = inputs.Grid(nx, ny, nz, 4.0, 2.0, 2.0, eps_wall=(0.8, 1.0), T_wall=(500.0, 1000.0))
        T, x = inputs.channel_fields(grid, 100 + k, x_mode="field")
        spec.append((grid, kd, T, x, None))
    assert _oracle_batch_check(spec, {}, 56, (0, 999), streams=2) >= 6
