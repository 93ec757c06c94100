"""GPU parity of the multigrid march (Section 4.3) with the FP64 oracle.

The oracle falls onto each coarser grid by restarting a face-distance march at
the ray's current point; the kernels keep the fine axis parameters and skip the
odd-numbered faces.  The two agree to rounding, draw for draw: rtol 1e-10 S in
FP64 mode and 1e-4 S in FP32 mode.  Multigrid results also keep the exact
path's properties: independence of the launch shape, bitwise shard unions,
batches equal to single solves, and the allocation-free solve.
"""
import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs, mcrt

pytestmark = pytest.mark.gpu

RTOL = {mcrt.MCRT_FP64: 1e-10, mcrt.MCRT_FP32: 1e-4}


def run_pair(grid, kd, T, x, rays, precision, levels, k, seed=0, tol=1e-4, box=None, origin=0):
    orc = oracle.solve(grid, kd, T, x, rays=rays, seed=seed, tol=tol, max_steps=1 << 20,
                       origin=origin, box=box, mg_levels=levels, mg_steps=k)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, s, st = S.solve(box=box, with_steps=True, rays=rays, seed=seed, tol=tol,
                       max_steps=1 << 20, origin=origin, precision=precision,
                       mg_levels=levels, mg_steps=k)
    S.close()
    return orc, q, s, st


def assert_parity(orc, q, st, precision):
    rtol = RTOL[precision]
    err = np.abs(q - orc["q"])
    bad = err > rtol * orc["scale"] + 1e-300
    assert not bad.any(), (f"{bad.sum()} cells beyond {rtol} S; worst "
                           f"{np.max(err / np.maximum(orc['scale'], 1e-300)):.3e}")
    if precision == mcrt.MCRT_FP64:
        assert np.array_equal(st, orc["steps"])
    else:
        assert abs(st.sum() / orc["steps"].sum() - 1.0) < 1e-3


@pytest.mark.parametrize("precision", [mcrt.MCRT_FP64, mcrt.MCRT_FP32])
@pytest.mark.parametrize("k", [1, 5])
def test_multigrid_channel_parity(precision, k):
    grid, kd, T, x = inputs.nongrey_channel(24, 24, 12, seed=31, x_mode="field")
    L = mcrt.mcrt_multigrid_levels(24, 24, 12)
    assert L == oracle.mg_max_levels(24, 24, 12) == 3
    orc, q, s, st = run_pair(grid, kd, T, x, 64, precision, L, k, seed=2)
    assert_parity(orc, q, st, precision)
    exact = oracle.solve(grid, kd, T, x, rays=64, seed=2, tol=1e-4, max_steps=1 << 20)
    assert orc["steps"].sum() < exact["steps"].sum()


@pytest.mark.parametrize("precision", [mcrt.MCRT_FP64, mcrt.MCRT_FP32])
@pytest.mark.parametrize("reflect", [0, 1])
def test_multigrid_grey_walls_parity(precision, reflect):
    """Reflections on coarse grids: fractions of the coarse cell, the axis
    parameters set up again on that grid."""
    grid, kd, T, x = inputs.nongrey_channel(16, 24, 12, seed=32, eps_wall=0.6, x_mode="field")
    grid.reflect = reflect
    orc, q, s, st = run_pair(grid, kd, T, x, 48, precision, 3, 2, seed=3, tol=1e-5,
                             box=(2, 14, 0, 24, 3, 9))
    assert_parity(orc, q, st, precision)


def test_multigrid_two_levels_ragged_center_origin():
    grid, kd, T, x = inputs.nongrey_channel(12, 10, 8, seed=33, eps_wall=0.8, x_mode="field")
    assert mcrt.mcrt_multigrid_levels(12, 10, 8) == 2
    for prec in (mcrt.MCRT_FP64, mcrt.MCRT_FP32):
        orc, q, s, st = run_pair(grid, kd, T, x, 37, prec, 2, 3, seed=4, origin=1,
                                 box=(1, 11, 0, 10, 2, 7))
        assert_parity(orc, q, st, prec)


def test_multigrid_isothermal_equals_exact_on_gpu():
    grid = inputs.Grid(24, 24, 12, 2.0, 1.0, 1.0, eps_wall=(0.7, 0.7), T_wall=(1500.0, 400.0))
    kd = inputs.make_kdist(3)
    T = np.full(grid.shape, 900.0)
    x = np.full(grid.shape, 0.12)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q0, _, st0 = S.solve(rays=128, seed=5, tol=1e-8, with_steps=True)
    q1, _, st1 = S.solve(rays=128, seed=5, tol=1e-8, with_steps=True, mg_levels=3, mg_steps=2)
    S.close()
    assert st1.sum() < 0.9 * st0.sum()
    np.testing.assert_allclose(q1, q0, rtol=2e-5, atol=2e-5 * np.abs(q0).max())


def test_multigrid_bitwise_properties():
    """Launch shape, shards, batches and the allocation-free solve change no bit
    of a multigrid solve."""
    import torch
    grid, kd, T, x = inputs.nongrey_channel(24, 24, 12, seed=34, eps_wall=0.8, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    kw = dict(rays=200, seed=6, mg_levels=3, mg_steps=4)
    q0, s0, st0 = S.solve(with_steps=True, **kw)
    for mb, kk in ((1, 1), (2, 4), (4, 2)):
        S.set_tuning(mb, kk, 0)
        q, s, st = S.solve(with_steps=True, **kw)
        assert np.array_equal(q, q0) and np.array_equal(s, s0) and np.array_equal(st, st0)
    S.set_tuning(0, 0, 0)
    parts = [S.solve(box=(0, 24, 0, 24, a, b), **kw) for a, b in ((0, 7), (7, 12))]
    assert np.array_equal(np.concatenate([p[0] for p in parts], axis=0), q0)
    # allocation-free entry point
    qd = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
    sd = torch.empty_like(qd)
    stream = torch.cuda.current_stream().cuda_stream
    mcrt.mcrt_solve_qrad_noalloc(S.ctx, S.params(**kw), qd.data_ptr(), sd.data_ptr(), stream)
    torch.cuda.synchronize()
    assert np.array_equal(qd.cpu().numpy(), q0) and np.array_equal(sd.cpu().numpy(), s0)
    # one graph launch over a batch of one
    qb = torch.empty_like(qd)
    sb = torch.empty_like(qd)
    b = mcrt.mcrt_batch_create([(S.ctx, qb.data_ptr(), sb.data_ptr(), 0)], S.params(**kw), streams=1)
    try:
        mcrt.mcrt_batch_run(b, 0, stream)
        mcrt.mcrt_batch_get_stats(b)
        assert np.array_equal(qb.cpu().numpy(), q0) and np.array_equal(sb.cpu().numpy(), s0)
    finally:
        mcrt.mcrt_batch_destroy(b)
    # argument checks
    for bad in (dict(mg_levels=4, mg_steps=5), dict(mg_levels=3, mg_steps=0), dict(mg_levels=-1)):
        with pytest.raises(mcrt.McrtError) as e:
            S.solve(rays=4, **bad)
        assert e.value.status == mcrt.MCRT_E_ARG
    S.close()


def test_multigrid_full_size_channel_sampled_cells():
    """The benchmark workload (64^3, 1000 rays, FP32) on 5 grids with the
    paper's 5 segments per grid, against the oracle on sampled cells."""
    grid, kd, T, x = inputs.nongrey_channel(64, 64, 64, seed=0)
    L = mcrt.mcrt_multigrid_levels(64, 64, 64)
    assert L == 5
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, s = S.solve(rays=1000, seed=0, tol=1e-4, max_steps=1 << 20, precision=mcrt.MCRT_FP32,
                   mg_levels=L, mg_steps=5)
    S.close()
    rng = np.random.default_rng(1)
    cells = [tuple(rng.integers(0, 64, 3)) for _ in range(10)] + [(0, 0, 0), (63, 63, 63), (5, 0, 9)]
    for (i, j, k) in cells:
        o = oracle.solve(grid, kd, T, x, rays=1000, seed=0, tol=1e-4, max_steps=1 << 20,
                         box=(i, i + 1, j, j + 1, k, k + 1), mg_levels=L, mg_steps=5)
        assert abs(q[k, j, i] - o["q"][0, 0, 0]) <= 1e-4 * o["scale"][0, 0, 0], (i, j, k)
