"""The warp-parallel march of long rays against the FP64 oracle.

Rays of optically thin bands that graze the walls are handed from the FP32
trace kernel to a second kernel in which a warp marches consecutive pieces of a
flight at once and combines them with a product scan.  Forcing the hand-off
early (after 4 segments, whatever the flight ahead) sends most rays through it:
its windows, its segment-by-segment flights, y faces, wall events with both
reflection laws, the tol and max_steps stopping rules inside a window,
stretched grids, boxes and batches.  Every case matches the oracle draw for draw
within the FP32 tolerance 1e-4 S_i, with the same segment count to 1e-3.
"""
import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs, mcrt

pytestmark = pytest.mark.gpu

RTOL = 1e-4


def _pair(grid, kd, T, x, rays, seed, tol=1e-4, max_steps=1 << 20, box=None, long_steps=4,
          flight=-1):
    orc = oracle.solve(grid, kd, T, x, rays=rays, seed=seed, tol=tol, max_steps=max_steps, box=box)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    S.set_tuning(long_ray_steps=long_steps, long_ray_flight=flight)
    q, s, st = S.solve(box=box, with_steps=True, rays=rays, seed=seed, tol=tol,
                       max_steps=max_steps, precision=mcrt.MCRT_FP32)
    stats = S.stats()
    S.close()
    err = np.abs(q - orc["q"])
    bad = err > RTOL * orc["scale"] + 1e-300
    assert not bad.any(), (f"{bad.sum()} cells beyond {RTOL} S; worst "
                           f"{np.max(err / np.maximum(orc['scale'], 1e-300)):.3e}")
    assert abs(st.sum() / orc["steps"].sum() - 1.0) < 1e-3
    assert stats["steps"] == st.sum()
    assert stats["long_overflow"] == 0
    return orc, q, stats


def test_forced_hand_off_black_walls():
    grid, kd, T, x = inputs.nongrey_channel(24, 16, 20, seed=51, x_mode="field")
    _, _, stats = _pair(grid, kd, T, x, 64, seed=1)
    assert stats["long_rays"] > 0.05 * grid.ncells * 64


@pytest.mark.parametrize("reflect", [0, 1])
def test_forced_hand_off_grey_walls(reflect):
    grid, kd, T, x = inputs.nongrey_channel(20, 12, 16, seed=52, eps_wall=0.3, x_mode="field")
    grid.reflect = reflect
    T, x = inputs.channel_fields(grid, 52, x_mode="field")
    _, _, stats = _pair(grid, kd, T, x, 48, seed=2, box=(2, 18, 0, 12, 3, 13))
    assert stats["long_rays"] > 0 and stats["wall_hits"] > 0


def test_forced_hand_off_stretched_grid():
    grid, kd, T, x = inputs.nongrey_channel(16, 24, 12, seed=53, eps_wall=0.7, x_mode="field")
    grid.yf = inputs.channel_faces(24, grid.ly, 1.7)
    T, x = inputs.channel_fields(grid, 53, x_mode="field")
    _, _, stats = _pair(grid, kd, T, x, 48, seed=3)
    assert stats["long_rays"] > 0


@pytest.mark.parametrize("max_steps,tol", [(40, 1e-4), (1 << 20, 1e-7)])
def test_forced_hand_off_stopping_rules(max_steps, tol):
    """The step cap and a tight tol both stop rays inside the lanes' intervals."""
    grid, kd, T, x = inputs.nongrey_channel(16, 12, 16, seed=54, x_mode="field")
    orc, _, stats = _pair(grid, kd, T, x, 48, seed=4, tol=tol, max_steps=max_steps)
    assert stats["long_rays"] > 0
    if max_steps == 40:
        assert stats["capped"] == int(orc["capped"].sum()) and stats["capped"] > 0


def test_default_thresholds_on_a_channel_crop():
    """Default thresholds (1024 segments, then 32 crossings left in the flight)
    on a whole 48^3 channel: the grazing rays of thin bands are handed off, and
    the central crop matches the oracle (cells do not depend on the box)."""
    grid, kd, T, x = inputs.nongrey_channel(48, 48, 48, seed=55)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, _, st = S.solve(with_steps=True, rays=200, seed=5, precision=mcrt.MCRT_FP32)
    stats = S.stats()
    S.close()
    assert stats["long_rays"] > 0 and stats["long_overflow"] == 0
    box = (16, 32, 0, 48, 16, 32)
    orc = oracle.solve(grid, kd, T, x, rays=200, seed=5, box=box)
    qc = q[16:32, :, 16:32]
    err = np.abs(qc - orc["q"])
    assert not (err > RTOL * orc["scale"] + 1e-300).any()
    assert abs(st[16:32, :, 16:32].sum() / orc["steps"].sum() - 1.0) < 1e-3


def test_hand_off_results_independent_of_launch_shape():
    grid, kd, T, x = inputs.nongrey_channel(20, 16, 12, seed=56, eps_wall=0.8, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    S.set_tuning(long_ray_steps=4, long_ray_flight=-1)
    q0, s0, st0 = S.solve(rays=200, seed=3, with_steps=True)
    n0 = S.stats()["long_rays"]
    assert n0 > 0
    for mb, k, mib in ((1, 1, 0), (3, 2, 0), (2, 4, 1), (4, 1, 3)):
        S.set_tuning(mb, k, mib, long_ray_steps=4, long_ray_flight=-1)
        q, s, st = S.solve(rays=200, seed=3, with_steps=True)
        assert np.array_equal(q, q0) and np.array_equal(s, s0) and np.array_equal(st, st0)
        assert S.stats()["long_rays"] == n0
    # off: the same estimate summed in another order
    S.set_tuning(long_ray_steps=-1)
    assert S.tuning()["long_ray_steps"] == -1
    q1, _, st1 = S.solve(rays=200, seed=3, with_steps=True)
    assert S.stats()["long_rays"] == 0 and S.stats()["launches"] == 2
    assert np.allclose(q1, q0, rtol=1e-5, atol=1e-5 * np.abs(q0).max())
    assert abs(int(st1.sum()) - int(st0.sum())) <= 1e-4 * st0.sum()
    S.close()


def test_batch_with_forced_hand_off_matches_single_solves():
    import torch
    kd = inputs.make_kdist(0)
    solvers, outs, items = [], [], []
    for k, (nx, ny, nz) in enumerate([(16, 12, 12), (12, 16, 8), (20, 12, 16)]):
        grid = inputs.Grid(nx, ny, nz, 4.0, 2.0, 2.0, eps_wall=(0.6, 1.0), T_wall=(500.0, 1000.0),
                           reflect=k % 2)
        if k == 1:
            grid.yf = inputs.channel_faces(ny, 2.0, 1.5)
        T, x = inputs.channel_fields(grid, 80 + k, x_mode="field")
        S = mcrt.Solver(grid, kd)
        S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
        S.set_tuning(long_ray_steps=4, long_ray_flight=-1)
        q = torch.full(grid.shape, float("nan"), dtype=torch.float64, device="cuda")
        s = torch.full_like(q, float("nan"))
        solvers.append(S)
        outs.append((q, s))
        items.append((S.ctx, q.data_ptr(), s.data_ptr(), 30 + k))
    rays = 120
    params = mcrt.Solver.params(rays=rays, seed=11, precision=mcrt.MCRT_FP32)
    stream = torch.cuda.current_stream().cuda_stream
    b = mcrt.mcrt_batch_create(items, params)
    try:
        for offset in (0, 4000):
            mcrt.mcrt_batch_run(b, offset, stream)
            st = mcrt.mcrt_batch_get_stats(b)
            assert st["launches"] == 3 and st["long_rays"] > 0 and st["long_overflow"] == 0
            total = 0
            for k, (S, (q, s)) in enumerate(zip(solvers, outs)):
                qr, sr = S.solve(rays=rays, seed=11, snapshot=30 + k, ray_offset=offset,
                                 precision=mcrt.MCRT_FP32)
                total += S.stats()["long_rays"]
                assert np.array_equal(q.cpu().numpy(), qr), (offset, k)
                assert np.array_equal(s.cpu().numpy(), sr), (offset, k)
            assert st["long_rays"] == total
    finally:
        mcrt.mcrt_batch_destroy(b)
    for S in solvers:
        S.close()


def test_forced_hand_off_with_a_cell_proposal():
    """Per-cell (n, g) and hemisphere proposals: the ray weight is fixed at set-up,
    so the handed-off rays carry it; both reflection laws, against the oracle."""
    import torch
    grid, kd, T, x = inputs.nongrey_channel(12, 16, 10, seed=57, eps_wall=0.5, x_mode="field")
    K = kd.n_bands * kd.n_g
    g = torch.Generator(device="cpu").manual_seed(9)
    qp = torch.rand((grid.ncells, K + 2), generator=g) ** 4 + 1e-3
    qp[:, :K] /= qp[:, :K].sum(dim=1, keepdim=True)
    qp[:, K] = 0.15 + 0.7 * torch.rand(grid.ncells, generator=g)
    for reflect in (0, 1):
        grid.reflect = reflect
        S = mcrt.Solver(grid, kd)
        S.set_fields(T, x)
        S.set_cell_proposal_probs(qp.float().cuda())
        S.set_tuning(long_ray_steps=4, long_ray_flight=-1)
        cn, cg, hemi = S.cell_proposal()
        box = (0, 12, 0, 16, 2, 5)
        sel = [i + 12 * (j + 16 * k) for k in range(2, 5) for j in range(16) for i in range(12)]
        prop = (cn.reshape(grid.ncells, kd.n_bands)[sel], cg.reshape(grid.ncells, K)[sel], hemi[sel])
        o = oracle.solve(grid, kd, T, x, rays=64, seed=6, box=box, proposal=prop)
        q, _ = S.solve(box=box, rays=64, seed=6, precision=mcrt.MCRT_FP32,
                       proposal=mcrt.MCRT_PROPOSAL_CELL)
        st = S.stats()
        S.close()
        assert st["long_rays"] > 0 and st["long_overflow"] == 0
        assert np.all(np.abs(q - o["q"]) <= RTOL * o["scale"] + 1e-300), reflect


def test_hand_off_stays_off_where_it_does_not_apply():
    """Multigrid marches, closed boxes and the FP64 parity mode hand nothing off
    (and launch no long-ray kernel), whatever the thresholds."""
    grid, kd, T, x = inputs.nongrey_channel(24, 24, 12, seed=58, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    S.set_tuning(long_ray_steps=4, long_ray_flight=-1)
    S.solve(rays=32, seed=1, mg_levels=3, mg_steps=3)
    st = S.stats()
    assert st["long_rays"] == 0 and st["launches"] == 2
    S.solve(rays=16, seed=1, precision=mcrt.MCRT_FP64)
    st = S.stats()
    assert st["long_rays"] == 0 and st["launches"] == 1
    S.close()
    grid, kd, T, x = inputs.sin_cube(12, 0.5)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    S.set_tuning(long_ray_steps=4, long_ray_flight=-1)
    S.solve(rays=32, seed=1)
    st = S.stats()
    assert st["long_rays"] == 0 and st["launches"] == 2
    S.close()
