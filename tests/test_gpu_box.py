"""GPU parity in closed boxes (black walls on all six faces): the paper's 3D
verification cases 3 and 4 (Table 1: 1 m cube, kappa = 0.5 and 5 1/m, sin
temperature profile, 32^3 cells, 2000 rays per cell), FP64 (1e-10 S) and FP32
(1e-4 S) against the oracle on the same draws, also on multigrid grids and
through the allocation-free entry point."""
import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs, mcrt

pytestmark = pytest.mark.gpu

RTOL = {mcrt.MCRT_FP64: 1e-10, mcrt.MCRT_FP32: 1e-4}


def _check(grid, kd, T, x, rays, precision, box=None, levels=1, k=5, origin=0, seed=0):
    o = oracle.solve(grid, kd, T, x, rays=rays, seed=seed, tol=1e-8, box=box, origin=origin,
                     mg_levels=levels, mg_steps=k)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, s, st = S.solve(box=box, with_steps=True, rays=rays, seed=seed, tol=1e-8, origin=origin,
                       precision=precision, mg_levels=levels, mg_steps=k)
    stats = S.stats()
    S.close()
    err = np.abs(q - o["q"])
    assert np.all(err <= RTOL[precision] * o["scale"] + 1e-300), np.max(err / o["scale"])
    if precision == mcrt.MCRT_FP64:
        assert np.array_equal(st, o["steps"])
    return q, s, stats


@pytest.mark.parametrize("precision", [mcrt.MCRT_FP64, mcrt.MCRT_FP32])
@pytest.mark.parametrize("kap", [0.5, 5.0])
def test_sin_cube_parity(precision, kap):
    grid, kd, T, x = inputs.sin_cube(16, kap)
    q, s, st = _check(grid, kd, T, x, 200, precision, seed=1)
    assert st["wall_hits"] > 0


@pytest.mark.parametrize("precision", [mcrt.MCRT_FP64, mcrt.MCRT_FP32])
def test_box_multigrid_parity(precision):
    grid, kd, T, x = inputs.sin_cube(24, 0.5)
    assert mcrt.mcrt_multigrid_levels(24, 24, 24) == 4  # 24^3, 12^3, 6^3, 3^3
    _check(grid, kd, T, x, 64, precision, levels=4, k=2, box=(0, 24, 10, 14, 8, 16), seed=2)


def test_sin_cube_case_3_32cubed_2000_rays_fp32():
    """The paper's own setting of case 3: 32^3 cells, 2000 rays per cell, the
    centre line y = z = 0.5 against the oracle cell by cell, and the line's
    symmetry about x = 0.5 within the sampled error."""
    grid, kd, T, x = inputs.sin_cube(32, 0.5)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, s = S.solve(rays=2000, seed=0, tol=1e-8, precision=mcrt.MCRT_FP32)
    S.close()
    o = oracle.solve(grid, kd, T, x, rays=2000, seed=0, tol=1e-8, box=(0, 32, 15, 17, 15, 17))
    line = q[15:17, 15:17, :]
    assert np.all(np.abs(line - o["q"]) <= 1e-4 * o["scale"])
    prof = q[15:17, 15:17, :].mean(axis=(0, 1))
    se = np.sqrt((s[15:17, 15:17, :] ** 2).sum(axis=(0, 1))) / 4
    z = (prof - prof[::-1]) / np.sqrt(se**2 + se[::-1] ** 2)
    assert np.max(np.abs(z)) < 4.0


def test_box_noalloc_and_rejections():
    import torch
    grid, kd, T, x = inputs.sin_cube(16, 5.0)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q0, s0 = S.solve(rays=128, seed=4, tol=1e-8)
    qd = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
    sd = torch.empty_like(qd)
    stream = torch.cuda.current_stream().cuda_stream
    mcrt.mcrt_solve_qrad_noalloc(S.ctx, S.params(rays=128, seed=4, tol=1e-8), qd.data_ptr(),
                                 sd.data_ptr(), stream)
    torch.cuda.synchronize()
    assert np.array_equal(qd.cpu().numpy(), q0) and np.array_equal(sd.cpu().numpy(), s0)
    with pytest.raises(mcrt.McrtError) as e:  # the features assume a channel
        S.features()
    assert e.value.status == mcrt.MCRT_E_UNSUPPORTED
    S.close()
