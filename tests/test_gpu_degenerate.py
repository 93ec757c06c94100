"""Degenerate cases of the estimator on the GPU, against the FP64 oracle draw for
draw (tolerances as in the parity tests: 1e-10 S_i in FP64, 1e-4 S_i in FP32).

- Grids of one cell, one row or one layer: a ray wraps onto its own cell in
  the periodic directions, or meets a wall at its first y crossing.
- An optically thick gas (kappa dx = 62.5): rays end inside the emitting cell,
  where exp(-kappa ds) underflows.
- A transmissivity cut-off close to 1 (Algorithm 1's tol): rays stop after one
  or two segments and dump the residual.
- A transparent gas: no band emits at T_max, so the plain pdf (Eq. 13) does not
  exist; the solve is refused with an argument error instead of dividing by 0.
"""
import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs, mcrt

pytestmark = pytest.mark.gpu

RTOL = {mcrt.MCRT_FP64: 1e-10, mcrt.MCRT_FP32: 1e-4}
PRECISIONS = [mcrt.MCRT_FP64, mcrt.MCRT_FP32]


def _fields(grid, seed):
    # uniform random fields: the spectral generator needs more than one cell per axis
    rng = np.random.default_rng(seed)
    T = 600.0 + 300.0 * rng.random(grid.shape)
    x = 0.05 + 0.1 * rng.random(grid.shape)
    return np.ascontiguousarray(T), np.ascontiguousarray(x)


def _check(grid, kd, T, x, precision, rays=96, seed=3, tol=1e-4, max_steps=1 << 20):
    orc = oracle.solve(grid, kd, T, x, rays=rays, seed=seed, tol=tol, max_steps=max_steps)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, s, st = S.solve(with_steps=True, rays=rays, seed=seed, tol=tol, max_steps=max_steps,
                       precision=precision)
    stats = S.stats()
    S.close()
    err = np.abs(q - orc["q"])
    assert np.all(err <= RTOL[precision] * orc["scale"] + 1e-300), np.max(err / orc["scale"])
    if precision == mcrt.MCRT_FP64:
        assert np.array_equal(st, orc["steps"])
    else:
        assert abs(st.sum() / orc["steps"].sum() - 1.0) < 1e-3
    return orc, q, stats


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 5, 1), (3, 1, 2), (2, 3, 1)])
def test_tiny_grids(shape, precision):
    nx, ny, nz = shape
    kd = inputs.make_kdist(0, n_bands=8, n_g=4)
    for reflect in (0, 1):
        grid = inputs.Grid(nx, ny, nz, 0.5 * nx, 0.5 * ny, 0.5 * nz, eps_wall=(0.6, 1.0),
                           T_wall=(500.0, 1000.0), reflect=reflect)
        T, x = _fields(grid, 11 + nx + 3 * ny + 7 * nz)
        _, _, stats = _check(grid, kd, T, x, precision)
        assert stats["wall_hits"] > 0


@pytest.mark.parametrize("precision", PRECISIONS)
def test_optically_thick_gas(precision):
    grid, kd, T, x = inputs.grey_slab_16x32x16(kappa=1000.0)
    orc, q, _ = _check(grid, kd, T, x, precision, rays=32)
    # the isothermal interior emits and absorbs in place (B_i - B_j = 0 on every
    # segment): only the rows next to the cold walls lose energy
    assert np.all(orc["q"][:, 2:-2, :] == 0.0) and np.all(q[:, 2:-2, :] == 0.0)
    # a ray reaches a cold wall only from within ln(1/tol) / kappa of it, and then it cools
    for row in (0, -1):
        assert np.all(q[:, row, :] >= 0.0) and q[:, row, :].sum() > 0.0
    # about 1.2 segments per ray: a second one only when the first is shorter than
    # ln(1/tol) / kappa
    assert orc["steps"].sum() <= 1.3 * grid.ncells * 32


@pytest.mark.parametrize("precision", PRECISIONS)
def test_cut_off_close_to_one(precision):
    grid = inputs.Grid(12, 10, 8, 2.0, 1.0, 1.0, eps_wall=(0.8, 0.8), T_wall=(500.0, 1000.0))
    kd = inputs.make_kdist(2, n_bands=10, n_g=4)
    T, x = _fields(grid, 5)
    orc, _, _ = _check(grid, kd, T, x, precision, tol=0.999)
    # almost every ray stops after its first segment
    assert orc["steps"].sum() <= 1.05 * grid.ncells * 96


def test_transparent_gas_is_an_argument_error():
    grid, _, T, x = inputs.grey_slab_16x32x16(kappa=1.0)
    S = mcrt.Solver(grid, inputs.make_grey_kdist(0.0))
    with pytest.raises(mcrt.McrtError) as e:
        S.set_fields(T, x)
        S.solve(rays=4)
    assert e.value.status == mcrt.MCRT_E_ARG
    S.close()
