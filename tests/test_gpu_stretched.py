"""GPU parity on stretched wall-normal grids (the channel DNS grids of Section 5).

The kernels advance the y crossings incrementally (the next row's height over
|d_y|), the oracle from the face positions relative to the ray's start; both
agree to rounding, draw for draw: rtol 1e-10 S in FP64 mode, 1e-4 S in FP32.
Also: the E3 cell averages on the GPU, multigrid on stretched grids, the
features, the bitwise launch-shape and shard properties, and face checks.
"""
import numpy as np
import pytest
from scipy.special import expn

import oracle
from paper_1810_00188_gb300 import inputs, mcrt

pytestmark = pytest.mark.gpu

RTOL = {mcrt.MCRT_FP64: 1e-10, mcrt.MCRT_FP32: 1e-4}


def _pair(grid, kd, T, x, rays, precision, seed=0, tol=1e-4, box=None, levels=1, k=5):
    orc = oracle.solve(grid, kd, T, x, rays=rays, seed=seed, tol=tol, max_steps=1 << 20, box=box,
                       mg_levels=levels, mg_steps=k)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, s, st = S.solve(box=box, with_steps=True, rays=rays, seed=seed, tol=tol, max_steps=1 << 20,
                       precision=precision, mg_levels=levels, mg_steps=k)
    S.close()
    err = np.abs(q - orc["q"])
    bad = err > RTOL[precision] * orc["scale"] + 1e-300
    assert not bad.any(), (f"{bad.sum()} cells beyond {RTOL[precision]} S; worst "
                           f"{np.max(err / np.maximum(orc['scale'], 1e-300)):.3e}")
    if precision == mcrt.MCRT_FP64:
        assert np.array_equal(st, orc["steps"])
    else:
        assert abs(st.sum() / orc["steps"].sum() - 1.0) < 1e-3
    return orc, q


@pytest.mark.parametrize("precision", [mcrt.MCRT_FP64, mcrt.MCRT_FP32])
def test_stretched_channel_parity(precision):
    grid, kd, T, x = inputs.nongrey_channel(16, 24, 12, seed=41, x_mode="field")
    grid.yf = inputs.channel_faces(24, grid.ly, 1.7)
    T, x = inputs.channel_fields(grid, 41, x_mode="field")
    _pair(grid, kd, T, x, 64, precision, seed=2)


@pytest.mark.parametrize("precision", [mcrt.MCRT_FP64, mcrt.MCRT_FP32])
@pytest.mark.parametrize("reflect", [0, 1])
def test_stretched_grey_walls_parity(precision, reflect):
    grid, kd, T, x = inputs.nongrey_channel(12, 16, 10, seed=42, eps_wall=0.7, x_mode="field")
    grid.yf = inputs.channel_faces(16, grid.ly, 2.0)
    grid.reflect = reflect
    T, x = inputs.channel_fields(grid, 42, x_mode="field")
    _pair(grid, kd, T, x, 48, precision, seed=3, tol=1e-5, box=(1, 11, 0, 16, 2, 8))


@pytest.mark.parametrize("precision", [mcrt.MCRT_FP64, mcrt.MCRT_FP32])
@pytest.mark.parametrize("k", [2, 5])
def test_stretched_multigrid_parity(precision, k):
    grid, kd, T, x = inputs.nongrey_channel(24, 24, 12, seed=43, eps_wall=0.8, x_mode="field")
    grid.yf = inputs.channel_faces(24, grid.ly, 1.6)
    T, x = inputs.channel_fields(grid, 43, x_mode="field")
    _pair(grid, kd, T, x, 48, precision, seed=4, levels=3, k=k, box=(0, 24, 0, 24, 3, 8))


def test_stretched_fp32_matches_E3_closed_form():
    grid, kd, T, x = inputs.grey_slab_16x32x16(1.0)
    grid.yf = inputs.channel_faces(32, grid.ly, 1.8)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, s = S.solve(rays=128, seed=0, tol=1e-6, precision=mcrt.MCRT_FP32)
    S.close()
    yf, L = grid.y_faces(), 2.0
    y0, y1 = yf[:-1], yf[1:]
    ref = 2 * inputs.SIGMA_SB * 1e12 / (y1 - y0) * (expn(3, y0) - expn(3, y1) + expn(3, L - y1)
                                                     - expn(3, L - y0))
    row = q.mean(axis=(0, 2))
    se = np.sqrt((s**2).sum(axis=(0, 2))) / 256
    z = (row - ref) / se
    assert np.max(np.abs(z)) < 4 and np.sqrt(np.mean(z**2)) < 1.6


def test_stretched_features_match_oracle():
    import torch
    grid, kd, T, x = inputs.nongrey_channel(10, 14, 8, seed=44, x_mode="field")
    grid.yf = inputs.channel_faces(14, grid.ly, 1.9)
    T, x = inputs.channel_fields(grid, 44, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    f = S.features().cpu().numpy()
    S.close()
    ref = oracle.features(grid, kd, T, x)
    np.testing.assert_allclose(f, ref, rtol=2e-5, atol=2e-6)


def test_stretched_bitwise_properties_and_face_checks():
    grid, kd, T, x = inputs.nongrey_channel(24, 24, 12, seed=45, eps_wall=0.8, x_mode="field")
    grid.yf = inputs.channel_faces(24, grid.ly, 1.5)
    T, x = inputs.channel_fields(grid, 45, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    kw = dict(rays=160, seed=6, mg_levels=3, mg_steps=3)
    q0, s0, st0 = S.solve(with_steps=True, **kw)
    for mb, kk in ((2, 2), (4, 1)):
        S.set_tuning(mb, kk, 0)
        q, s, st = S.solve(with_steps=True, **kw)
        assert np.array_equal(q, q0) and np.array_equal(s, s0) and np.array_equal(st, st0)
    S.set_tuning(0, 0, 0)
    parts = [S.solve(box=(0, 24, 0, 24, a, b), **kw) for a, b in ((0, 5), (5, 12))]
    assert np.array_equal(np.concatenate([p[0] for p in parts], axis=0), q0)
    S.close()
    for bad in (np.linspace(0.0, 2.0, 25)[::-1], np.linspace(0.1, 2.0, 25),
                np.concatenate([[0.0, 0.5, 0.5], np.linspace(0.6, 2.0, 22)])):
        g2 = inputs.Grid(24, 24, 12, grid.lx, grid.ly, grid.lz, yf=bad)
        with pytest.raises(mcrt.McrtError) as e:
            mcrt.Solver(g2, kd)
        assert e.value.status == mcrt.MCRT_E_ARG
