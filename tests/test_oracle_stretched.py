"""Oracle pins on stretched wall-normal grids (the channel DNS grids of Section 5).

* The E3 cell averages of the isothermal grey slab hold for any face positions:
  Q_j = (2 sigma T^4 / dy_j) [E3(k y_j) - E3(k y_j+1) + E3(k (L - y_j+1)) - E3(k (L - y_j))].
* An independent path integral with the y planes taken from the face list agrees
  with the oracle's march to rounding, on the single grid and on multigrid grids
  (coarse faces every other face, coarse fields volume-weighted means).
* Faces that happen to be uniform reproduce the uniform march to rounding.
* Isothermal media: multigrid equals the single grid to rounding.
* Features: y_c is the midpoint of the faces and dT/dy of a profile linear in
  y is exact on any spacing.
"""
import math

import numpy as np
import pytest
from scipy.special import expn

import oracle
from paper_1810_00188_gb300 import inputs

SIG = inputs.SIGMA_SB


def stretched_slab(kap, gamma=1.8, ny=32):
    grid, kd, T, x = inputs.grey_slab_16x32x16(kap)
    grid.yf = inputs.channel_faces(ny, grid.ly, gamma)
    return grid, kd, T, x


def E3_cell_average(kap, yf, L, coef):
    y0, y1 = yf[:-1], yf[1:]
    e = lambda v: expn(3, v)  # noqa: E731
    return coef / (y1 - y0) * (e(kap * y0) - e(kap * y1) + e(kap * (L - y1)) - e(kap * (L - y0)))


@pytest.mark.parametrize("kap", [1.0, 10.0])
def test_stretched_isothermal_black_cell_average_E3(kap):
    grid, kd, T, x = stretched_slab(kap)
    yf = grid.y_faces()
    assert (yf[1] - yf[0]) < 0.3 * (2.0 / 32)  # strongly refined at the walls
    res = oracle.solve(grid, kd, T, x, rays=128, seed=0, tol=1e-12)
    ref = E3_cell_average(kap, yf, 2.0, 2.0 * SIG * 1000.0**4)
    q = res["q"].mean(axis=(0, 2))
    se = np.sqrt((res["sigma"] ** 2).sum(axis=(0, 2))) / (res["q"].shape[0] * res["q"].shape[2])
    z = (q - ref) / se
    assert np.max(np.abs(z)) < 4.0 and np.sqrt(np.mean(z**2)) < 1.6, np.round(z, 2)


def _coarse(a, levels, yf):
    """Level fields of a stretched grid: 2x2x2 means weighted by the children's heights."""
    out, faces = [np.asarray(a, dtype=np.float64)], [np.asarray(yf, dtype=np.float64)]
    for _ in range(1, levels):
        f, y = out[-1], faces[-1]
        nz, ny, nx = f.shape
        w = np.diff(y).reshape(ny // 2, 2)
        blocks = f.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2)
        num = (blocks * w[None, None, :, :, None, None]).sum(axis=(1, 3, 5))
        den = 4.0 * w.sum(axis=1)[None, :, None]
        out.append(num / den)
        faces.append(y[::2])
    return out, faces


def segment_list_X(grid, kd, T, x, n, g, cell, frac, d, tol, levels=1, k=1 << 30):
    """Independent path integral between black walls on y faces from a list;
    with levels > 1 the first k segments of each grid, then the next grid."""
    yf0 = grid.y_faces()
    dx, dz = grid.lx / grid.nx, grid.lz / grid.nz
    N0 = np.array([grid.nx, grid.ny, grid.nz])
    p0 = np.array([(cell[0] + frac[0]) * dx,
                   yf0[cell[1]] + frac[1] * (yf0[cell[1] + 1] - yf0[cell[1]]),
                   (cell[2] + frac[2]) * dz])
    d = np.asarray(d, dtype=np.float64)
    t_wall = ((grid.ly - p0[1]) / d[1]) if d[1] > 0 else (-p0[1] / d[1])
    Ts, faces = _coarse(T, levels, yf0)
    xs, _ = _coarse(x, levels, yf0)
    nodes = kd.T_nodes()
    c0 = cell[0] + N0[0] * (cell[1] + N0[1] * cell[2])
    kap_i = np.interp(T.reshape(-1)[c0], nodes, kd.kappa[n, g]) * x.reshape(-1)[c0] / kd.x_ref
    B_i = np.interp(T.reshape(-1)[c0], nodes, kd.B[n])
    X, tau, t_cur, steps = 0.0, 1.0, 0.0, 0
    for lev in range(levels):
        N = N0 // 2**lev
        dl = np.array([dx * 2**lev, 0.0, dz * 2**lev])
        times = [np.array([t_wall])]
        for a in (0, 2):
            if d[a] == 0:
                continue
            lo, hi = sorted([p0[a], p0[a] + t_wall * d[a]])
            planes = np.arange(math.floor(lo / dl[a]), math.ceil(hi / dl[a]) + 1) * dl[a]
            times.append((planes - p0[a]) / d[a])
        times.append((faces[lev] - p0[1]) / d[1])
        t = np.concatenate(times)
        t = t[(t > t_cur * (1 + 1e-12) + 1e-15) & (t <= t_wall)]
        t = np.concatenate([[t_cur], np.unique(t)])
        if lev + 1 < levels:
            t = t[:k + 1]
        mid = 0.5 * (t[:-1] + t[1:])
        ds = np.diff(t)
        pos = p0[None, :] + mid[:, None] * d[None, :]
        ix = np.floor(pos[:, 0] / dl[0]).astype(np.int64) % N[0]
        iz = np.floor(pos[:, 2] / dl[2]).astype(np.int64) % N[2]
        iy = np.searchsorted(faces[lev], pos[:, 1], side="right") - 1
        assert np.all((iy >= 0) & (iy < N[1]))
        lin = ix + N[0] * (iy + N[1] * iz)
        Tf, xf = Ts[lev].reshape(-1), xs[lev].reshape(-1)
        kap = np.interp(Tf[lin], nodes, kd.kappa[n, g]) * xf[lin] / kd.x_ref
        B = np.interp(Tf[lin], nodes, kd.B[n])
        for s in range(ds.size):
            a = -math.expm1(-kap[s] * ds[s])
            X += kap_i * (B_i - B[s]) * tau * a
            tau *= math.exp(-kap[s] * ds[s])
            steps += 1
            if tau <= tol:
                return X + kap_i * (B_i - B[s]) * tau, steps
        t_cur = t[-1]
        if t_cur >= t_wall * (1 - 1e-12):
            break
    w = 0 if d[1] < 0 else 1
    Bw = np.interp(grid.T_wall[w], nodes, kd.B[n])
    return X + kap_i * (B_i - Bw) * tau, steps


@pytest.mark.parametrize("levels,k", [(1, 1 << 30), (3, 2), (3, 5)])
def test_stretched_march_matches_independent_segment_list(levels, k):
    grid = inputs.Grid(24, 24, 12, 4.0, 2.0, 3.0, T_wall=(500.0, 1000.0))
    grid.yf = inputs.channel_faces(24, 2.0, 1.6)
    kd = inputs.make_kdist(1)
    T, x = inputs.channel_fields(grid, 23, fluct=0.15, x_mode="field")
    rng = np.random.default_rng(24 + levels + k)
    nodes = kd.T_nodes()
    kmin = np.array([[np.interp(T.min(), nodes, kd.kappa[n, g]) for g in range(kd.n_g)]
                     for n in range(kd.n_bands)]) * 0.05 / kd.x_ref
    kmax = np.array([[np.interp(T.max(), nodes, kd.kappa[n, g]) for g in range(kd.n_g)]
                     for n in range(kd.n_bands)]) * 0.2 / kd.x_ref
    ok = np.argwhere((kmin > 0.01) & (kmax < 3.0))
    checked = 0
    for _ in range(70):
        n, g = ok[rng.integers(len(ok))]
        cell = (rng.integers(grid.nx), rng.integers(grid.ny), rng.integers(grid.nz))
        frac = rng.uniform(0.0, 1.0, 3)
        mu = rng.uniform(-1, 1)
        if abs(mu) < 0.05:
            continue
        phi = rng.uniform(0, 2 * math.pi)
        s = math.sqrt(1 - mu * mu)
        d = (s * math.cos(phi), mu, s * math.sin(phi))
        ref, nseg = segment_list_X(grid, kd, T, x, int(n), int(g), cell, frac, d, 1e-6, levels, k)
        got = oracle.trace_ray(grid, kd, T, x, int(n), int(g), cell, frac, d, tol=1e-6,
                               mg_levels=levels, mg_steps=k)
        assert got["X"] == pytest.approx(ref, rel=1e-9, abs=1e-12 * abs(got["abs_terms"]))
        assert got["steps"] == nseg
        checked += 1
    assert checked > 50


def test_uniform_faces_reproduce_the_uniform_march():
    grid, kd, T, x = inputs.nongrey_channel(12, 16, 10, seed=25, eps_wall=0.7, x_mode="field")
    kw = dict(rays=48, seed=3, box=(0, 12, 0, 16, 2, 4))
    ref = oracle.solve(grid, kd, T, x, **kw)
    grid.yf = np.linspace(0.0, grid.ly, grid.ny + 1)
    got = oracle.solve(grid, kd, T, x, **kw)
    np.testing.assert_allclose(got["q"], ref["q"], rtol=1e-9, atol=1e-11 * np.abs(ref["scale"]).max())
    assert np.array_equal(got["steps"], ref["steps"])


@pytest.mark.parametrize("reflect", [0, 1])
def test_stretched_isothermal_multigrid_equals_single_grid(reflect):
    grid = inputs.Grid(24, 24, 12, 2.0, 1.0, 1.0, eps_wall=(0.6, 0.6), T_wall=(1500.0, 400.0),
                       reflect=reflect)
    grid.yf = inputs.channel_faces(24, 1.0, 1.7)
    kd = inputs.make_kdist(3)
    T = np.full(grid.shape, 900.0)
    x = np.full(grid.shape, 0.12)
    kw = dict(rays=96, seed=4, tol=1e-8, box=(0, 24, 0, 24, 2, 4))
    ex = oracle.solve(grid, kd, T, x, **kw)
    mg = oracle.solve(grid, kd, T, x, mg_levels=3, mg_steps=2, **kw)
    assert mg["steps"].sum() < 0.9 * ex["steps"].sum()
    np.testing.assert_allclose(mg["q"], ex["q"], rtol=1e-9, atol=1e-12 * np.abs(ex["scale"]).max())


def test_stretched_features_linear_profile():
    grid = inputs.Grid(6, 10, 4, 3.0, 2.0, 2.0, T_wall=(500.0, 900.0))
    grid.yf = inputs.channel_faces(10, 2.0, 1.5)
    kd = inputs.make_kdist(0)
    yc = grid.cell_centers_y()
    T = np.broadcast_to((600.0 + 150.0 * yc)[None, :, None], grid.shape).copy()
    f = oracle.features(grid, kd, T, None)
    f = f.reshape(grid.nz, grid.ny, grid.nx, -1)
    np.testing.assert_allclose(f[0, :, 0, 2], yc / 1.0 - 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(f[..., 6], 1.0 * 150.0 / 1000.0, rtol=1e-12)
