"""Oracle pins of the multigrid march (Section 4.3 of the paper).

The paper overlays grids coarsened by 2, down to a smallest 3^3 mesh; a ray
marches a fixed number of segments on each grid, falls onto the next coarser
grid at its current point, and runs to depletion on the coarsest one.  The
coarse temperatures come from the fine solution.

* Grid counts: Section 5 lists 3 grids for 16^3, 4 for 32^3, 5 for 48^3 and
  64^3, 6 for 96^3, 128^3 and 160^3; Section 4.3 uses 7 for 192^3.
* An independent path integral (numpy): on each grid every face crossing of the
  straight ray is listed, the first k segments after the current point are taken
  with each segment's cell from its midpoint, and the fields are the 2x2x2 means
  of the finer grid.  The oracle's per-ray sum must agree to rounding.
* In an isothermal medium every grid holds the same T and x, so coarsening
  only merges segments: the per-cell estimate equals the single-grid one to
  rounding, also with grey, diffusely reflecting walls.
* One grid, or more segments per grid than any ray takes, is the exact march.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs


def test_grid_counts_follow_the_paper():
    for n, L in ((16, 3), (32, 4), (48, 5), (64, 5), (96, 6), (128, 6), (160, 6), (192, 7)):
        assert oracle.mg_max_levels(n, n, n) == L, n
    assert oracle.mg_max_levels(256, 192, 128) == 6
    assert oracle.mg_max_levels(12, 10, 8) == 2
    assert oracle.mg_max_levels(5, 8, 8) == 1


def _coarse(a, levels):
    """Level fields: 2x2x2 means, [nz, ny, nx] layout."""
    out = [np.asarray(a, dtype=np.float64)]
    for _ in range(1, levels):
        f = out[-1]
        nz, ny, nx = f.shape
        out.append(f.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(1, 3, 5)))
    return out


def mg_segment_list_X(grid, kd, T, x, n, g, cell, frac, d, tol, levels, k):
    """Independent multigrid path integral of one ray between black walls."""
    delta0 = np.array([grid.lx / grid.nx, grid.ly / grid.ny, grid.lz / grid.nz])
    N0 = np.array([grid.nx, grid.ny, grid.nz])
    p0 = (np.asarray(cell) + np.asarray(frac)) * delta0
    d = np.asarray(d, dtype=np.float64)
    t_wall = ((grid.ly - p0[1]) / d[1]) if d[1] > 0 else (-p0[1] / d[1])
    Ts, xs = _coarse(T, levels), _coarse(x, levels)
    nodes = kd.T_nodes()
    Tf0, xf0 = T.reshape(-1), x.reshape(-1)
    c0 = cell[0] + N0[0] * (cell[1] + N0[1] * cell[2])
    kap_i = np.interp(Tf0[c0], nodes, kd.kappa[n, g]) * xf0[c0] / kd.x_ref
    B_i = np.interp(Tf0[c0], nodes, kd.B[n])
    X, tau, t_cur, steps, B_last = 0.0, 1.0, 0.0, 0, B_i
    for lev in range(levels):
        delta = delta0 * 2.0**lev
        N = N0 // 2**lev
        times = [np.array([t_wall])]
        for a in range(3):
            if d[a] == 0:
                continue
            lo, hi = sorted([p0[a], p0[a] + t_wall * d[a]])
            planes = np.arange(math.floor(lo / delta[a]), math.ceil(hi / delta[a]) + 1) * delta[a]
            t = (planes - p0[a]) / d[a]
            times.append(t[(t > t_cur * (1 + 1e-12) + 1e-15) & (t < t_wall)])
        t = np.concatenate([[t_cur], np.unique(np.concatenate(times))])
        if lev + 1 < levels:
            t = t[:k + 1]
        mid = 0.5 * (t[:-1] + t[1:])
        ds = np.diff(t)
        pos = p0[None, :] + mid[:, None] * d[None, :]
        idx = np.floor(pos / delta[None, :]).astype(np.int64)
        idx[:, 0] %= N[0]
        idx[:, 2] %= N[2]
        assert np.all((idx[:, 1] >= 0) & (idx[:, 1] < N[1]))
        Tf, xf = Ts[lev].reshape(-1), xs[lev].reshape(-1)
        lin = idx[:, 0] + N[0] * (idx[:, 1] + N[1] * idx[:, 2])
        kap = np.interp(Tf[lin], nodes, kd.kappa[n, g]) * xf[lin] / kd.x_ref
        B = np.interp(Tf[lin], nodes, kd.B[n])
        for s in range(ds.size):
            a = -math.expm1(-kap[s] * ds[s])
            X += kap_i * (B_i - B[s]) * tau * a
            tau *= math.exp(-kap[s] * ds[s])
            steps += 1
            B_last = B[s]
            if tau <= tol:
                return X + kap_i * (B_i - B_last) * tau, steps
        t_cur = t[-1]
        if t_cur >= t_wall * (1 - 1e-12):
            break
    w = 0 if d[1] < 0 else 1
    Bw = np.interp(grid.T_wall[w], nodes, kd.B[n])
    return X + kap_i * (B_i - Bw) * tau, steps


@pytest.mark.parametrize("k", [1, 2, 5])
def test_multigrid_march_matches_independent_segment_list(k):
    grid = inputs.Grid(24, 24, 12, 4.0, 2.0, 3.0, T_wall=(500.0, 1000.0))
    levels = oracle.mg_max_levels(grid.nx, grid.ny, grid.nz)
    assert levels == 3
    kd = inputs.make_kdist(1)
    T, x = inputs.channel_fields(grid, 21, fluct=0.15, x_mode="field")
    rng = np.random.default_rng(22 + k)
    nodes = kd.T_nodes()
    kmin = np.array([[np.interp(T.min(), nodes, kd.kappa[n, g]) for g in range(kd.n_g)]
                     for n in range(kd.n_bands)]) * 0.05 / kd.x_ref
    kmax = np.array([[np.interp(T.max(), nodes, kd.kappa[n, g]) for g in range(kd.n_g)]
                     for n in range(kd.n_bands)]) * 0.2 / kd.x_ref
    ok = np.argwhere((kmin > 0.01) & (kmax < 3.0))
    checked = switched = 0
    for _ in range(80):
        n, g = ok[rng.integers(len(ok))]
        cell = (rng.integers(grid.nx), rng.integers(grid.ny), rng.integers(grid.nz))
        frac = rng.uniform(0.0, 1.0, 3)
        mu = rng.uniform(-1, 1)
        if abs(mu) < 0.05:
            continue
        phi = rng.uniform(0, 2 * math.pi)
        s = math.sqrt(1 - mu * mu)
        d = (s * math.cos(phi), mu, s * math.sin(phi))
        ref, nseg = mg_segment_list_X(grid, kd, T, x, int(n), int(g), cell, frac, d, 1e-6, levels, k)
        got = oracle.trace_ray(grid, kd, T, x, int(n), int(g), cell, frac, d, tol=1e-6,
                               mg_levels=levels, mg_steps=k)
        exact = oracle.trace_ray(grid, kd, T, x, int(n), int(g), cell, frac, d, tol=1e-6)
        assert got["X"] == pytest.approx(ref, rel=1e-9, abs=1e-12 * abs(got["abs_terms"]))
        assert got["steps"] == nseg
        assert got["steps"] <= exact["steps"]
        if got["steps"] > k:
            switched += 1
            # the coarse grids only merge segments: same geometric path to the wall
            if got["walls"] > 0 and exact["walls"] > 0:
                assert got["path"] == pytest.approx(exact["path"], rel=1e-12)
        checked += 1
    assert checked > 60 and switched > 20


@pytest.mark.parametrize("eps,reflect", [(1.0, 0), (0.6, 0), (0.6, 1)])
def test_isothermal_multigrid_equals_single_grid(eps, reflect):
    grid = inputs.Grid(24, 24, 12, 2.0, 1.0, 1.0, eps_wall=(eps, eps), T_wall=(1500.0, 400.0),
                       reflect=reflect)
    kd = inputs.make_kdist(3)
    T = np.full(grid.shape, 900.0)
    x = np.full(grid.shape, 0.12)
    kw = dict(rays=96, seed=4, tol=1e-8, box=(0, 24, 0, 24, 2, 4))
    ex = oracle.solve(grid, kd, T, x, **kw)
    L = oracle.mg_max_levels(grid.nx, grid.ny, grid.nz)
    assert L == 3
    mg = oracle.solve(grid, kd, T, x, mg_levels=L, mg_steps=2, **kw)
    assert np.all(mg["steps"] <= ex["steps"])
    assert mg["steps"].sum() < 0.9 * ex["steps"].sum()
    np.testing.assert_allclose(mg["q"], ex["q"], rtol=1e-9, atol=1e-12 * np.abs(ex["scale"]).max())


def test_one_grid_or_unreachable_switch_is_the_exact_march():
    grid, kd, T, x = inputs.nongrey_channel(16, 16, 16, seed=5, eps_wall=0.8, x_mode="field")
    kw = dict(rays=64, seed=2, box=(0, 16, 0, 16, 3, 5))
    ex = oracle.solve(grid, kd, T, x, **kw)
    one = oracle.solve(grid, kd, T, x, mg_levels=1, mg_steps=1, **kw)
    far = oracle.solve(grid, kd, T, x, mg_levels=3, mg_steps=1 << 30, **kw)
    for r in (one, far):
        assert np.array_equal(r["sum_y"], ex["sum_y"])
        assert np.array_equal(r["steps"], ex["steps"])
    with pytest.raises(ValueError):
        oracle.solve(grid, kd, T, x, mg_levels=4, mg_steps=5, **kw)
