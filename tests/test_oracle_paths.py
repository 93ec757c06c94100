"""Oracle pins in 3D: path integrals, conservation, reciprocity, quadrature.

* The oracle marches a ray cell by cell with face distances (Algorithm 1
  "March").  An independent algorithm here lists every face crossing of the
  straight ray, sorts them, and finds each segment's cell from its midpoint; the
  per-ray sum of Eq. 14 terms must agree to rounding.
* Energy conservation: summed over all cells, the medium-medium part of the
  reciprocal estimate vanishes in expectation (the reciprocity principle, Eq. 11),
  so sum_i V_i Q_i equals the net wall exchange.
* Reciprocity (Eq. 11): the exchange factors G_ij = E[w kappa_i tau alpha_j] of
  equal cells satisfy G_ij = G_ji.
* Unbiasedness of the sampling (Eqs. 4, 9, 16, 17): the Monte Carlo mean agrees
  with a deterministic quadrature of the same estimand within 3 sigma, and its
  error shrinks like 1/sqrt(N).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs


def _field(grid, seed):
    T, x = inputs.channel_fields(grid, seed, fluct=0.15, x_mode="field")
    return T, x


def segment_list_X(grid, kd, T, x, n, g, cell, frac, d, tol):
    """Independent path integral of one ray between black walls."""
    delta = np.array([grid.lx / grid.nx, grid.ly / grid.ny, grid.lz / grid.nz])
    N = np.array([grid.nx, grid.ny, grid.nz])
    p0 = (np.asarray(cell) + np.asarray(frac)) * delta
    d = np.asarray(d, dtype=np.float64)
    t_wall = ((grid.ly - p0[1]) / d[1]) if d[1] > 0 else (-p0[1] / d[1])
    times = [np.array([0.0, t_wall])]
    for a in range(3):
        if d[a] == 0:
            continue
        lo, hi = sorted([p0[a], p0[a] + t_wall * d[a]])
        planes = np.arange(math.floor(lo / delta[a]), math.ceil(hi / delta[a]) + 1) * delta[a]
        t = (planes - p0[a]) / d[a]
        times.append(t[(t > 0) & (t < t_wall)])
    t = np.unique(np.concatenate(times))
    mid = 0.5 * (t[:-1] + t[1:])
    ds = np.diff(t)
    pos = p0[None, :] + mid[:, None] * d[None, :]
    idx = np.floor(pos / delta[None, :]).astype(np.int64)
    idx[:, 0] %= N[0]
    idx[:, 2] %= N[2]
    assert np.all((idx[:, 1] >= 0) & (idx[:, 1] < N[1]))
    Tf, xf = T.reshape(-1), x.reshape(-1)
    lin = idx[:, 0] + N[0] * (idx[:, 1] + N[1] * idx[:, 2])
    nodes = kd.T_nodes()
    kap = np.interp(Tf[lin], nodes, kd.kappa[n, g]) * xf[lin] / kd.x_ref
    B = np.interp(Tf[lin], nodes, kd.B[n])
    c0 = cell[0] + N[0] * (cell[1] + N[1] * cell[2])
    kap_i = np.interp(Tf[c0], nodes, kd.kappa[n, g]) * xf[c0] / kd.x_ref
    B_i = np.interp(Tf[c0], nodes, kd.B[n])
    X, tau = 0.0, 1.0
    for s in range(ds.size):
        a = -math.expm1(-kap[s] * ds[s])
        X += kap_i * (B_i - B[s]) * tau * a
        tau *= math.exp(-kap[s] * ds[s])
        if tau <= tol:
            return X + kap_i * (B_i - B[s]) * tau, s + 1, tau
    w = 0 if d[1] < 0 else 1
    Bw = np.interp(grid.T_wall[w], nodes, kd.B[n])
    return X + kap_i * (B_i - Bw) * tau, ds.size, 0.0


def test_march_matches_independent_segment_list():
    grid = inputs.Grid(6, 8, 5, 4.0 * math.pi, 2.0, 2.0 * math.pi, T_wall=(500.0, 1000.0))
    kd = inputs.make_kdist(1)
    T, x = _field(grid, 11)
    rng = np.random.default_rng(12)
    nodes = kd.T_nodes()
    kmin = np.array([[np.interp(T.min(), nodes, kd.kappa[n, g]) for g in range(kd.n_g)]
                     for n in range(kd.n_bands)]) * 0.05 / kd.x_ref
    ok = np.argwhere(kmin > 0.02)
    checked = 0
    for _ in range(60):
        n, g = ok[rng.integers(len(ok))]
        cell = (rng.integers(grid.nx), rng.integers(grid.ny), rng.integers(grid.nz))
        frac = rng.uniform(0.0, 1.0, 3)
        mu = rng.uniform(-1, 1)
        if abs(mu) < 0.05:
            continue
        phi = rng.uniform(0, 2 * math.pi)
        s = math.sqrt(1 - mu * mu)
        d = (s * math.cos(phi), mu, s * math.sin(phi))
        ref, nseg, tau = segment_list_X(grid, kd, T, x, int(n), int(g), cell, frac, d, 1e-6)
        got = oracle.trace_ray(grid, kd, T, x, int(n), int(g), cell, frac, d, tol=1e-6)
        assert got["X"] == pytest.approx(ref, rel=1e-9, abs=1e-12 * abs(got["abs_terms"]))
        assert got["steps"] == nseg
        checked += 1
    assert checked > 40


def test_energy_conservation_medium_exchange_sums_to_zero():
    grid = inputs.Grid(6, 10, 6, 3.0, 2.0, 3.0, T_wall=(500.0, 1000.0))
    kd = inputs.make_kdist(0)
    T, x = _field(grid, 13)
    res = oracle.solve(grid, kd, T, x, rays=1024, seed=9, tol=1e-9, max_steps=1 << 20)
    V = (grid.lx / grid.nx) * (grid.ly / grid.ny) * (grid.lz / grid.nz)
    q_mm = res["q"] - res["q_wall"]
    total_mm = V * q_mm.sum()
    # conservative standard error of the medium part: sigma_mm <= sigma + sigma_wall
    se = V * np.sqrt(((res["sigma"] + res["sigma_wall"]) ** 2).sum())
    assert abs(total_mm) < 3.0 * se, (total_mm, se)
    # the medium-medium exchange is large cell by cell, only its sum cancels
    assert V * np.abs(q_mm).sum() > 20.0 * se
    # so the volume integral of Q equals the net wall exchange
    assert abs(V * res["q"].sum() - V * res["q_wall"].sum()) < 3.0 * se


def _grey_kdist_kappa_of_T():
    """One band, kappa = 0.8 (T/1000)^2 at x_ref (so kappa differs cell to cell)."""
    Tn = np.linspace(0.0, 2000.0, 21)
    return inputs.KDist(w_g=np.array([1.0]), T0=0.0, dT=100.0, nT=21,
                        kappa=(0.8 * (np.maximum(Tn, 300.0) / 1000.0) ** 2)[None, None, :].copy(),
                        B=(inputs.SIGMA_SB * Tn**4 / math.pi)[None, :].copy(), x_ref=0.1)


def test_reciprocity_of_exchange_factors():
    grid = inputs.Grid(4, 8, 4, 2.0, 2.0, 2.0, T_wall=(500.0, 1000.0))
    kd = _grey_kdist_kappa_of_T()
    T, x = _field(grid, 14)
    G, se, _, _ = oracle.exchange(grid, kd, T, x, rays=3000, seed=15, tol=1e-9)
    iu = np.triu_indices(grid.ncells, 1)
    a, b = G[iu], G.T[iu]
    s = np.sqrt(se[iu] ** 2 + se.T[iu] ** 2)
    keep = (s > 0) & (np.maximum(a, b) > 5 * s)
    z = (a[keep] - b[keep]) / s[keep]
    assert keep.sum() > 4000
    assert np.mean(np.abs(z) > 3) < 0.01
    assert abs(z.mean()) < 4 / math.sqrt(z.size)
    assert np.max(np.abs(z)) < 5.5
    # the identity is not trivial: exchange factors without the emitting cell's
    # kappa_i (a plausible slip in Eq. 14) are far from symmetric
    kap = np.interp(T.reshape(-1), kd.T_nodes(), kd.kappa[0, 0]) * x.reshape(-1) / kd.x_ref
    ki, kj = kap[iu[0]][keep], kap[iu[1]][keep]
    zbad = (a[keep] / ki - b[keep] / kj) / (s[keep] / np.sqrt(ki * kj))
    assert np.mean(np.abs(zbad) > 3) > 0.3


def _small_kdist():
    kd = inputs.make_kdist(3, n_bands=3, n_g=2)
    return kd


def test_mc_mean_matches_deterministic_quadrature_centre_origin():
    grid = inputs.Grid(4, 8, 4, 2.0, 2.0, 2.0, T_wall=(500.0, 1000.0))
    kd = _small_kdist()
    T, x = _field(grid, 16)
    q_quad = oracle.quadrature(grid, kd, T, x, nmu_panels=48, nmu_per_panel=4, nphi=192,
                               origin=1, tol=1e-12)
    res = oracle.solve(grid, kd, T, x, rays=4096, seed=17, tol=1e-12, origin=1)
    z = (res["q"].reshape(-1) - q_quad) / res["sigma"].reshape(-1)
    assert np.max(np.abs(z)) < 4.5, np.round(z, 2)
    assert np.sqrt(np.mean(z**2)) < 1.4
    # error shrinks like 1/sqrt(N): 16x fewer rays, ~4x larger RMS error
    small = oracle.solve(grid, kd, T, x, rays=256, seed=18, tol=1e-12, origin=1)
    e_small = np.sqrt(np.mean((small["q"].reshape(-1) - q_quad) ** 2))
    e_big = np.sqrt(np.mean((res["q"].reshape(-1) - q_quad) ** 2))
    assert 2.5 < e_small / e_big < 6.5


def test_mc_uniform_origin_matches_quadrature_over_random_origins():
    """f_V = 1/V_i (Eq. 4): the uniform-origin MC mean equals the angular
    quadrature averaged over origins drawn independently (numpy) in the cell; the
    comparison carries both sampling errors.  The cell average is far from the
    centre value here, so a wrong origin law would show."""
    grid = inputs.Grid(4, 8, 4, 2.0, 2.0, 2.0, T_wall=(500.0, 1000.0))
    kd = _small_kdist()
    T, x = _field(grid, 16)
    cells = np.array([0, 37, 77, 127])
    origins = np.random.default_rng(19).uniform(0.0, 1.0, (64, 3))
    per_origin = np.array([oracle.quadrature(grid, kd, T, x, cells=cells, nmu_panels=16,
                                             nmu_per_panel=4, nphi=64, origin=0,
                                             origins=o[None, :], tol=1e-12)
                           for o in origins])
    q_ref = per_origin.mean(axis=0)
    se_ref = per_origin.std(axis=0, ddof=1) / math.sqrt(len(origins))
    res = oracle.solve(grid, kd, T, x, rays=8192, seed=17, tol=1e-12, origin=0)
    q_mc = res["q"].reshape(-1)[cells]
    s_mc = res["sigma"].reshape(-1)[cells]
    z = (q_mc - q_ref) / np.sqrt(s_mc**2 + se_ref**2)
    assert np.max(np.abs(z)) < 4.0, np.round(z, 2)
    centre = oracle.quadrature(grid, kd, T, x, cells=cells, nmu_panels=16, nmu_per_panel=4,
                               nphi=64, origin=1, tol=1e-12)
    assert np.max(np.abs(q_ref - centre) / np.sqrt(s_mc**2 + se_ref**2)) > 5.0
