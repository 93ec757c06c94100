"""Oracle pins of the absorption-based reciprocal estimate (ARMC, Section 2).

The paper names two reciprocal formulations: the emission-based one (ERMC,
Eq. 14's per-ray form; cell i's exchanges from cell i's own rays) and the
absorption-based one, which estimates the power cell i absorbs from the rays
emitted elsewhere; Eq. FM and the reciprocity relation make the two estimates of
the same Q^R_i.  `oracle.solve_armc` takes cell i's exchange with every other
medium cell from the rays of that cell absorbed in i, and its exchange with the
walls from its own rays.  These tests hold it to:
  * the exact layered solution of the paper's Table 1 cases 1 and 2;
  * an identity on the same draws: the medium exchange it moves between cells
    sums (volume-weighted) to minus the emission-based medium exchange, while
    the wall parts are the same terms -- so sum V Q_A = sum V (2 Q_E,wall - Q_E);
  * equality with the emission-based estimate when the medium is isothermal;
  * no bias against the emission-based estimate on a 3D turbulent field;
  * the variance property the paper states for cold zones.
"""
import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs

from test_oracle_slab import _layer_exact, _paper_cases, assert_rows


def _volumes(grid):
    dy = np.diff(grid.yf) if getattr(grid, "yf", None) is not None else np.full(grid.ny, grid.ly / grid.ny)
    return (grid.lx / grid.nx) * (grid.lz / grid.nz) * dy[None, :, None] * np.ones((grid.nz, 1, grid.nx))


def _row_z_batches(res, ref):
    """z-scores of the x-z averaged rows, the standard error from the batch means
    of the row averages (deposits of one ray land in several cells of a row)."""
    qb = res["q_batches"].mean(axis=(1, 3))  # [K, ny]
    K = qb.shape[0]
    se = qb.std(axis=0, ddof=1) / np.sqrt(K)
    return (res["q"].mean(axis=(0, 2)) - ref) / se


@pytest.mark.parametrize("name", ["case1", "case2"])
def test_armc_paper_grey_cases_layer_exact(name):
    """Table 1 cases 1 (lin1) and 2 (parab): the absorption-based estimate of the
    layered slab between black walls matches its exact solution (E3 layer-to-layer
    kernels in closed form)."""
    c = _paper_cases()[name]
    ny = 32
    grid = inputs.Grid(4, ny, 4, 1.0, c["L"], 1.0, eps_wall=(1.0, 1.0), T_wall=c["Tw"])
    kd = inputs.make_grey_kdist(c["kap"], T_max=2000.0, nT=21)
    y = grid.cell_centers_y()
    prof = 500.0 + 1000.0 * y if c["profile"] == "lin1" else 500.0 - 2000.0 * y**2 + 2000.0 * y
    T = np.broadcast_to(prof[None, :, None], grid.shape).copy()
    nodes = kd.T_nodes()
    Bm = np.interp(prof, nodes, kd.B[0])
    Bw = [np.interp(t, nodes, kd.B[0]) for t in c["Tw"]]
    ref = _layer_exact(c["kap"], c["L"], ny, Bm, Bw[0], Bw[1])
    res = oracle.solve_armc(grid, kd, T, None, rays=2048, seed=7, tol=1e-12, batches=32)
    assert_rows(_row_z_batches(res, ref))


@pytest.mark.parametrize("stretched", [False, True, "box"])
def test_armc_moves_the_medium_exchange_on_the_same_draws(stretched):
    """Same draws: each ray deposits minus its emission-based medium terms (and
    residual) into the cells that absorb, scaled by the volume ratio, and keeps its
    wall terms in its own cell (the black x and z walls of a closed box too).
    Hence, exactly up to rounding, sum_i V_i Q_A,i = sum_i V_i (2 Q_E,wall,i -
    Q_E,i).  A wrong sign, a dropped deposit, a residual in the wrong cell or a
    missing volume ratio breaks it."""
    if stretched == "box":
        grid, kd, T, x = inputs.sin_cube(6, 0.5)
    else:
        grid, kd, T, x = inputs.nongrey_channel(8, 10, 6, seed=3, eps_wall=0.8, x_mode="field")
    if stretched is True:
        grid.yf = inputs.channel_faces(grid.ny, grid.ly, 1.5)
    a = oracle.solve_armc(grid, kd, T, x, rays=32, seed=1)
    e = oracle.solve(grid, kd, T, x, rays=32, seed=1)
    V = _volumes(grid)
    lhs = (V * a["q"]).sum()
    rhs = (V * (2.0 * e["q_wall"] - e["q"])).sum()
    assert abs(lhs - rhs) <= 1e-12 * (V * e["scale"]).sum()
    # the deposits are not trivially zero: the medium part is a large fraction
    assert np.abs(a["q"] - e["q_wall"]).sum() > 0.1 * np.abs(e["q_wall"]).sum()
    assert np.array_equal(a["steps"], e["steps"])


def test_armc_equals_ermc_in_an_isothermal_medium():
    """Isothermal gas between cold black walls: every medium deposit is zero
    (B_j = B_i), so both estimates are the wall exchange of each cell's own rays
    (the E3 closed form pins that one)."""
    grid, kd, T, x = inputs.grey_slab_16x32x16(1.0)
    grid = inputs.Grid(4, 16, 4, 0.25, 1.0, 0.25, eps_wall=grid.eps_wall, T_wall=grid.T_wall)
    T = np.full(grid.shape, 1000.0)
    a = oracle.solve_armc(grid, kd, T, None, rays=64, seed=4, tol=1e-6)
    e = oracle.solve(grid, kd, T, None, rays=64, seed=4, tol=1e-6)
    np.testing.assert_allclose(a["q"], e["q"], rtol=1e-12, atol=1e-9 * np.abs(e["q"]).max())


def test_armc_unbiased_against_ermc():
    """Independent draws on a 3D turbulent channel: the two estimates of the same
    Q^R agree -- per cell (|z| > 4 in at most 0.5% of the cells, the batch-means
    standard error having 15 degrees of freedom) and for the grid total over
    several seeds (batch means of the absorption-based totals; the emission-based
    cells are independent)."""
    grid, kd, T, x = inputs.nongrey_channel(12, 16, 12, seed=5)
    zs = []
    for sd in (11, 21, 31, 41):
        a = oracle.solve_armc(grid, kd, T, x, rays=128, seed=sd)
        e = oracle.solve(grid, kd, T, x, rays=128, seed=sd + 1)
        z = (a["q"] - e["q"]) / np.sqrt(a["sigma"] ** 2 + e["sigma"] ** 2)
        assert np.mean(np.abs(z) > 4) <= 0.005
        K = a["q_batches"].shape[0]
        tot = a["q_batches"].reshape(K, -1).sum(1)
        se = np.hypot(tot.std(ddof=1) / np.sqrt(K), np.sqrt((e["sigma"] ** 2).sum()))
        zs.append((a["q"].sum() - e["q"].sum()) / se)
    assert abs(np.sum(zs) / np.sqrt(len(zs))) < 3.0, zs


def test_armc_lower_variance_in_the_cold_zone():
    """Section 2: the absorption-based estimate has the lower variance where the
    gas is cold and absorbs radiation from hotter zones.  On the channel (walls
    500 / 1000 K, T_max spectral pdf for both), the median standard error of the
    coldest tenth of the cells is clearly lower at the same rays per cell."""
    grid, kd, T, x = inputs.nongrey_channel(12, 16, 12, seed=5)
    a = oracle.solve_armc(grid, kd, T, x, rays=256, seed=11)
    e = oracle.solve(grid, kd, T, x, rays=256, seed=12)
    Tf = T.reshape(-1)
    cold = Tf <= np.percentile(Tf, 10)
    ratio = np.median(a["sigma"].reshape(-1)[cold] / e["sigma"].reshape(-1)[cold])
    assert ratio < 0.85, ratio
