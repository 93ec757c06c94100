"""GPU parity of the absorption-based estimate (ARMC) and of its combination
with the emission-based one, against the oracle (oracle.solve_armc) on the same
draws.

The kernel deposits binary32 segment terms with binary64 atomic adds, the
oracle sums binary64 terms in a fixed order, so the comparison uses the FP32
tolerance of the emission-based parity tests, |Q - Q_oracle| <= 1e-4 S_i, with
S_i the oracle's mean absolute deposit into cell i (its exchange terms can
cancel, as the emission-based ones do).  The batch-means standard errors come
from the same batches of ray indices on both sides.
"""
import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs, mcrt

pytestmark = pytest.mark.gpu


def _solve(grid, kd, T, x, est, rays, seed, precision=mcrt.MCRT_FP32, **kw):
    import torch
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    q = torch.full(grid.shape, float("nan"), dtype=torch.float64, device="cuda")
    s = torch.full_like(q, float("nan"))
    st = torch.zeros(grid.shape, dtype=torch.int64, device="cuda")
    S.solve_into(S.params(rays=rays, seed=seed, precision=precision, estimator=est, **kw), q, s, st)
    stats = S.stats()
    S.close()
    return q.cpu().numpy(), s.cpu().numpy(), st.cpu().numpy(), stats


@pytest.mark.parametrize("reflect", [0, 1])
def test_armc_and_hybrid_against_oracle(reflect):
    grid, kd, T, x = inputs.nongrey_channel(16, 16, 12, seed=31, eps_wall=0.8, x_mode="field")
    grid.reflect = reflect
    rays, seed = 80, 13
    orc = oracle.solve_armc(grid, kd, T, x, rays=rays, seed=seed, hybrid=True)
    e = oracle.solve(grid, kd, T, x, rays=rays, seed=seed)
    qa, sa, st, stats = _solve(grid, kd, T, x, mcrt.MCRT_EST_ARMC, rays, seed)
    scale = np.maximum(orc["scale"], 1e-300)
    err = np.abs(qa - orc["q"]) / scale
    assert err.max() <= 1e-4, err.max()
    big = orc["sigma"] > 1e-3 * scale
    np.testing.assert_allclose(sa[big], orc["sigma"][big], rtol=2e-2)
    # the cells' own rays: the same step counts as the emission-based solve
    assert abs(st.sum() / e["steps"].sum() - 1.0) < 1e-3
    assert stats["rays"] == grid.ncells * rays
    qh, sh, _, _ = _solve(grid, kd, T, x, mcrt.MCRT_EST_HYBRID, rays, seed)
    sc = np.maximum(np.maximum(orc["scale"], e["scale"]), 1e-300)
    errh = np.abs(qh - orc["q_hybrid"]) / sc
    assert errh.max() <= 1e-4, errh.max()
    bigh = orc["sigma_hybrid"] > 1e-3 * sc
    np.testing.assert_allclose(sh[bigh], orc["sigma_hybrid"][bigh], rtol=2e-2)


def test_armc_with_long_rays_handed_off():
    """Rays handed to the warp-parallel long-ray march (here after 8 segments,
    whatever the flight: thousands of them) make their deposits there -- each
    lane's pieces with the transmissivity at the lane's start, the stopping lane's
    up to the stop, walls and the residual by one lane: ARMC and the hybrid still
    agree with the oracle, and the cells' own rays take the same steps."""
    import torch
    grid, kd, T, x = inputs.nongrey_channel(16, 16, 12, seed=31, eps_wall=0.8, x_mode="field")
    rays, seed = 80, 13
    orc = oracle.solve_armc(grid, kd, T, x, rays=rays, seed=seed, hybrid=True)
    e = oracle.solve(grid, kd, T, x, rays=rays, seed=seed)
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    S.set_tuning(long_ray_steps=8, long_ray_flight=-1)
    for est, key, skey in ((mcrt.MCRT_EST_ARMC, "q", "sigma"), (mcrt.MCRT_EST_HYBRID, "q_hybrid", "sigma_hybrid")):
        q = torch.full(grid.shape, float("nan"), dtype=torch.float64, device="cuda")
        s = torch.full_like(q, float("nan"))
        st = torch.zeros(grid.shape, dtype=torch.int64, device="cuda")
        S.solve_into(S.params(rays=rays, seed=seed, precision=mcrt.MCRT_FP32, estimator=est), q, s, st)
        stats = S.stats()
        assert stats["long_rays"] > 1000 and stats["long_overflow"] == 0, stats
        sc = orc["scale"] if est == mcrt.MCRT_EST_ARMC else np.maximum(orc["scale"], e["scale"])
        sc = np.maximum(sc, 1e-300)
        err = np.abs(q.cpu().numpy() - orc[key]) / sc
        assert err.max() <= 1e-4, (est, err.max())
        big = orc[skey] > 1e-3 * sc
        np.testing.assert_allclose(s.cpu().numpy()[big], orc[skey][big], rtol=2e-2)
        assert abs(st.cpu().numpy().sum() / e["steps"].sum() - 1.0) < 1e-3
    S.close()


@pytest.mark.parametrize("geometry", ["channel", "stretched", "box"])
def test_armc_fp64_against_oracle(geometry):
    """The FP64 parity mode of the absorption-based estimate: binary64 deposits
    into the same per-batch sums, so Q and the hybrid agree with the oracle to
    rounding (10^-10 S_i; the atomic adds reorder the binary64 sums), sigma too,
    and the cells' own rays take the oracle's steps exactly."""
    if geometry == "box":
        grid, kd, T, x = inputs.sin_cube(10, 5.0)
    else:
        grid, kd, T, x = inputs.nongrey_channel(10, 12, 8, seed=37, eps_wall=0.8, x_mode="field")
        if geometry == "stretched":
            grid.yf = inputs.channel_faces(grid.ny, grid.ly, 1.5)
            T, x = inputs.channel_fields(grid, 37, x_mode="field")
    rays, seed = 40, 19
    orc = oracle.solve_armc(grid, kd, T, x, rays=rays, seed=seed, hybrid=True)
    e = oracle.solve(grid, kd, T, x, rays=rays, seed=seed)
    qa, sa, st, _ = _solve(grid, kd, T, x, mcrt.MCRT_EST_ARMC, rays, seed, precision=mcrt.MCRT_FP64)
    scale = np.maximum(orc["scale"], 1e-300)
    assert (np.abs(qa - orc["q"]) / scale).max() <= 1e-10
    big = orc["sigma"] > 1e-6 * scale
    np.testing.assert_allclose(sa[big], orc["sigma"][big], rtol=1e-6)
    assert np.array_equal(st, e["steps"].astype(np.int64))
    qh, _, _, _ = _solve(grid, kd, T, x, mcrt.MCRT_EST_HYBRID, rays, seed, precision=mcrt.MCRT_FP64)
    sc = np.maximum(np.maximum(orc["scale"], e["scale"]), 1e-300)
    assert (np.abs(qh - orc["q_hybrid"]) / sc).max() <= 1e-10


def test_armc_few_rays_and_ragged_grid():
    """Fewer rays than batches (K = rays) on a ragged grid, per-cell proposals."""
    grid, kd, T, x = inputs.nongrey_channel(7, 9, 5, seed=32, x_mode="field")
    rays, seed = 11, 3
    rng = np.random.default_rng(8)
    nc, nb, ng = grid.ncells, kd.n_bands, kd.n_g

    def cum(rows, k):
        c = rng.integers(1, 2**26, size=(rows, k)).astype(np.int64)
        c[:, -1] += 2**32 - c.sum(axis=1)
        return np.cumsum(c, axis=1).astype(np.uint64)

    prop = (cum(nc, nb), cum(nc * nb, ng).reshape(nc, nb, ng), rng.integers(1, 2**23, size=nc).astype(np.uint32))
    orc = oracle.solve_armc(grid, kd, T, x, rays=rays, seed=seed,
                            proposal=(prop[0], prop[1].reshape(nc, nb * ng), prop[2]))
    import torch
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    S.set_cell_proposal(*prop)
    q, s = S.solve(rays=rays, seed=seed, precision=mcrt.MCRT_FP32, proposal=mcrt.MCRT_PROPOSAL_CELL,
                   estimator=mcrt.MCRT_EST_ARMC)
    S.close()
    err = np.abs(q - orc["q"]) / np.maximum(orc["scale"], 1e-300)
    assert err.max() <= 1e-4, err.max()


def test_armc_equals_ermc_in_an_isothermal_medium():
    """Isothermal gas: every deposit is zero and both estimates are the cells'
    wall exchange from their own rays, so they agree to binary32 rounding (a
    ray's wall terms are summed in binary32 in its sample, deposited one by one
    into the binary64 sums by the absorption-based kernel)."""
    grid = inputs.Grid(8, 16, 8, 0.5, 1.0, 0.5, eps_wall=(1.0, 0.6), T_wall=(300.0, 600.0))
    kd = inputs.make_kdist(0)
    T = np.full(grid.shape, 900.0)
    x = np.full(grid.shape, 0.1)
    qa, _, _, _ = _solve(grid, kd, T, x, mcrt.MCRT_EST_ARMC, 48, 5)
    qe, _, _, _ = _solve(grid, kd, T, x, mcrt.MCRT_EST_ERMC, 48, 5)
    np.testing.assert_allclose(qa, qe, rtol=1e-6, atol=1e-9 * np.abs(qe).max())


def test_armc_refuses_what_it_does_not_support():
    import ctypes as C

    import torch
    grid, kd, T, x = inputs.nongrey_channel(8, 8, 8, seed=33)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    for kw in (dict(box=(0, 4, 0, 8, 0, 8)), dict(mg_levels=2, mg_steps=3),
               dict(precision=mcrt.MCRT_FP64, mg_levels=2, mg_steps=3)):
        kw.setdefault("precision", mcrt.MCRT_FP32)
        with pytest.raises(mcrt.McrtError) as e:
            S.solve(rays=4, estimator=mcrt.MCRT_EST_ARMC, **kw)
        assert e.value.status == mcrt.MCRT_E_UNSUPPORTED
    with pytest.raises(mcrt.McrtError) as e:
        S.solve(rays=4, estimator=7)
    assert e.value.status == mcrt.MCRT_E_ARG
    L = mcrt.load()
    q = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    p = S.params(rays=4, precision=mcrt.MCRT_FP32, estimator=mcrt.MCRT_EST_HYBRID)
    assert L.mcrt_solve_qrad_noalloc(S.ctx, C.byref(p), C.c_void_p(q.data_ptr()), None, None) == \
        mcrt.MCRT_E_UNSUPPORTED
    S.close()


@pytest.mark.parametrize("geometry", ["stretched", "box"])
def test_armc_stretched_grid_and_closed_box_against_oracle(geometry):
    """A wall-refined channel grid (each deposit scaled by the volume ratio of
    the emitting and the absorbing cell; long rays handed off with their
    deposits) and the paper's closed sin cube (the black x and z walls' terms kept
    in the emitting cell): ARMC and the hybrid against the oracle on the same
    draws."""
    if geometry == "stretched":
        grid, kd, T, x = inputs.nongrey_channel(14, 16, 10, seed=35, eps_wall=0.8, x_mode="field")
        grid.yf = inputs.channel_faces(grid.ny, grid.ly, 1.5)
        T, x = inputs.channel_fields(grid, 35, x_mode="field")
    else:
        grid, kd, T, x = inputs.sin_cube(12, 0.5)
    rays, seed = 64, 17
    orc = oracle.solve_armc(grid, kd, T, x, rays=rays, seed=seed, hybrid=True)
    e = oracle.solve(grid, kd, T, x, rays=rays, seed=seed)
    qa, sa, st, stats = _solve(grid, kd, T, x, mcrt.MCRT_EST_ARMC, rays, seed)
    scale = np.maximum(orc["scale"], 1e-300)
    err = np.abs(qa - orc["q"]) / scale
    assert err.max() <= 1e-4, err.max()
    big = orc["sigma"] > 1e-3 * scale
    np.testing.assert_allclose(sa[big], orc["sigma"][big], rtol=2e-2)
    assert abs(st.sum() / e["steps"].sum() - 1.0) < 1e-3
    qh, sh, _, _ = _solve(grid, kd, T, x, mcrt.MCRT_EST_HYBRID, rays, seed)
    sc = np.maximum(np.maximum(orc["scale"], e["scale"]), 1e-300)
    assert (np.abs(qh - orc["q_hybrid"]) / sc).max() <= 1e-4
