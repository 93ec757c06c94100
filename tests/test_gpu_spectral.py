"""GPU per-cell spectral proposals at the cells' own temperatures (the classic
ERMC draw and its temperature-weighted mix with Zhang's T_max pdf): the
quantised counts against the oracle's FP64 probabilities, and solves with them
at parity with the oracle on the same counts."""
import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs, mcrt

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [mcrt.MCRT_SPECTRAL_LOCAL, mcrt.MCRT_SPECTRAL_HYBRID])
def test_spectral_proposal_counts_and_solve_parity(mode):
    grid, kd, T, x = inputs.nongrey_channel(12, 16, 8, seed=51, eps_wall=0.8, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    S.set_spectral_proposal(mode)
    cn, cg, hemi = S.cell_proposal()
    nb, ng = kd.n_bands, kd.n_g
    q = oracle.spectral_proposal(grid, kd, T, x, mode=mode)
    cnf = cn.reshape(grid.ncells, nb).astype(np.float64)
    cgf = cg.reshape(grid.ncells, nb, ng).astype(np.float64)
    pn = np.diff(np.concatenate([np.zeros((grid.ncells, 1)), cnf], axis=1), axis=1) * 2.0**-32
    pg = np.diff(np.concatenate([np.zeros((grid.ncells, nb, 1)), cgf], axis=2), axis=2) * 2.0**-32
    p = (pn[:, :, None] * pg).reshape(grid.ncells, -1)
    # FP32 weights against FP64 probabilities, after quantisation to 2^32 counts
    qn = q.reshape(grid.ncells, nb, ng).sum(axis=2)
    assert np.all(np.abs(pn - qn) <= 2e-5 * qn + 4.7e-10)
    assert np.all(np.abs(p - q) <= 5e-3 * q + 1e-9)
    assert np.all(hemi == (1 << 22))
    # solves with the device's counts: FP32 and FP64 at parity with the oracle
    box = (0, 12, 0, 16, 3, 5)
    sel = [i + 12 * (j + 16 * k) for k in range(3, 5) for j in range(16) for i in range(12)]
    prop = (cn.reshape(grid.ncells, nb)[sel], cg.reshape(grid.ncells, nb * ng)[sel], hemi[sel])
    o = oracle.solve(grid, kd, T, x, rays=96, seed=4, box=box, proposal=prop)
    for prec, rtol in ((mcrt.MCRT_FP64, 1e-10), (mcrt.MCRT_FP32, 1e-4)):
        qq, _ = S.solve(box=box, rays=96, seed=4, precision=prec, proposal=mcrt.MCRT_PROPOSAL_CELL)
        assert np.all(np.abs(qq - o["q"]) <= rtol * o["scale"]), prec
    with pytest.raises(mcrt.McrtError):
        S.set_spectral_proposal(7)
    S.close()


def test_band_intensities_computed_by_the_library():
    """B = NULL with band centres and widths: the library's FP64 Planck table
    gives the same solves as the supplied table (and the oracle's), including a
    T axis that starts at 0 K, where the intensity is 0; missing or
    non-positive band data are argument errors."""
    import dataclasses
    grid = inputs.Grid(12, 16, 8, 4.0, 2.0, 2.0, eps_wall=(0.7, 1.0), T_wall=(0.0, 1000.0))
    kd = inputs.make_kdist(3, n_bands=12, n_g=4, T0=0.0, dT=25.0, nT=64, clamp_below=300.0)
    T, x = inputs.channel_fields(grid, 61, x_mode="field")
    kd_nob = dataclasses.replace(kd, B=None)
    box = (0, 12, 0, 16, 2, 4)
    o = oracle.solve(grid, kd, T, x, rays=64, seed=7, box=box)
    out = {}
    for name, k in (("given", kd), ("computed", kd_nob)):
        S = mcrt.Solver(grid, k)
        S.set_fields(T, x)
        out[name] = [S.solve(box=box, rays=64, seed=7, precision=p)[0]
                     for p in (mcrt.MCRT_FP64, mcrt.MCRT_FP32)]
        out[name].append(S.plain_probs())
        S.close()
    g64, g32, gp = out["given"]
    c64, c32, cp = out["computed"]
    assert np.array_equal(gp, cp)
    assert np.all(np.abs(c64 - g64) <= 1e-12 * o["scale"])
    assert np.all(np.abs(c32 - g32) <= 1e-6 * o["scale"])
    assert np.all(np.abs(c64 - o["q"]) <= 1e-10 * o["scale"])
    S = mcrt.Solver(grid, kd)
    for bad in (dataclasses.replace(kd_nob, nu_c=None),
                dataclasses.replace(kd_nob, dnu=np.where(np.arange(kd.n_bands) == 3, 0.0, kd.dnu)),
                dataclasses.replace(kd_nob, nu_c=np.where(np.arange(kd.n_bands) == 5, np.nan, kd.nu_c))):
        with pytest.raises(mcrt.McrtError) as e:
            S.set_kdist(bad)
        assert e.value.status == mcrt.MCRT_E_ARG
    S.close()
