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
