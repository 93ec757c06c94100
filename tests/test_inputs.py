"""Checks of the synthetic input generators (not of the method)."""
import math

import numpy as np

from paper_1810_00188_gb300 import inputs


def test_planck_bands_sum_to_stefan_boltzmann():
    # 1/cm-wide bands over 0.5 .. 30000 1/cm hold sigma T^4 / pi to 1e-5
    nu = np.arange(0.5, 30000.0, 1.0)
    for T in (300.0, 1000.0, 2000.0):
        B = inputs.planck_band_intensity(nu, np.ones_like(nu), np.array([T]))[:, 0]
        assert abs(B.sum() / (inputs.SIGMA_SB * T**4 / math.pi) - 1.0) < 1e-5


def test_planck_wien_peak_and_zero_kelvin():
    nu = np.linspace(10.0, 10000.0, 20000)
    B = inputs.planck_band_intensity(nu, np.ones_like(nu), np.array([1000.0, 0.0]))
    # Wien's law in wavenumber: nu_max = 1.9609 cm^-1/K * T
    assert abs(nu[np.argmax(B[:, 0])] / 1960.9 - 1.0) < 2e-3
    assert np.all(B[:, 1] == 0.0)


def test_kdist_table_shapes_and_coverage():
    kd = inputs.make_kdist(0)
    assert kd.kappa.shape == (40, 8, 64) and kd.B.shape == (40, 64)
    assert abs(kd.w_g.sum() - 1.0) < 1e-14
    assert kd.T_nodes()[-1] == 300.0 + 20.0 * 63
    # the 40 bands of 200 1/cm hold > 98% of sigma T^4 / pi at 1000 K
    it = int((1000.0 - kd.T0) / kd.dT)
    assert kd.B[:, it].sum() / (inputs.SIGMA_SB * 1e12 / math.pi) > 0.98
    assert 1e-6 < kd.kappa.min() and kd.kappa.max() < 1e4


def test_random_field_statistics():
    g = inputs.Grid(32, 32, 32, 4 * math.pi, 2.0, 2 * math.pi)
    G = inputs.gaussian_random_field(g.shape, (g.lz, g.ly, g.lx), 0)
    assert abs(G.mean()) < 1e-12 and abs(G.std() - 1.0) < 1e-12
    T, x = inputs.channel_fields(g, 0, x_mode="field")
    assert 0.05 <= x.min() and x.max() <= 0.2
    prof = T.mean(axis=(0, 2))
    assert np.allclose(prof, 500.0 + 500.0 * g.cell_centers_y() / 2.0, rtol=0.02)
