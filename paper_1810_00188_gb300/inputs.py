"""Seeded synthetic inputs: grids, temperature / H2O fields and k-distribution tables.

This module produces the *inputs* of the Q_rad solve and nothing else: it holds
none of the estimator's arithmetic (no sampling, marching, tallies or proposal
construction).  Both the CUDA library and the CPU oracle consume what it builds.

The paper's own inputs (HITRAN-fitted narrow-band correlated-k tables, DNS
temperature snapshots) are not available; these generators stand in for them
with the shapes of the paper's workloads:

* property tables on uniform temperature nodes, looked up with linear
  interpolation in T (the paper tabulates the blackbody intensity per narrow band
  and the absorption coefficient per band and quadrature point, Section 2.2);
* narrow bands with Gauss quadrature points and weights (Section 2.1, Eq. 16);
* a channel geometry (walls normal to y, periodic in x and z) as in the paper's
  DNS coupling (Section 5) and the performance case (Section 3).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# CODATA 2018 exact SI constants and the derived Stefan-Boltzmann constant.
H_PLANCK = 6.62607015e-34
C_LIGHT = 299792458.0
K_BOLTZ = 1.380649e-23
SIGMA_SB = 5.670374419e-8


@dataclasses.dataclass
class Grid:
    """Cartesian grid; y is wall-normal, x and z are periodic and uniform.  y is
    uniform too unless ``yf`` holds the ny + 1 wall-normal face coordinates
    0 = y_0 < ... < y_ny = ly of a stretched grid."""

    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    eps_wall: tuple = (1.0, 1.0)   # emissivity of the walls at y=0 and y=ly
    T_wall: tuple = (0.0, 0.0)     # temperature [K] of the walls at y=0 and y=ly
    reflect: int = 0               # 0 diffuse, 1 specular reflection at grey walls
    yf: object = None              # [ny + 1] wall-normal faces of a stretched grid, or None
    xz_walls: int = 0              # 1: black walls on the x and z faces too (a closed box)
    T_xz: tuple = (0.0, 0.0, 0.0, 0.0)  # their temperatures: x = 0, x = lx, z = 0, z = lz

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self) -> tuple:
        """numpy shape of a field array: [nz][ny][nx], x fastest."""
        return (self.nz, self.ny, self.nx)

    def y_faces(self) -> np.ndarray:
        if self.yf is not None:
            return np.asarray(self.yf, dtype=np.float64)
        return np.arange(self.ny + 1) * (self.ly / self.ny)

    def cell_centers_y(self) -> np.ndarray:
        if self.yf is not None:
            f = np.asarray(self.yf, dtype=np.float64)
            return 0.5 * (f[:-1] + f[1:])
        dy = self.ly / self.ny
        return (np.arange(self.ny) + 0.5) * dy


def sin_cube(n: int = 32, kappa: float = 0.5):
    """The paper's grey verification cases 3 (kappa = 0.5 1/m) and 4 (kappa = 5):
    a 1 m cube with cold black walls on all six faces and
    T = (sin(pi x) sin(pi y) sin(pi z) pi / sigma)^(1/4) at the cell centres
    (so sigma T^4 / pi = sin sin sin)."""
    grid = Grid(n, n, n, 1.0, 1.0, 1.0, eps_wall=(1.0, 1.0), T_wall=(0.0, 0.0), xz_walls=1)
    c = (np.arange(n) + 0.5) / n
    s = np.sin(np.pi * c)
    E = s[None, None, :] * s[None, :, None] * s[:, None, None]   # [z, y, x]
    T = (E * np.pi / SIGMA_SB) ** 0.25
    kd = make_grey_kdist(kappa, T_max=float(T.max()) * 1.05 + 1.0, nT=512)
    return grid, kd, T, np.full(grid.shape, kd.x_ref)


def channel_faces(ny: int, ly: float, gamma: float = 1.5) -> np.ndarray:
    """Wall-normal faces of a channel grid refined towards both walls with the
    hyperbolic-tangent stretching common in channel DNS:
    y_j = ly/2 (1 + tanh(gamma (2 j / ny - 1)) / tanh(gamma)); gamma -> 0 is
    uniform.  The end faces are exactly 0 and ly."""
    j = np.arange(ny + 1)
    y = 0.5 * ly * (1.0 + np.tanh(gamma * (2.0 * j / ny - 1.0)) / np.tanh(gamma))
    y[0], y[-1] = 0.0, ly
    return y


@dataclasses.dataclass
class KDist:
    """Narrow-band correlated-k tables on uniform T nodes.

    kappa[n][g][t] is the absorption coefficient [1/m] at H2O mole fraction
    x_ref; B[n][t] is the band blackbody intensity dnu_n * I_b(nu_n, T_t)
    [W m^-2 sr^-1]; w_g are the quadrature weights (summing to 1).
    """

    w_g: np.ndarray
    T0: float
    dT: float
    nT: int
    kappa: np.ndarray
    B: np.ndarray | None             # None: the solver computes it from nu_c and dnu
    x_ref: float = 0.1
    nu_c: np.ndarray | None = None   # band centres [1/cm]
    dnu: np.ndarray | None = None    # band widths [1/cm]

    @property
    def n_bands(self) -> int:
        return int(self.kappa.shape[0])

    @property
    def n_g(self) -> int:
        return int(self.kappa.shape[1])

    def T_nodes(self) -> np.ndarray:
        return self.T0 + self.dT * np.arange(self.nT)


def gauss_legendre_01(n: int):
    """n-point Gauss-Legendre nodes and weights mapped to [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def planck_band_intensity(nu_c_cm: np.ndarray, dnu_cm: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Band blackbody intensity dnu * 2 h c^2 nu^3 / (exp(h c nu / k T) - 1).

    nu in wavenumber [1/m] (input in 1/cm); returns [len(nu), len(T)] in
    W m^-2 sr^-1.  T = 0 gives 0.
    """
    nu = 100.0 * np.asarray(nu_c_cm, dtype=np.float64)[:, None]
    dnu = 100.0 * np.asarray(dnu_cm, dtype=np.float64)[:, None]
    T = np.asarray(T, dtype=np.float64)[None, :]
    with np.errstate(over="ignore", divide="ignore"):
        x = np.where(T > 0, H_PLANCK * C_LIGHT * nu / (K_BOLTZ * np.where(T > 0, T, 1.0)), np.inf)
        out = dnu * 2.0 * H_PLANCK * C_LIGHT**2 * nu**3 / np.expm1(x)
    return np.where(T > 0, out, 0.0)


def make_grey_kdist(kappa: float, T_max: float = 2000.0, nT: int = 21) -> KDist:
    """One band, one g-point, constant kappa, B = sigma T^4 / pi on nodes 0..T_max.

    Used for grey cases (the paper keeps the band machinery for grey gases,
    Section 2.3).  Node 0 is 0 K so that cold walls have B = 0 exactly.
    """
    T = np.linspace(0.0, T_max, nT)
    return KDist(
        w_g=np.array([1.0]),
        T0=0.0,
        dT=float(T[1] - T[0]),
        nT=nT,
        kappa=np.full((1, 1, nT), float(kappa)),
        B=(SIGMA_SB * T**4 / math.pi)[None, :].copy(),
        x_ref=0.1,
    )


def make_kdist(seed: int = 0, n_bands: int = 40, n_g: int = 8, T0: float = 300.0,
               dT: float = 20.0, nT: int = 64, nu0_cm: float = 200.0,
               dnu_cm: float = 200.0, x_ref: float = 0.1,
               clamp_below: float | None = None) -> KDist:
    """Synthetic H2O-like narrow-band correlated-k tables.

    kappa_{n,g}(T) = k0_n (T/1000)^{a_n} exp(s_n Phi^{-1}(g_g)) at x_ref, with
    k0_n log-uniform in [1e-3, 1e2] 1/m, a_n ~ U[-1, 1], s_n ~ U[0.5, 2]
    (drawn in that order from default_rng(seed)), g_g the Gauss-Legendre nodes on
    [0, 1].  Bands are centred at nu0, nu0 + dnu, ... with width dnu [1/cm].

    clamp_below: nodes below this temperature take the kappa value at that
    temperature (lets a table start at 0 K so that cold walls have B = 0).
    """
    from scipy.special import ndtri

    rng = np.random.default_rng(seed)
    k0 = 10.0 ** rng.uniform(-3.0, 2.0, n_bands)
    a = rng.uniform(-1.0, 1.0, n_bands)
    s = rng.uniform(0.5, 2.0, n_bands)
    g, w = gauss_legendre_01(n_g)
    Tn = T0 + dT * np.arange(nT)
    Tk = Tn if clamp_below is None else np.maximum(Tn, clamp_below)
    kappa = (k0[:, None, None] * (Tk[None, None, :] / 1000.0) ** a[:, None, None]
             * np.exp(s[:, None, None] * ndtri(g)[None, :, None]))
    nu_c = nu0_cm + dnu_cm * np.arange(n_bands)
    dnu = np.full(n_bands, dnu_cm)
    B = planck_band_intensity(nu_c, dnu, Tn)
    return KDist(w_g=w, T0=T0, dT=dT, nT=nT, kappa=np.ascontiguousarray(kappa),
                 B=np.ascontiguousarray(B), x_ref=x_ref, nu_c=nu_c, dnu=dnu)


def gaussian_random_field(shape_zyx: tuple, lengths_zyx: tuple, seed: int,
                          spectrum_exponent: float = -5.0 / 3.0) -> np.ndarray:
    """Zero-mean, unit-variance periodic Gaussian random field.

    Its 3D energy spectrum E(k) ~ k^spectrum_exponent, i.e. Fourier amplitudes
    ~ k^((spectrum_exponent - 2)/2) with random phases (white noise filtered by
    FFT); the k = 0 mode is removed.
    """
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape_zyx)
    ks = [2.0 * np.pi * np.fft.fftfreq(n, d=L / n) for n, L in zip(shape_zyx, lengths_zyx)]
    kz, ky, kx = np.meshgrid(*ks, indexing="ij")
    kmag = np.sqrt(kx**2 + ky**2 + kz**2)
    amp = np.zeros_like(kmag)
    nz = kmag > 0
    amp[nz] = kmag[nz] ** ((spectrum_exponent - 2.0) / 2.0)
    f = np.fft.ifftn(np.fft.fftn(noise) * amp).real
    f -= f.mean()
    sd = f.std()
    return f / sd if sd > 0 else f


def channel_fields(grid: Grid, seed: int, T_lo: float = 500.0, T_hi: float = 1000.0,
                   fluct: float = 0.05, x_mode: str = "const", x_const: float = 0.1):
    """Synthetic turbulent-channel fields (T [K], x_H2O) with shape [nz][ny][nx].

    T = (T_lo + (T_hi - T_lo) y / ly) (1 + fluct G), G a k^-5/3 Gaussian random
    field.  x_mode "const" gives x = x_const; "field" gives
    x = 0.05 + 0.15 Phi(G2) with an independent field G2 of the same spectrum.
    """
    from scipy.special import ndtr

    lengths = (grid.lz, grid.ly, grid.lx)
    y = grid.cell_centers_y()
    base = T_lo + (T_hi - T_lo) * y / grid.ly
    G = gaussian_random_field(grid.shape, lengths, seed)
    T = base[None, :, None] * (1.0 + fluct * G)
    if x_mode == "const":
        x = np.full(grid.shape, x_const)
    elif x_mode == "field":
        G2 = gaussian_random_field(grid.shape, lengths, seed + 7919)
        x = 0.05 + 0.15 * ndtr(G2)
    else:
        raise ValueError(x_mode)
    return np.ascontiguousarray(T), np.ascontiguousarray(x)


# --- named workloads ------------------------------------------------------------

def grey_slab_16x32x16(kappa: float = 1.0, T: float = 1000.0):
    """Grey isothermal slab 16x32x16, cubic cells of 1/16 m (1 x 2 x 1 m),
    periodic x, z, cold black walls at y = 0 and y = 2 m."""
    grid = Grid(16, 32, 16, 1.0, 2.0, 1.0, eps_wall=(1.0, 1.0), T_wall=(0.0, 0.0))
    kd = make_grey_kdist(kappa)
    Tf = np.full(grid.shape, float(T))
    xf = np.full(grid.shape, kd.x_ref)
    return grid, kd, Tf, xf


def nongrey_channel(nx: int = 64, ny: int = 64, nz: int = 64, seed: int = 0,
                    kdist_seed: int = 0, eps_wall: float = 1.0, x_mode: str = "const"):
    """Non-grey channel 4 pi x 2 x 2 pi m with 40 x 8 synthetic k-distribution,
    black (or grey) walls at 500 K (y = 0) and 1000 K (y = 2 m), linear mean T
    with 5% k^-5/3 fluctuations."""
    grid = Grid(nx, ny, nz, 4.0 * math.pi, 2.0, 2.0 * math.pi,
                eps_wall=(eps_wall, eps_wall), T_wall=(500.0, 1000.0))
    kd = make_kdist(kdist_seed)
    T, x = channel_fields(grid, seed, x_mode=x_mode)
    return grid, kd, T, x


SNAPSHOT_SHAPES = ((32, 32, 32), (48, 64, 48), (96, 96, 96), (128, 128, 128))


def snapshot_batch(n: int = 32, seed: int = 0, shapes=SNAPSHOT_SHAPES, x_mode: str = "field"):
    """Independent channel snapshots of uneven grid sizes: shape k drawn from
    `shapes` with default_rng(seed), fields seeded with seed + 1 + k (x_H2O a
    random field by default), black walls at 500 / 1000 K, one shared 40 x 8
    k-distribution.  Returns (kdist, [(grid, T, x), ...])."""
    rng = np.random.default_rng(seed)
    picks = rng.integers(0, len(shapes), n)
    kd = make_kdist(0)
    snaps = []
    for k, i in enumerate(picks):
        nx, ny, nz = shapes[int(i)]
        grid = Grid(nx, ny, nz, 4.0 * math.pi, 2.0, 2.0 * math.pi, T_wall=(500.0, 1000.0))
        T, x = channel_fields(grid, seed + 1 + k, x_mode=x_mode)
        snaps.append((grid, T, x))
    return kd, snaps
