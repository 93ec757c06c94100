"""FP64 CPU oracle of the ERMC Q_rad estimator -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
binding) never does.  The C source ``mcrt_oracle.c`` follows Section 2 and
Algorithm 1 of Silvestri & Pecnik (arXiv:1810.00188); this module compiles it
with gcc and marshals numpy arrays through ctypes.  Q_i, sigma_i and the parity
scale S_i are formed here from the oracle's per-cell FP64 sums (Eq. 8: the
estimate is the mean of the per-ray samples).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcrt_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "learn_oracle.c")]
_LIB = os.path.join(_HERE, "_build", "libmcrt_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            [os.path.getmtime(f) for f in _SRCS] + [os.path.getmtime(os.path.join(_HERE, "mcrt_oracle.h"))]):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-pthread", "-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("T", C.POINTER(C.c_double)), ("xh2o", C.POINTER(C.c_double)),
                ("eps_wall", C.c_double * 2), ("T_wall", C.c_double * 2),
                ("reflect", C.c_int), ("n_bands", C.c_int), ("n_g", C.c_int),
                ("w_g", C.POINTER(C.c_double)), ("T0", C.c_double), ("dT", C.c_double),
                ("nT", C.c_int), ("kappa", C.POINTER(C.c_double)),
                ("B", C.POINTER(C.c_double)), ("x_ref", C.c_double),
                ("yf", C.POINTER(C.c_double)), ("xz_walls", C.c_int), ("T_xz", C.c_double * 4)]


class Params(C.Structure):
    _fields_ = [("rays_per_cell", C.c_int), ("ray_offset", C.c_uint64), ("seed", C.c_uint64),
                ("snapshot", C.c_uint32), ("tol", C.c_double), ("max_steps", C.c_int),
                ("origin", C.c_int), ("use_box", C.c_int), ("box", C.c_int * 6),
                ("nthreads", C.c_int), ("cell_cn", C.POINTER(C.c_uint64)),
                ("cell_cg", C.POINTER(C.c_uint64)), ("cell_hemi", C.POINTER(C.c_uint32)),
                ("tally", C.POINTER(C.c_double)), ("tally_cost", C.POINTER(C.c_double)),
                ("mg_levels", C.c_int), ("mg_steps", C.c_int)]


class CellSums(C.Structure):
    _fields_ = [("sum_y", C.POINTER(C.c_double)), ("sum_y2", C.POINTER(C.c_double)),
                ("sum_abs", C.POINTER(C.c_double)), ("sum_wall", C.POINTER(C.c_double)),
                ("sum_wall2", C.POINTER(C.c_double)), ("steps", C.POINTER(C.c_uint64)),
                ("capped", C.POINTER(C.c_uint64))]


class RayIn(C.Structure):
    _fields_ = [("n", C.c_int), ("g", C.c_int), ("cell", C.c_int * 3), ("frac", C.c_double * 3),
                ("dir", C.c_double * 3), ("tol", C.c_double), ("max_steps", C.c_int),
                ("seed", C.c_uint64), ("ray", C.c_uint32), ("snapshot", C.c_uint32)]


class RayOut(C.Structure):
    _fields_ = [("X", C.c_double), ("abs_terms", C.c_double), ("X_wall", C.c_double),
                ("tau_end", C.c_double), ("steps", C.c_int64), ("capped", C.c_int),
                ("walls", C.c_int), ("path", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, up = C.POINTER(C.c_double), C.POINTER(C.c_uint64)
            L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
            L.orc_philox_batch.argtypes = [C.POINTER(C.c_uint32), C.c_int64,
                                           C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.orc_uniform.argtypes = [C.c_uint32]
            L.orc_uniform.restype = C.c_double
            L.orc_interp.argtypes = [dp, C.c_double, C.c_double, C.c_int, C.c_double]
            L.orc_interp.restype = C.c_double
            L.orc_quantize.argtypes = [dp, C.c_int, up]
            L.orc_plain_proposal.argtypes = [C.POINTER(Problem), up, up, dp]
            L.orc_trace_ray.argtypes = [C.POINTER(Problem), C.POINTER(RayIn), C.POINTER(RayOut)]
            L.orc_trace_ray_mg.argtypes = [C.POINTER(Problem), C.POINTER(RayIn), C.c_int, C.c_int,
                                           C.POINTER(RayOut)]
            L.orc_mg_max_levels.argtypes = [C.c_int, C.c_int, C.c_int]
            L.orc_solve.argtypes = [C.POINTER(Problem), C.POINTER(Params), C.POINTER(CellSums)]
            L.orc_exchange.argtypes = [C.POINTER(Problem), C.POINTER(Params), dp, dp, dp, dp]
            L.orc_solve_armc.argtypes = [C.POINTER(Problem), C.POINTER(Params), C.c_int, dp, dp, dp,
                                         C.POINTER(C.c_uint64)]
            L.orc_quadrature.argtypes = [C.POINTER(Problem), dp, dp, C.c_int, C.c_int, dp, dp,
                                         C.c_int, C.c_int, C.c_double, C.c_int,
                                         C.POINTER(C.c_int), C.c_int, C.c_int, dp]
            i64 = C.c_int64
            L.orc_features.argtypes = [C.POINTER(Problem), C.POINTER(C.c_int32), i64, C.c_double, dp]
            L.orc_mlp_nparams.argtypes = [C.c_int]
            L.orc_mlp_nparams.restype = i64
            L.orc_mlp_forward.argtypes = [dp, C.c_int, dp, dp, dp, i64, dp, C.c_int, C.c_double, dp]
            L.orc_mlp_loss_grad.argtypes = [dp, C.c_int, dp, dp, dp, dp, dp, C.c_double, dp, dp,
                                            C.c_int, i64, C.c_double, dp, dp]
            L.orc_adam.argtypes = [dp, dp, dp, dp, i64, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_int]
            L.orc_learned_counts.argtypes = [dp, C.c_int, C.c_int, C.c_double, up, up,
                                             C.POINTER(C.c_uint32)]
            L.orc_spectral_proposal.argtypes = [C.POINTER(Problem), C.c_int, C.c_double, C.c_double,
                                                dp, C.POINTER(C.c_int32), i64, dp]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Keep:
    """Holds the numpy arrays a ctypes Problem points into."""


def make_problem(grid, kd, T, x=None):
    keep = _Keep()
    keep.T = _f64(T).reshape(-1)
    keep.x = None if x is None else _f64(x).reshape(-1)
    keep.w = _f64(kd.w_g)
    keep.k = _f64(kd.kappa).reshape(-1)
    keep.B = _f64(kd.B).reshape(-1)
    assert keep.T.size == grid.ncells
    P = Problem()
    P.nx, P.ny, P.nz = grid.nx, grid.ny, grid.nz
    P.lx, P.ly, P.lz = grid.lx, grid.ly, grid.lz
    P.T = _dp(keep.T)
    P.xh2o = _dp(keep.x) if keep.x is not None else C.POINTER(C.c_double)()
    P.eps_wall[0], P.eps_wall[1] = grid.eps_wall
    P.T_wall[0], P.T_wall[1] = grid.T_wall
    P.reflect = grid.reflect
    P.n_bands, P.n_g = kd.n_bands, kd.n_g
    P.w_g = _dp(keep.w)
    P.T0, P.dT, P.nT = kd.T0, kd.dT, kd.nT
    P.kappa = _dp(keep.k)
    P.B = _dp(keep.B)
    P.x_ref = kd.x_ref
    yf = getattr(grid, "yf", None)
    keep.yf = None if yf is None else _f64(yf)
    if keep.yf is not None:
        assert keep.yf.size == grid.ny + 1
    P.yf = _dp(keep.yf) if keep.yf is not None else C.POINTER(C.c_double)()
    P.xz_walls = int(getattr(grid, "xz_walls", 0))
    for f, t in enumerate(getattr(grid, "T_xz", (0.0, 0.0, 0.0, 0.0))):
        P.T_xz[f] = float(t)
    P._keep = keep
    return P


def philox(ctr, key):
    """Philox4x32-10 of counters ctr [n,4] (uint32) under key [2] -> [n,4] uint32."""
    ctr = np.ascontiguousarray(np.atleast_2d(ctr), dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty_like(ctr)
    u32 = C.POINTER(C.c_uint32)
    lib().orc_philox_batch(ctr.ctypes.data_as(u32), ctr.shape[0], key.ctypes.data_as(u32),
                           out.ctypes.data_as(u32))
    return out


def uniform(w):
    return ((np.asarray(w, dtype=np.uint32) >> 9).astype(np.float64) + 0.5) * 2.0**-23


def interp(v, T0, dT, T):
    v = _f64(v)
    return lib().orc_interp(_dp(v), T0, dT, v.size, float(T))


def quantize(w):
    w = _f64(w)
    cum = np.zeros(w.size, dtype=np.uint64)
    rc = lib().orc_quantize(_dp(w), w.size, cum.ctypes.data_as(C.POINTER(C.c_uint64)))
    if rc != 0:
        raise ValueError("no positive weight")
    return cum


def plain_proposal(grid, kd, T, x=None):
    """Cumulative band counts [nb], g counts [nb, ng] and T_max of the plain proposal."""
    P = make_problem(grid, kd, T, x)
    cn = np.zeros(kd.n_bands, dtype=np.uint64)
    cg = np.zeros(kd.n_bands * kd.n_g, dtype=np.uint64)
    tm = C.c_double()
    up = C.POINTER(C.c_uint64)
    rc = lib().orc_plain_proposal(C.byref(P), cn.ctypes.data_as(up), cg.ctypes.data_as(up),
                                  C.byref(tm))
    if rc != 0:
        raise ValueError(f"orc_plain_proposal failed: {rc}")
    return cn, cg.reshape(kd.n_bands, kd.n_g), tm.value


def trace_ray(grid, kd, T, x, n, g, cell, frac, direction, tol=1e-4, max_steps=1 << 30,
              seed=0, ray=0, snapshot=0, mg_levels=1, mg_steps=5):
    """One ray's march (Algorithm 1); with mg_levels > 1 on overlaid coarsened
    grids (Section 4.3)."""
    P = make_problem(grid, kd, T, x)
    R = RayIn()
    R.n, R.g = n, g
    for a in range(3):
        R.cell[a] = int(cell[a])
        R.frac[a] = float(frac[a])
        R.dir[a] = float(direction[a])
    R.tol, R.max_steps, R.seed, R.ray, R.snapshot = tol, max_steps, seed, ray, snapshot
    O = RayOut()
    if mg_levels > 1:
        rc = lib().orc_trace_ray_mg(C.byref(P), C.byref(R), mg_levels, mg_steps, C.byref(O))
    else:
        rc = lib().orc_trace_ray(C.byref(P), C.byref(R), C.byref(O))
    if rc != 0:
        raise ValueError(f"bad ray ({rc})")
    return {f: getattr(O, f) for f, _ in RayOut._fields_}


def mg_max_levels(nx, ny, nz):
    """Number of overlaid grids the multigrid march can use on an nx x ny x nz grid."""
    return int(lib().orc_mg_max_levels(nx, ny, nz))


def default_threads():
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())


def _params(rays, seed, snapshot, ray_offset, tol, max_steps, origin, box, nthreads):
    S = Params()
    S.rays_per_cell, S.ray_offset, S.seed, S.snapshot = rays, ray_offset, seed, snapshot
    S.tol, S.max_steps, S.origin = tol, max_steps, origin
    S.use_box = 0 if box is None else 1
    if box is not None:
        for i in range(6):
            S.box[i] = int(box[i])
    S.nthreads = default_threads() if nthreads is None else nthreads
    return S


def solve(grid, kd, T, x=None, rays=128, seed=0, snapshot=0, ray_offset=0, tol=1e-4,
          max_steps=1 << 30, origin=0, box=None, nthreads=None, proposal=None, tally=False,
          mg_levels=1, mg_steps=5):
    """Per-cell ERMC estimate over the box (whole grid when box is None).

    Returns a dict of arrays shaped [bnz, bny, bnx]: q (Q_i, W/m^3), sigma
    (standard error of q), scale (S_i = mean of w sum|terms|), q_wall and
    sigma_wall (the wall-exchange part), steps and capped counts, and the raw
    sums.  ``proposal`` = (cell_cn [nc, nb], cell_cg [nc, nb, ng], cell_hemi
    [nc]) overrides the plain T_max proposal per emitting cell.  mg_levels > 1
    marches rays on that many overlaid grids, mg_steps segments per grid
    (Section 4.3).  With
    ``tally`` the result also holds "tally" [bnz, bny, bnx, nb * ng, 2]: per
    spectral point and hemisphere (0 upward), (1/N) sum of Y^2 p(n,g) p(h) over
    the rays that drew them, and "tally_cost" (same shape): (1/N) sum of
    steps / (p(n,g) p(h)).
    """
    P = make_problem(grid, kd, T, x)
    S = _params(rays, seed, snapshot, ray_offset, tol, max_steps, origin, box, nthreads)
    S.mg_levels, S.mg_steps = mg_levels, mg_steps
    b = box if box is not None else (0, grid.nx, 0, grid.ny, 0, grid.nz)
    shape = (max(b[5] - b[4], 0), max(b[3] - b[2], 0), max(b[1] - b[0], 0))
    nc = int(np.prod(shape))
    keep = []
    if proposal is not None:
        cn, cg, hemi = proposal
        cn = np.ascontiguousarray(cn, dtype=np.uint64).reshape(nc, kd.n_bands)
        cg = np.ascontiguousarray(cg, dtype=np.uint64).reshape(nc, kd.n_bands * kd.n_g)
        hemi = np.ascontiguousarray(hemi, dtype=np.uint32).reshape(nc)
        keep += [cn, cg, hemi]
        S.cell_cn = cn.ctypes.data_as(C.POINTER(C.c_uint64))
        S.cell_cg = cg.ctypes.data_as(C.POINTER(C.c_uint64))
        S.cell_hemi = hemi.ctypes.data_as(C.POINTER(C.c_uint32))
    if tally:
        tl = np.zeros((nc, kd.n_bands * kd.n_g, 2))
        tc = np.zeros((nc, kd.n_bands * kd.n_g, 2))
        S.tally = _dp(tl)
        S.tally_cost = _dp(tc)
    out = {k: np.zeros(nc) for k in ("sum_y", "sum_y2", "sum_abs", "sum_wall", "sum_wall2")}
    out["steps"] = np.zeros(nc, dtype=np.uint64)
    out["capped"] = np.zeros(nc, dtype=np.uint64)
    Cs = CellSums()
    for k in ("sum_y", "sum_y2", "sum_abs", "sum_wall", "sum_wall2"):
        setattr(Cs, k, _dp(out[k]))
    Cs.steps = out["steps"].ctypes.data_as(C.POINTER(C.c_uint64))
    Cs.capped = out["capped"].ctypes.data_as(C.POINTER(C.c_uint64))
    rc = lib().orc_solve(C.byref(P), C.byref(S), C.byref(Cs))
    if rc != 0:
        raise ValueError(f"orc_solve failed: {rc}")
    N = float(rays)
    res = {k: v.reshape(shape) for k, v in out.items()}
    if tally:
        res["tally"] = tl.reshape(shape + (kd.n_bands * kd.n_g, 2))
        res["tally_cost"] = tc.reshape(shape + (kd.n_bands * kd.n_g, 2))
    res["q"] = res["sum_y"] / N
    res["scale"] = res["sum_abs"] / N
    res["q_wall"] = res["sum_wall"] / N
    if rays > 1:
        res["sigma"] = np.sqrt(np.maximum(res["sum_y2"] / N - res["q"] ** 2, 0.0) / (N - 1.0))
        res["sigma_wall"] = np.sqrt(np.maximum(res["sum_wall2"] / N - res["q_wall"] ** 2, 0.0)
                                    / (N - 1.0))
    else:
        res["sigma"] = np.zeros(shape)
        res["sigma_wall"] = np.zeros(shape)
    return res


def solve_armc(grid, kd, T, x=None, rays=128, seed=0, snapshot=0, ray_offset=0, tol=1e-4,
               max_steps=1 << 30, origin=0, box=None, nthreads=None, proposal=None, batches=16,
               hybrid=False):
    """Absorption-based reciprocal estimate (the paper's ARMC, Section 2: Eq. FM with
    the reciprocity relation): every cell of the grid emits `rays` rays; cell i's
    exchange with the other medium cells comes from the rays of those cells
    absorbed in i, its exchange with the walls from its own rays.  Returns arrays
    shaped [bnz, bny, bnx] over the box: q, sigma (batch means over K = min(batches,
    rays) batches of ray indices r mod K), scale (mean over rays of the absolute
    deposits), and the per-batch estimates q_batches [K, ...].  ``proposal`` =
    (cell_cn [nc, nb], cell_cg [nc, nb * ng], cell_hemi [nc]) over the WHOLE grid.
    With ``hybrid`` the result also holds the combination of the two estimates
    cell by cell, lam_i Q_E,i + (1 - lam_i) Q_A,i with lam_i = (T_i - T_min) /
    (T_max - T_min) over the medium (the emission-based estimate where the gas
    is hot, the absorption-based one where it is cold): "q_hybrid",
    "sigma_hybrid" (batch means of the combined batch estimates), and the
    emission-based "q_ermc" of the same draws."""
    P = make_problem(grid, kd, T, x)
    S = _params(rays, seed, snapshot, ray_offset, tol, max_steps, origin, None, nthreads)
    S.mg_levels, S.mg_steps = 1, 5
    nc = grid.ncells
    keep = []
    if proposal is not None:
        cn, cg, hemi = proposal
        cn = np.ascontiguousarray(cn, dtype=np.uint64).reshape(nc, kd.n_bands)
        cg = np.ascontiguousarray(cg, dtype=np.uint64).reshape(nc, kd.n_bands * kd.n_g)
        hemi = np.ascontiguousarray(hemi, dtype=np.uint32).reshape(nc)
        keep += [cn, cg, hemi]
        S.cell_cn = cn.ctypes.data_as(C.POINTER(C.c_uint64))
        S.cell_cg = cg.ctypes.data_as(C.POINTER(C.c_uint64))
        S.cell_hemi = hemi.ctypes.data_as(C.POINTER(C.c_uint32))
    K = max(1, min(int(batches), int(rays)))
    acc = np.zeros((K, nc))
    absacc = np.zeros(nc)
    accE = np.zeros((K, nc)) if hybrid else None
    steps = np.zeros(nc, dtype=np.uint64)
    rc = lib().orc_solve_armc(C.byref(P), C.byref(S), K, _dp(acc), _dp(absacc),
                              _dp(accE) if hybrid else C.POINTER(C.c_double)(),
                              steps.ctypes.data_as(C.POINTER(C.c_uint64)))
    if rc != 0:
        raise ValueError(f"orc_solve_armc failed: {rc}")
    b = box if box is not None else (0, grid.nx, 0, grid.ny, 0, grid.nz)
    shape3 = (grid.nz, grid.ny, grid.nx)
    crop = (slice(b[4], b[5]), slice(b[2], b[3]), slice(b[0], b[1]))
    nk = np.array([len(range(k, rays, K)) for k in range(K)], dtype=np.float64)
    qb = acc / nk[:, None]
    res = {"q": (acc.sum(0) / rays).reshape(shape3)[crop],
           "scale": (absacc / rays).reshape(shape3)[crop],
           "steps": steps.reshape(shape3)[crop],
           "q_batches": qb.reshape((K,) + shape3)[(slice(None),) + crop]}
    if K > 1:
        var = qb.var(axis=0, ddof=1) / K
        res["sigma"] = np.sqrt(var).reshape(shape3)[crop]
    else:
        res["sigma"] = np.zeros(shape3)[crop]
    if hybrid:
        Tf = np.asarray(T, dtype=np.float64).reshape(-1)
        lam = np.clip((Tf - Tf.min()) / max(Tf.max() - Tf.min(), 1e-300), 0.0, 1.0)
        qe = accE / nk[:, None]
        qh = lam[None, :] * qe + (1.0 - lam[None, :]) * qb
        res["q_ermc"] = (accE.sum(0) / rays).reshape(shape3)[crop]
        res["q_hybrid"] = (lam * accE.sum(0) / rays + (1.0 - lam) * acc.sum(0) / rays).reshape(shape3)[crop]
        res["sigma_hybrid"] = (np.sqrt(qh.var(axis=0, ddof=1) / K) if K > 1 else np.zeros(nc)).reshape(shape3)[crop]
    return res


def exchange(grid, kd, T, x=None, rays=128, seed=0, tol=1e-9, max_steps=1 << 30, origin=0):
    """Per-pair exchange estimates G[i, j] = E[w kappa_i tau alpha_j] and their
    standard errors, plus the wall exchange Gw[i, 2]."""
    P = make_problem(grid, kd, T, x)
    S = _params(rays, seed, 0, 0, tol, max_steps, origin, None, 1)
    nc = grid.ncells
    G, G2 = np.zeros((nc, nc)), np.zeros((nc, nc))
    Gw, Gw2 = np.zeros((nc, 2)), np.zeros((nc, 2))
    rc = lib().orc_exchange(C.byref(P), C.byref(S), _dp(G), _dp(G2), _dp(Gw), _dp(Gw2))
    if rc != 0:
        raise ValueError(f"orc_exchange failed: {rc}")
    N = float(rays)
    mean, meanw = G / N, Gw / N
    se = np.sqrt(np.maximum(G2 / N - mean**2, 0.0) / (N - 1.0))
    sew = np.sqrt(np.maximum(Gw2 / N - meanw**2, 0.0) / (N - 1.0))
    return mean, se, meanw, sew


def quadrature(grid, kd, T, x=None, cells=None, nmu_panels=32, nmu_per_panel=4, nphi=128,
               nv=3, origin=0, tol=1e-12, max_steps=1 << 30, nthreads=None, origins=None):
    """Deterministic quadrature of Q_i (same estimand, no random draws): composite
    Gauss-Legendre in mu, midpoint in phi, and over the cell a Gauss-Legendre
    tensor rule with nv points per axis, the mean over an explicit list of
    origin fractions ``origins`` [m, 3] (origin 0), or the cell centre (origin 1)."""
    P = make_problem(grid, kd, T, x)
    xg, wg = np.polynomial.legendre.leggauss(nmu_per_panel)
    edges = np.linspace(-1.0, 1.0, nmu_panels + 1)
    mu = np.concatenate([0.5 * (b - a) * xg + 0.5 * (a + b) for a, b in zip(edges[:-1], edges[1:])])
    mw = np.concatenate([0.5 * (b - a) * wg for a, b in zip(edges[:-1], edges[1:])])
    if origins is not None:
        vn = np.ascontiguousarray(origins, dtype=np.float64).reshape(-1)
        vw = np.full(vn.size // 3, 3.0 / vn.size)
        nv = -(vn.size // 3)
    else:
        xv, wv = np.polynomial.legendre.leggauss(nv)
        vn, vw = 0.5 * (xv + 1.0), 0.5 * wv
    if cells is None:
        cells = np.arange(grid.ncells)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    q = np.zeros(cells.size)
    rc = lib().orc_quadrature(C.byref(P), _dp(_f64(mu)), _dp(_f64(mw)), mu.size, nphi,
                              _dp(_f64(vn)), _dp(_f64(vw)), int(nv), origin, tol, max_steps,
                              cells.ctypes.data_as(C.POINTER(C.c_int)), cells.size,
                              default_threads() if nthreads is None else nthreads, _dp(q))
    if rc != 0:
        raise ValueError(f"orc_quadrature failed: {rc}")
    return q


# ---- learned proposal (see learn_oracle.c) ----------------------------------

NFEAT, HIDDEN = 12, 64


def features(grid, kd, T, x=None, cells=None, T_max=None):
    """The 12 local features [n, 12] of the listed cells (whole grid if None);
    T_max defaults to the plain proposal's."""
    P = make_problem(grid, kd, T, x)
    if T_max is None:
        T_max = plain_proposal(grid, kd, T, x)[2]
    cells = np.arange(grid.ncells, dtype=np.int32) if cells is None else np.asarray(cells)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    out = np.zeros((cells.size, NFEAT))
    rc = lib().orc_features(C.byref(P), cells.ctypes.data_as(C.POINTER(C.c_int32)), cells.size,
                            float(T_max), _dp(out))
    if rc != 0:
        raise ValueError("bad cell index")
    return out


def mlp_nparams(K):
    return int(lib().orc_mlp_nparams(int(K)))


def mlp_forward(theta, K, fmean, finv, feat, p0, mix=0.1):
    """Mixed proposal probabilities [n, K + 2] (spectral points, then up, down).
    p0 is [K] (shared) or [n, K]."""
    theta, fmean, finv = _f64(theta), _f64(fmean), _f64(finv)
    feat = _f64(feat).reshape(-1, NFEAT)
    p0 = _f64(p0)
    stride = 0 if p0.ndim == 1 else K
    q = np.zeros((feat.shape[0], K + 2))
    rc = lib().orc_mlp_forward(_dp(theta), K, _dp(fmean), _dp(finv), _dp(feat), feat.shape[0],
                               _dp(p0), stride, float(mix), _dp(q))
    if rc != 0:
        raise ValueError("orc_mlp_forward failed")
    return q


def mlp_loss_grad(theta, K, fmean, finv, feat, m, p0, mix=0.1, cost=None, c0=0.0, wgt=None,
                  mode=0):
    """(loss, gradient [nparams]); m, cost [n, K, 2] (cost None: second moment
    only), p0 [n, K].  mode 0: mean over samples of the per-cell work ratio;
    mode 1: the batch time ratio with sample weights wgt [n] (None: 1)."""
    theta, fmean, finv = _f64(theta), _f64(fmean), _f64(finv)
    feat = _f64(feat).reshape(-1, NFEAT)
    n = feat.shape[0]
    m = _f64(m).reshape(n, K, 2)
    p0 = _f64(p0).reshape(n, K)
    cst = None if cost is None else _f64(cost).reshape(n, K, 2)
    w = None if wgt is None else _f64(wgt).reshape(n)
    grad = np.zeros(mlp_nparams(K))
    loss = C.c_double()
    null = C.POINTER(C.c_double)()
    rc = lib().orc_mlp_loss_grad(_dp(theta), K, _dp(fmean), _dp(finv), _dp(feat), _dp(m),
                                 _dp(cst) if cst is not None else null, float(c0), _dp(p0),
                                 _dp(w) if w is not None else null, int(mode), n, float(mix),
                                 C.byref(loss), _dp(grad))
    if rc != 0:
        raise ValueError("orc_mlp_loss_grad failed")
    return loss.value, grad


def adam(theta, grad, m1, m2, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place on FP64 copies; returns (theta, m1, m2)."""
    theta, grad, m1, m2 = (np.array(a, dtype=np.float64) for a in (theta, grad, m1, m2))
    lib().orc_adam(_dp(theta), _dp(grad), _dp(m1), _dp(m2), theta.size, lr, beta1, beta2, eps, int(t))
    return theta, m1, m2


def learned_counts(q, nb, ng, q_up):
    """Integer proposal (cn [nb], cg [nb, ng], hemi) of one cell from its
    probabilities q [nb * ng] and q_up (counts decided in binary32, the rule of
    the device's per-cell proposals)."""
    q = _f64(q).reshape(-1)
    cn = np.zeros(nb, dtype=np.uint64)
    cg = np.zeros(nb * ng, dtype=np.uint64)
    hemi = C.c_uint32()
    up = C.POINTER(C.c_uint64)
    rc = lib().orc_learned_counts(_dp(q), nb, ng, float(q_up), cn.ctypes.data_as(up),
                                  cg.ctypes.data_as(up), C.byref(hemi))
    if rc != 0:
        raise ValueError("orc_learned_counts failed")
    return cn, cg.reshape(nb, ng), hemi.value


def spectral_proposal(grid, kd, T, x=None, mode=0, cells=None):
    """Per-cell spectral probabilities [n, K] at the cells' own temperatures:
    mode 0 the local emission spectrum, 1 mixed with the T_max proposal by
    lam = (T_i - T_min) / (T_max - T_min)."""
    cn, cg, T_max = plain_proposal(grid, kd, T, x)
    nb, ng = kd.n_bands, kd.n_g
    c = np.diff(np.concatenate([[0], cn.astype(np.float64)])) * 2.0**-32
    g = np.diff(np.concatenate([np.zeros((nb, 1)), cg.astype(np.float64)], axis=1), axis=1) * 2.0**-32
    p0 = np.ascontiguousarray((c[:, None] * g).reshape(-1))
    P = make_problem(grid, kd, T, x)
    cells = np.arange(grid.ncells, dtype=np.int32) if cells is None else np.asarray(cells)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    q = np.zeros((cells.size, nb * ng))
    Tf = np.asarray(T, dtype=np.float64).reshape(-1)
    lib().orc_spectral_proposal(C.byref(P), int(mode), float(Tf.min()), float(T_max), _dp(p0),
                                cells.ctypes.data_as(C.POINTER(C.c_int32)), cells.size, _dp(q))
    return q

