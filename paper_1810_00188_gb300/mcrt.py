"""Thin ctypes binding of the C ABI in include/mcrt.h (argument marshalling only).

The functions keep the C names (``mcrt_create``, ``mcrt_set_kdist``,
``mcrt_set_fields``, ``mcrt_set_cell_proposal``, ``mcrt_solve_qrad``,
``mcrt_get_stats``, ``mcrt_destroy``); every step of a solve runs in the CUDA
library.  ``Solver`` wraps a context for numpy / torch callers.  Loading fails
loudly when the compiled library is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

MCRT_OK, MCRT_E_ARG, MCRT_E_STATE, MCRT_E_CUDA, MCRT_E_OOM, MCRT_E_RANGE, MCRT_E_TIMEOUT, \
    MCRT_E_UNSUPPORTED = range(8)
MCRT_MEM_HOST, MCRT_MEM_DEVICE = 0, 1
MCRT_FP32, MCRT_FP64 = 0, 1
MCRT_ORIGIN_UNIFORM, MCRT_ORIGIN_CENTER = 0, 1
MCRT_PROPOSAL_PLANCK_TMAX, MCRT_PROPOSAL_CELL = 0, 1
MCRT_EST_ERMC, MCRT_EST_ARMC, MCRT_EST_HYBRID = 0, 1, 2
MCRT_REFLECT_DIFFUSE, MCRT_REFLECT_SPECULAR = 0, 1


class McrtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mcrt status {status} ({STATUS_NAMES.get(status, '?')}): {msg}")
        self.status = status


STATUS_NAMES = {0: "ok", 1: "E_ARG", 2: "E_STATE", 3: "E_CUDA", 4: "E_OOM", 5: "E_RANGE",
                6: "E_TIMEOUT", 7: "E_UNSUPPORTED"}


class mcrt_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("lx", C.c_double),
                ("ly", C.c_double), ("lz", C.c_double), ("eps_wall", C.c_double * 2),
                ("T_wall", C.c_double * 2), ("reflect", C.c_int), ("device", C.c_int),
                ("yf", C.POINTER(C.c_double)), ("xz_walls", C.c_int), ("T_xz", C.c_double * 4)]


class mcrt_kdist_desc(C.Structure):
    _fields_ = [("n_bands", C.c_int), ("n_g", C.c_int), ("w_g", C.POINTER(C.c_double)),
                ("T0", C.c_double), ("dT", C.c_double), ("nT", C.c_int),
                ("kappa", C.POINTER(C.c_double)), ("B", C.POINTER(C.c_double)),
                ("x_ref", C.c_double), ("nu_c", C.POINTER(C.c_double)), ("dnu", C.POINTER(C.c_double))]


class mcrt_solve_params(C.Structure):
    _fields_ = [("rays_per_cell", C.c_int), ("max_steps", C.c_int), ("tol", C.c_double),
                ("seed", C.c_uint64), ("ray_offset", C.c_uint64), ("snapshot", C.c_uint32),
                ("precision", C.c_int), ("origin", C.c_int), ("proposal", C.c_int),
                ("use_box", C.c_int), ("box", C.c_int * 6), ("steps_out", C.c_void_p),
                ("mg_levels", C.c_int), ("mg_steps", C.c_int), ("estimator", C.c_int)]


class mcrt_tuning(C.Structure):
    _fields_ = [("min_blocks_per_sm", C.c_int), ("steps_per_round", C.c_int),
                ("scratch_mib", C.c_int), ("long_ray_steps", C.c_int), ("long_ray_flight", C.c_int),
                ("tally_binary32", C.c_int), ("tally_plain_loads", C.c_int), ("claim_rays", C.c_int),
                ("batch_per_snapshot", C.c_int)]


class mcrt_batch_item(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("q_out", C.c_void_p), ("sigma_out", C.c_void_p),
                ("snapshot", C.c_uint32)]


class mcrt_solve_stats(C.Structure):
    _fields_ = [("steps", C.c_uint64), ("rays", C.c_uint64), ("capped", C.c_uint64),
                ("wall_hits", C.c_uint64), ("max_ray_steps", C.c_uint64), ("T_max", C.c_double),
                ("kernel_ms", C.c_float),
                ("launches", C.c_int), ("long_rays", C.c_uint64), ("long_overflow", C.c_uint64),
                ("trace_ms", C.c_float), ("long_ms", C.c_float), ("reduce_ms", C.c_float)]


_lib = None
_lock = threading.Lock()
EXPORTS = ("mcrt_create", "mcrt_set_kdist", "mcrt_set_fields", "mcrt_set_cell_proposal",
           "mcrt_solve_qrad", "mcrt_get_stats", "mcrt_destroy", "mcrt_status_string",
           "mcrt_last_error", "mcrt_set_tuning", "mcrt_get_tuning", "mcrt_solve_qrad_noalloc",
           "mcrt_batch_create", "mcrt_batch_run", "mcrt_batch_get_stats", "mcrt_batch_last_error",
           "mcrt_batch_destroy", "mcrt_mlp_nparams", "mcrt_mlp_create", "mcrt_mlp_set_params",
           "mcrt_mlp_get_params", "mcrt_mlp_forward", "mcrt_mlp_loss_grad", "mcrt_mlp_adam_step",
           "mcrt_mlp_last_loss", "mcrt_mlp_last_error", "mcrt_mlp_destroy", "mcrt_cell_features",
           "mcrt_tally_moments", "mcrt_get_plain_probs", "mcrt_set_cell_proposal_probs",
           "mcrt_get_cell_proposal", "mcrt_set_learned_proposal", "mcrt_multigrid_levels",
           "mcrt_set_spectral_proposal", "mcrt_probe_ex2", "mcrt_probe_gather")
_NOT_INT = ("mcrt_status_string", "mcrt_last_error", "mcrt_batch_last_error", "mcrt_mlp_last_error",
            "mcrt_mlp_nparams")
MCRT_NFEAT, MCRT_NHIDDEN = 12, 64
MCRT_LOSS_CELL, MCRT_LOSS_BATCH = 0, 1


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libmcrt.so (building it in-tree with nvcc if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and _build.needs_build():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run paper_1810_00188_gb300.build)")
        L = C.CDLL(path)
        vp = C.c_void_p
        L.mcrt_create.argtypes = [C.POINTER(mcrt_grid_desc), C.POINTER(vp)]
        L.mcrt_set_kdist.argtypes = [vp, C.POINTER(mcrt_kdist_desc)]
        L.mcrt_set_fields.argtypes = [vp, vp, vp, C.c_int, C.c_int, vp]
        L.mcrt_set_cell_proposal.argtypes = [vp, vp, vp, vp, C.c_int, vp]
        L.mcrt_solve_qrad.argtypes = [vp, C.POINTER(mcrt_solve_params), vp, vp, C.c_int, vp]
        L.mcrt_solve_qrad_noalloc.argtypes = [vp, C.POINTER(mcrt_solve_params), vp, vp, vp]
        L.mcrt_get_stats.argtypes = [vp, C.POINTER(mcrt_solve_stats)]
        L.mcrt_set_tuning.argtypes = [vp, C.POINTER(mcrt_tuning)]
        L.mcrt_get_tuning.argtypes = [vp, C.POINTER(mcrt_tuning)]
        L.mcrt_destroy.argtypes = [vp]
        L.mcrt_status_string.argtypes = [C.c_int]
        L.mcrt_status_string.restype = C.c_char_p
        L.mcrt_last_error.argtypes = [vp]
        L.mcrt_last_error.restype = C.c_char_p
        L.mcrt_batch_create.argtypes = [C.POINTER(mcrt_batch_item), C.c_int,
                                        C.POINTER(mcrt_solve_params), C.POINTER(C.c_double),
                                        C.c_int, C.POINTER(vp)]
        L.mcrt_batch_run.argtypes = [vp, C.c_uint64, vp]
        L.mcrt_batch_get_stats.argtypes = [vp, C.POINTER(mcrt_solve_stats)]
        L.mcrt_batch_last_error.argtypes = [vp]
        L.mcrt_batch_last_error.restype = C.c_char_p
        L.mcrt_batch_destroy.argtypes = [vp]
        i64, f32 = C.c_int64, C.c_float
        L.mcrt_mlp_nparams.argtypes = [C.c_int]
        L.mcrt_mlp_nparams.restype = i64
        L.mcrt_mlp_create.argtypes = [C.c_int, C.c_int, C.POINTER(vp)]
        L.mcrt_mlp_set_params.argtypes = [vp, vp, vp, vp]
        L.mcrt_mlp_get_params.argtypes = [vp, vp, vp]
        L.mcrt_mlp_forward.argtypes = [vp, vp, i64, vp, C.c_int, f32, vp, vp]
        L.mcrt_mlp_loss_grad.argtypes = [vp, vp, vp, vp, f32, vp, C.c_int, vp, C.c_int, i64, vp, i64,
                                         f32, vp, vp]
        L.mcrt_mlp_adam_step.argtypes = [vp, vp, f32, f32, f32, f32, vp]
        L.mcrt_mlp_last_loss.argtypes = [vp, C.POINTER(C.c_double)]
        L.mcrt_mlp_last_error.argtypes = [vp]
        L.mcrt_mlp_last_error.restype = C.c_char_p
        L.mcrt_mlp_destroy.argtypes = [vp]
        L.mcrt_cell_features.argtypes = [vp, vp, i64, vp, vp]
        L.mcrt_tally_moments.argtypes = [vp, C.POINTER(mcrt_solve_params), vp, i64, vp, vp, vp, vp, vp]
        L.mcrt_get_plain_probs.argtypes = [vp, vp]
        L.mcrt_set_cell_proposal_probs.argtypes = [vp, vp, vp]
        L.mcrt_get_cell_proposal.argtypes = [vp, vp, vp, vp]
        L.mcrt_set_learned_proposal.argtypes = [vp, vp, f32, vp]
        L.mcrt_multigrid_levels.argtypes = [C.c_int, C.c_int, C.c_int]
        L.mcrt_set_spectral_proposal.argtypes = [vp, C.c_int, vp]
        L.mcrt_probe_ex2.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.mcrt_probe_gather.argtypes = [C.c_int, C.c_uint64, C.POINTER(C.c_double)]
        for f in EXPORTS:
            if f not in _NOT_INT:
                getattr(L, f).restype = C.c_int
        _lib = L
        return _lib


def _check(rc, ctx=None):
    if rc != MCRT_OK:
        msg = load().mcrt_last_error(ctx).decode() if ctx else ""
        raise McrtError(rc, msg)


# --- the C entry points, same names ---------------------------------------------

def mcrt_multigrid_levels(nx: int, ny: int, nz: int) -> int:
    return int(load().mcrt_multigrid_levels(nx, ny, nz))


def mcrt_probe_ex2(device: int = 0):
    """(base-2 exponentials per second, mean SM clock in MHz) of the GPU."""
    r, mhz = C.c_double(), C.c_double()
    _check(load().mcrt_probe_ex2(int(device), C.byref(r), C.byref(mhz)))
    return r.value, mhz.value


def mcrt_probe_gather(device: int, nbytes: int) -> float:
    """Random 8-byte loads per second from a buffer of nbytes (a power of two)."""
    r = C.c_double()
    _check(load().mcrt_probe_gather(int(device), int(nbytes), C.byref(r)))
    return r.value


def mcrt_create(grid: mcrt_grid_desc) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().mcrt_create(C.byref(grid), C.byref(h)))
    return h


def mcrt_set_kdist(ctx, kd: mcrt_kdist_desc):
    _check(load().mcrt_set_kdist(ctx, C.byref(kd)), ctx)


def mcrt_set_fields(ctx, T_ptr, x_ptr, dtype_is_fp64: int, mem: int, stream: int = 0):
    _check(load().mcrt_set_fields(ctx, T_ptr, x_ptr, dtype_is_fp64, mem, stream), ctx)


def mcrt_set_cell_proposal(ctx, cn_ptr, cg_ptr, hemi_ptr, mem: int, stream: int = 0):
    _check(load().mcrt_set_cell_proposal(ctx, cn_ptr, cg_ptr, hemi_ptr, mem, stream), ctx)


def mcrt_solve_qrad(ctx, params: mcrt_solve_params, q_ptr, sigma_ptr, mem: int, stream: int = 0):
    _check(load().mcrt_solve_qrad(ctx, C.byref(params), q_ptr, sigma_ptr, mem, stream), ctx)


def mcrt_solve_qrad_noalloc(ctx, params: mcrt_solve_params, q_ptr, sigma_ptr, stream: int = 0):
    """The allocation-free solve: FP32, device outputs, scratch in a static 64 MiB
    device array (see include/mcrt.h)."""
    _check(load().mcrt_solve_qrad_noalloc(ctx, C.byref(params), q_ptr, sigma_ptr, stream), ctx)


def mcrt_batch_create(items, params: mcrt_solve_params, weights=None, streams: int = 2):
    """items: list of (ctx, q_ptr, sigma_ptr or None, snapshot)."""
    arr = (mcrt_batch_item * len(items))()
    for k, (ctx, q, s, snap) in enumerate(items):
        arr[k].ctx = ctx.value if hasattr(ctx, "value") else ctx
        arr[k].q_out = q.value if hasattr(q, "value") else q
        arr[k].sigma_out = None if s is None else (s.value if hasattr(s, "value") else s)
        arr[k].snapshot = snap
    w = None
    if weights is not None:
        w = (C.c_double * len(items))(*[float(v) for v in weights])
    h = C.c_void_p()
    rc = load().mcrt_batch_create(arr, len(items), C.byref(params), w, streams, C.byref(h))
    if rc != MCRT_OK:
        raise McrtError(rc, load().mcrt_last_error(arr[0].ctx).decode() if len(items) else "")
    return h


def mcrt_batch_run(batch, ray_offset: int = 0, stream: int = 0):
    rc = load().mcrt_batch_run(batch, ray_offset, stream)
    if rc != MCRT_OK:
        raise McrtError(rc, load().mcrt_batch_last_error(batch).decode())


def mcrt_batch_get_stats(batch) -> dict:
    st = mcrt_solve_stats()
    rc = load().mcrt_batch_get_stats(batch, C.byref(st))
    if rc != MCRT_OK:
        raise McrtError(rc, load().mcrt_batch_last_error(batch).decode())
    return {f: getattr(st, f) for f, _ in mcrt_solve_stats._fields_}


def mcrt_batch_destroy(batch):
    if batch:
        load().mcrt_batch_destroy(batch)


def mcrt_get_stats(ctx) -> dict:
    st = mcrt_solve_stats()
    _check(load().mcrt_get_stats(ctx, C.byref(st)), ctx)
    return {f: getattr(st, f) for f, _ in mcrt_solve_stats._fields_}


def mcrt_set_tuning(ctx, min_blocks_per_sm: int = 0, steps_per_round: int = 0,
                    scratch_mib: int = 0, long_ray_steps: int = 0, long_ray_flight: int = 0,
                    tally_binary32: int = 0, batch_per_snapshot: int = 0, claim_rays: int = 0,
                    tally_plain_loads: int = 0):
    t = mcrt_tuning()
    t.tally_binary32 = tally_binary32
    t.tally_plain_loads = tally_plain_loads
    t.claim_rays = claim_rays
    t.batch_per_snapshot = batch_per_snapshot
    t.min_blocks_per_sm = min_blocks_per_sm
    t.steps_per_round = steps_per_round
    t.scratch_mib = scratch_mib
    t.long_ray_steps = long_ray_steps
    t.long_ray_flight = long_ray_flight
    _check(load().mcrt_set_tuning(ctx, C.byref(t)), ctx)


def mcrt_get_tuning(ctx) -> dict:
    t = mcrt_tuning()
    _check(load().mcrt_get_tuning(ctx, C.byref(t)), ctx)
    return {f: getattr(t, f) for f, _ in mcrt_tuning._fields_}


def mcrt_destroy(ctx):
    if ctx:
        load().mcrt_destroy(ctx)


def mcrt_status_string(status: int) -> str:
    return load().mcrt_status_string(status).decode()


# --- convenience wrapper ----------------------------------------------------------

# --- learned proposal ------------------------------------------------------------

def _mcheck(rc, m):
    if rc != MCRT_OK:
        raise McrtError(rc, load().mcrt_mlp_last_error(m).decode() if m else "")


def mcrt_mlp_nparams(K: int) -> int:
    return int(load().mcrt_mlp_nparams(K))


def mcrt_mlp_create(device: int, K: int):
    h = C.c_void_p()
    _check(load().mcrt_mlp_create(device, K, C.byref(h)))
    return h


def mcrt_mlp_set_params(m, theta, feat_mean, feat_inv_std):
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    fm = np.ascontiguousarray(feat_mean, dtype=np.float32)
    fi = np.ascontiguousarray(feat_inv_std, dtype=np.float32)
    _mcheck(load().mcrt_mlp_set_params(m, _ptr(theta), _ptr(fm), _ptr(fi)), m)


def mcrt_mlp_get_params(m, K: int, used: bool = False):
    n = mcrt_mlp_nparams(K)
    th = np.zeros(n, dtype=np.float32)
    tu = np.zeros(n, dtype=np.float32) if used else None
    _mcheck(load().mcrt_mlp_get_params(m, _ptr(th), _ptr(tu)), m)
    return (th, tu) if used else th


def mcrt_mlp_forward(m, feat_ptr, n: int, p0_ptr, p0_stride: int, mix: float, q_ptr, stream=0):
    _mcheck(load().mcrt_mlp_forward(m, feat_ptr, n, p0_ptr, p0_stride, mix, q_ptr, stream), m)


def mcrt_mlp_loss_grad(m, feat_ptr, mom_ptr, cost_ptr, c0: float, p0_ptr, p0_stride: int, wgt_ptr,
                       mode: int, n_data: int, idx_ptr, n: int, mix: float, grad_ptr=None, stream=0):
    _mcheck(load().mcrt_mlp_loss_grad(m, feat_ptr, mom_ptr, cost_ptr, c0, p0_ptr, p0_stride, wgt_ptr,
                                      mode, n_data, idx_ptr, n, mix, grad_ptr, stream), m)


def mcrt_mlp_adam_step(m, grad_ptr=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=0):
    _mcheck(load().mcrt_mlp_adam_step(m, grad_ptr, lr, beta1, beta2, eps, stream), m)


def mcrt_mlp_last_loss(m) -> float:
    v = C.c_double()
    _mcheck(load().mcrt_mlp_last_loss(m, C.byref(v)), m)
    return v.value


def mcrt_mlp_destroy(m):
    load().mcrt_mlp_destroy(m)


def mcrt_cell_features(ctx, cells_ptr, n: int, out_ptr, stream=0):
    _check(load().mcrt_cell_features(ctx, cells_ptr, n, out_ptr, stream), ctx)


def mcrt_tally_moments(ctx, params, cells_ptr, n: int, mom_ptr, cost_ptr, q_ptr=None,
                       sigma_ptr=None, stream=0):
    _check(load().mcrt_tally_moments(ctx, C.byref(params), cells_ptr, n, mom_ptr, cost_ptr, q_ptr,
                                     sigma_ptr, stream), ctx)


def mcrt_get_plain_probs(ctx, K: int):
    p0 = np.zeros(K, dtype=np.float32)
    _check(load().mcrt_get_plain_probs(ctx, _ptr(p0)), ctx)
    return p0


def mcrt_set_cell_proposal_probs(ctx, q_ptr, stream=0):
    _check(load().mcrt_set_cell_proposal_probs(ctx, q_ptr, stream), ctx)


def mcrt_get_cell_proposal(ctx, ncells: int, nb: int, ng: int):
    cn = np.zeros((ncells, nb), dtype=np.uint64)
    cg = np.zeros((ncells, nb, ng), dtype=np.uint64)
    hemi = np.zeros(ncells, dtype=np.uint32)
    _check(load().mcrt_get_cell_proposal(ctx, _ptr(cn), _ptr(cg), _ptr(hemi)), ctx)
    return cn, cg, hemi


MCRT_SPECTRAL_LOCAL, MCRT_SPECTRAL_HYBRID = 0, 1


def mcrt_set_spectral_proposal(ctx, mode: int, stream=0):
    _check(load().mcrt_set_spectral_proposal(ctx, mode, stream), ctx)


def mcrt_set_learned_proposal(ctx, m, mix: float = 0.1, stream=0):
    _check(load().mcrt_set_learned_proposal(ctx, m, mix, stream), ctx)


class Mlp:
    """The proposal network (device-resident FP32 master weights, FP16 copy,
    Adam state).  Arrays passed to the methods are torch CUDA tensors."""

    def __init__(self, K: int, device: int = 0):
        self.K = K
        self.device = device
        self.handle = mcrt_mlp_create(device, K)
        self.nparams = mcrt_mlp_nparams(K)

    def close(self):
        if getattr(self, "handle", None):
            mcrt_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta, feat_mean=None, feat_inv_std=None):
        fm = np.zeros(MCRT_NFEAT) if feat_mean is None else feat_mean
        fi = np.ones(MCRT_NFEAT) if feat_inv_std is None else feat_inv_std
        mcrt_mlp_set_params(self.handle, theta, fm, fi)

    def params(self, used: bool = False):
        return mcrt_mlp_get_params(self.handle, self.K, used)

    def forward(self, feat, p0, mix=0.1, out=None, stream=0):
        import torch
        n = feat.shape[0]
        if out is None:
            out = torch.empty((n, self.K + 2), dtype=torch.float32, device=feat.device)
        stride = 0 if p0.dim() == 1 else self.K
        mcrt_mlp_forward(self.handle, _ptr(feat), n, _ptr(p0), stride, mix, _ptr(out), stream)
        return out

    def loss_grad(self, feat, mom, p0, cost=None, c0=0.0, idx=None, n=None, mix=0.1, grad=None,
                  wgt=None, mode=0, stream=0):
        n = (idx.shape[0] if idx is not None else feat.shape[0]) if n is None else n
        stride = 0 if p0.dim() == 1 else self.K
        mcrt_mlp_loss_grad(self.handle, _ptr(feat), _ptr(mom), _ptr(cost), c0, _ptr(p0), stride,
                           _ptr(wgt), mode, feat.shape[0], _ptr(idx), n, mix, _ptr(grad), stream)

    def adam(self, grad=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=0):
        mcrt_mlp_adam_step(self.handle, _ptr(grad), lr, beta1, beta2, eps, stream)

    def last_loss(self) -> float:
        return mcrt_mlp_last_loss(self.handle)


def _ptr(a):
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _is_device(a):
    return hasattr(a, "is_cuda") and a.is_cuda


class Solver:
    """One library context for a grid.  Inputs may be numpy arrays (host) or
    torch CUDA tensors (device); outputs follow the ``out`` argument's memory."""

    def __init__(self, grid, kd=None, device: int = 0):
        g = mcrt_grid_desc()
        g.nx, g.ny, g.nz = grid.nx, grid.ny, grid.nz
        g.lx, g.ly, g.lz = grid.lx, grid.ly, grid.lz
        g.eps_wall[0], g.eps_wall[1] = grid.eps_wall
        g.T_wall[0], g.T_wall[1] = grid.T_wall
        g.reflect = grid.reflect
        g.device = device
        yf = getattr(grid, "yf", None)
        self._yf_keep = None if yf is None else np.ascontiguousarray(yf, dtype=np.float64)
        if self._yf_keep is not None:
            g.yf = self._yf_keep.ctypes.data_as(C.POINTER(C.c_double))
        g.xz_walls = int(getattr(grid, "xz_walls", 0))
        for f, t in enumerate(getattr(grid, "T_xz", (0.0, 0.0, 0.0, 0.0))):
            g.T_xz[f] = float(t)
        self.grid = grid
        self.device = device
        self.ctx = mcrt_create(g)
        if kd is not None:
            self.set_kdist(kd)

    def close(self):
        if getattr(self, "ctx", None):
            mcrt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_kdist(self, kd):
        """Upload the tables.  With kd.B None the library computes the band
        intensities from kd.nu_c and kd.dnu."""
        def arr(v):
            return None if v is None else np.ascontiguousarray(v, dtype=np.float64)

        def ptr(a):
            return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))

        self._kd_keep = [arr(kd.w_g), arr(kd.kappa), arr(kd.B), arr(kd.nu_c), arr(kd.dnu)]
        d = mcrt_kdist_desc()
        d.n_bands, d.n_g = kd.n_bands, kd.n_g
        d.w_g = ptr(self._kd_keep[0])
        d.T0, d.dT, d.nT = kd.T0, kd.dT, kd.nT
        d.kappa = ptr(self._kd_keep[1])
        d.B = ptr(self._kd_keep[2])
        d.x_ref = kd.x_ref
        d.nu_c = ptr(self._kd_keep[3])
        d.dnu = ptr(self._kd_keep[4])
        mcrt_set_kdist(self.ctx, d)
        self.kd = kd

    def set_fields(self, T, x=None, stream: int = 0):
        dev = _is_device(T)
        if dev:
            fp64 = 1 if str(T.dtype) == "torch.float64" else 0
            T = T.contiguous()
            x = None if x is None else x.contiguous()
        else:
            fp64 = 0 if np.asarray(T).dtype == np.float32 else 1
            dt = np.float64 if fp64 else np.float32
            T = np.ascontiguousarray(T, dtype=dt)
            x = None if x is None else np.ascontiguousarray(x, dtype=dt)
        mcrt_set_fields(self.ctx, _ptr(T), _ptr(x), fp64, MCRT_MEM_DEVICE if dev else MCRT_MEM_HOST,
                        stream)

    def set_cell_proposal(self, cn, cg, hemi, stream: int = 0):
        dev = _is_device(cn)
        if not dev:
            cn = np.ascontiguousarray(cn, dtype=np.uint64)
            cg = np.ascontiguousarray(cg, dtype=np.uint64)
            hemi = np.ascontiguousarray(hemi, dtype=np.uint32)
        mcrt_set_cell_proposal(self.ctx, _ptr(cn), _ptr(cg), _ptr(hemi),
                               MCRT_MEM_DEVICE if dev else MCRT_MEM_HOST, stream)

    @staticmethod
    def params(rays=128, seed=0, snapshot=0, ray_offset=0, tol=1e-4, max_steps=1 << 30,
               precision=MCRT_FP32, origin=MCRT_ORIGIN_UNIFORM, proposal=MCRT_PROPOSAL_PLANCK_TMAX,
               box=None, mg_levels=1, mg_steps=5, estimator=MCRT_EST_ERMC):
        p = mcrt_solve_params()
        p.rays_per_cell, p.max_steps, p.tol = rays, max_steps, tol
        p.mg_levels, p.mg_steps = mg_levels, mg_steps
        p.estimator = estimator
        p.seed, p.ray_offset, p.snapshot = seed, ray_offset, snapshot
        p.precision, p.origin, p.proposal = precision, origin, proposal
        p.use_box = 0 if box is None else 1
        if box is not None:
            for i in range(6):
                p.box[i] = int(box[i])
        return p

    def box_shape(self, box):
        b = box if box is not None else (0, self.grid.nx, 0, self.grid.ny, 0, self.grid.nz)
        return (b[5] - b[4], b[3] - b[2], b[1] - b[0])

    def solve_into(self, params, q, sigma=None, steps=None, stream: int = 0):
        """Solves into caller-owned buffers q / sigma / steps (all numpy or all
        torch CUDA tensors, box-sized)."""
        dev = _is_device(q)
        params.steps_out = None if steps is None else _ptr(steps).value
        mcrt_solve_qrad(self.ctx, params, _ptr(q), _ptr(sigma),
                        MCRT_MEM_DEVICE if dev else MCRT_MEM_HOST, stream)

    def solve(self, box=None, with_steps=False, **kw):
        """Host convenience: returns numpy q, sigma (and steps) shaped [bz, by, bx]."""
        shape = self.box_shape(box)
        q = np.zeros(shape)
        s = np.zeros(shape)
        st = np.zeros(shape, dtype=np.uint64) if with_steps else None
        self.solve_into(self.params(box=box, **kw), q, s, st)
        return (q, s, st) if with_steps else (q, s)

    def stats(self) -> dict:
        return mcrt_get_stats(self.ctx)

    def set_tuning(self, min_blocks_per_sm: int = 0, steps_per_round: int = 0,
                   scratch_mib: int = 0, long_ray_steps: int = 0, long_ray_flight: int = 0,
                   tally_binary32: int = 0, batch_per_snapshot: int = 0, claim_rays: int = 0,
                   tally_plain_loads: int = 0):
        mcrt_set_tuning(self.ctx, min_blocks_per_sm, steps_per_round, scratch_mib, long_ray_steps,
                        long_ray_flight, tally_binary32, batch_per_snapshot, claim_rays, tally_plain_loads)

    def tuning(self) -> dict:
        return mcrt_get_tuning(self.ctx)

    # learned proposal
    def features(self, cells=None, out=None, stream: int = 0):
        """Features [n, 12] (torch CUDA float32) of cells (torch int32, or None: all)."""
        import torch
        n = self.grid.ncells if cells is None else cells.shape[0]
        if out is None:
            out = torch.empty((n, MCRT_NFEAT), dtype=torch.float32, device=f"cuda:{self.device}")
        mcrt_cell_features(self.ctx, _ptr(cells), n, _ptr(out), stream)
        return out

    def tally(self, params, cells, mom=None, cost=None, q=None, sigma=None, stream: int = 0):
        """Second-moment and cost tallies [n, K, 2] of the listed cells from one
        FP32 solve (whole grid)."""
        import torch
        K = self.kd.n_bands * self.kd.n_g
        n = cells.shape[0]
        dev = f"cuda:{self.device}"
        if mom is None:
            mom = torch.empty((n, K, 2), dtype=torch.float32, device=dev)
        if cost is None:
            cost = torch.empty((n, K, 2), dtype=torch.float32, device=dev)
        mcrt_tally_moments(self.ctx, params, _ptr(cells), n, _ptr(mom), _ptr(cost), _ptr(q),
                           _ptr(sigma), stream)
        return mom, cost

    def plain_probs(self):
        return mcrt_get_plain_probs(self.ctx, self.kd.n_bands * self.kd.n_g)

    def set_cell_proposal_probs(self, q, stream: int = 0):
        mcrt_set_cell_proposal_probs(self.ctx, _ptr(q), stream)

    def cell_proposal(self):
        return mcrt_get_cell_proposal(self.ctx, self.grid.ncells, self.kd.n_bands, self.kd.n_g)

    def set_spectral_proposal(self, mode, stream: int = 0):
        """Per-cell spectral proposal at the cells' own temperatures (LOCAL) or
        mixed with the T_max proposal by temperature (HYBRID)."""
        mcrt_set_spectral_proposal(self.ctx, mode, stream)

    def set_learned_proposal(self, mlp, mix=0.1, stream: int = 0):
        mcrt_set_learned_proposal(self.ctx, mlp.handle, mix, stream)
