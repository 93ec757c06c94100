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
                ("T_wall", C.c_double * 2), ("reflect", C.c_int), ("device", C.c_int)]


class mcrt_kdist_desc(C.Structure):
    _fields_ = [("n_bands", C.c_int), ("n_g", C.c_int), ("w_g", C.POINTER(C.c_double)),
                ("T0", C.c_double), ("dT", C.c_double), ("nT", C.c_int),
                ("kappa", C.POINTER(C.c_double)), ("B", C.POINTER(C.c_double)),
                ("x_ref", C.c_double)]


class mcrt_solve_params(C.Structure):
    _fields_ = [("rays_per_cell", C.c_int), ("max_steps", C.c_int), ("tol", C.c_double),
                ("seed", C.c_uint64), ("ray_offset", C.c_uint64), ("snapshot", C.c_uint32),
                ("precision", C.c_int), ("origin", C.c_int), ("proposal", C.c_int),
                ("use_box", C.c_int), ("box", C.c_int * 6), ("steps_out", C.c_void_p)]


class mcrt_tuning(C.Structure):
    _fields_ = [("min_blocks_per_sm", C.c_int), ("steps_per_round", C.c_int),
                ("scratch_mib", C.c_int)]


class mcrt_batch_item(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("q_out", C.c_void_p), ("sigma_out", C.c_void_p),
                ("snapshot", C.c_uint32)]


class mcrt_solve_stats(C.Structure):
    _fields_ = [("steps", C.c_uint64), ("rays", C.c_uint64), ("capped", C.c_uint64),
                ("wall_hits", C.c_uint64), ("max_ray_steps", C.c_uint64), ("T_max", C.c_double),
                ("kernel_ms", C.c_float),
                ("launches", C.c_int)]


_lib = None
_lock = threading.Lock()
EXPORTS = ("mcrt_create", "mcrt_set_kdist", "mcrt_set_fields", "mcrt_set_cell_proposal",
           "mcrt_solve_qrad", "mcrt_get_stats", "mcrt_destroy", "mcrt_status_string",
           "mcrt_last_error", "mcrt_set_tuning", "mcrt_get_tuning", "mcrt_solve_qrad_noalloc",
           "mcrt_batch_create", "mcrt_batch_run", "mcrt_batch_get_stats", "mcrt_batch_last_error",
           "mcrt_batch_destroy")


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
        for f in EXPORTS:
            if f not in ("mcrt_status_string", "mcrt_last_error", "mcrt_batch_last_error"):
                getattr(L, f).restype = C.c_int
        _lib = L
        return _lib


def _check(rc, ctx=None):
    if rc != MCRT_OK:
        msg = load().mcrt_last_error(ctx).decode() if ctx else ""
        raise McrtError(rc, msg)


# --- the C entry points, same names ---------------------------------------------

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
                    scratch_mib: int = 0):
    t = mcrt_tuning()
    t.min_blocks_per_sm = min_blocks_per_sm
    t.steps_per_round = steps_per_round
    t.scratch_mib = scratch_mib
    _check(load().mcrt_set_tuning(ctx, C.byref(t)), ctx)


def mcrt_get_tuning(ctx) -> dict:
    t = mcrt_tuning()
    _check(load().mcrt_get_tuning(ctx, C.byref(t)), ctx)
    return {"min_blocks_per_sm": t.min_blocks_per_sm, "steps_per_round": t.steps_per_round,
            "scratch_mib": t.scratch_mib}


def mcrt_destroy(ctx):
    if ctx:
        load().mcrt_destroy(ctx)


def mcrt_status_string(status: int) -> str:
    return load().mcrt_status_string(status).decode()


# --- convenience wrapper ----------------------------------------------------------

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
        self._kd_keep = [np.ascontiguousarray(kd.w_g, dtype=np.float64),
                         np.ascontiguousarray(kd.kappa, dtype=np.float64),
                         np.ascontiguousarray(kd.B, dtype=np.float64)]
        d = mcrt_kdist_desc()
        d.n_bands, d.n_g = kd.n_bands, kd.n_g
        d.w_g = self._kd_keep[0].ctypes.data_as(C.POINTER(C.c_double))
        d.T0, d.dT, d.nT = kd.T0, kd.dT, kd.nT
        d.kappa = self._kd_keep[1].ctypes.data_as(C.POINTER(C.c_double))
        d.B = self._kd_keep[2].ctypes.data_as(C.POINTER(C.c_double))
        d.x_ref = kd.x_ref
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
               box=None):
        p = mcrt_solve_params()
        p.rays_per_cell, p.max_steps, p.tol = rays, max_steps, tol
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
                   scratch_mib: int = 0):
        mcrt_set_tuning(self.ctx, min_blocks_per_sm, steps_per_round, scratch_mib)

    def tuning(self) -> dict:
        return mcrt_get_tuning(self.ctx)
