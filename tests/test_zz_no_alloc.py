"""The allocation-free solve (collected last on purpose).

Callers that may not allocate device memory while they run (hosts that reserve
the GPU's memory up front) use mcrt_solve_qrad_noalloc, whose scratch lives in a
static device array.  Through the C ABI it must give what the regular FP32 solve
gives, within the FP32 parity tolerance (1e-4 of the oracle's per-cell scale),
on two calls in a row -- the second call finds the first call's data in the
shared array.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs, mcrt

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_solve_matches_regular_solve_on_two_calls():
    import torch
    L = mcrt.load()
    grid, kd, T, x = inputs.nongrey_channel(20, 16, 12, seed=21, eps_wall=0.8, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    stream = torch.cuda.current_stream().cuda_stream
    q_ref = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    s_ref = torch.zeros_like(q_ref)
    S.solve_into(S.params(rays=300, seed=5, precision=mcrt.MCRT_FP32), q_ref, s_ref, stream=stream)
    torch.cuda.synchronize()
    scale = oracle.solve(grid, kd, T, x, rays=300, seed=5)["scale"]
    for call in range(2):
        q = torch.full(grid.shape, float("nan"), dtype=torch.float64, device="cuda")
        s = torch.full_like(q, float("nan"))
        params = S.params(rays=300, seed=5, precision=mcrt.MCRT_FP32)
        rc = L.mcrt_solve_qrad_noalloc(S.ctx, C.byref(params), _ptr(q), _ptr(s), C.c_void_p(stream))
        torch.cuda.synchronize()
        assert rc == mcrt.MCRT_OK, L.mcrt_last_error(S.ctx)
        qn, qr = q.cpu().numpy(), q_ref.cpu().numpy()
        assert np.all(np.isfinite(qn)), call
        assert np.all(np.abs(qn - qr) <= 1e-4 * scale), call
        sn, sr = s.cpu().numpy(), s_ref.cpu().numpy()
        assert np.allclose(sn, sr, rtol=1e-4, atol=1e-4 * scale.max()), call
    S.close()


def test_noalloc_rejects_what_does_not_fit_and_non_fp32():
    import torch
    L = mcrt.load()
    grid, kd, T, x = inputs.nongrey_channel(4, 4, 4, seed=22)
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    q = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    too_many = S.params(rays=20_000_000, seed=1, precision=mcrt.MCRT_FP32)
    rc = L.mcrt_solve_qrad_noalloc(S.ctx, C.byref(too_many), _ptr(q), None, None)
    assert rc == mcrt.MCRT_E_ARG
    assert b"static scratch" in L.mcrt_last_error(S.ctx)
    fp64 = S.params(rays=8, seed=1, precision=mcrt.MCRT_FP64)
    assert L.mcrt_solve_qrad_noalloc(S.ctx, C.byref(fp64), _ptr(q), None, None) == mcrt.MCRT_E_ARG
    S.close()
