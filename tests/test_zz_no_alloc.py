"""The allocation-free solve (collected last on purpose).

Callers that may not allocate device memory while they run (hosts that reserve
the GPU's memory up front) use mcrt_solve_qrad_noalloc, whose scratch lives in a
static device array.  Through the C ABI it must give what the regular FP32 solve
gives, bit for bit (the same kernels, the same long-ray hand-off), on two calls in
a row -- the second call finds the first call's data in the shared array -- and a
call after the first must leave the device's free memory unchanged.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs, mcrt

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("long_steps", [0, 32])
def test_noalloc_solve_matches_regular_solve_on_two_calls(long_steps):
    import torch
    L = mcrt.load()
    grid, kd, T, x = inputs.nongrey_channel(20, 16, 12, seed=21, eps_wall=0.8, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    # 0: the default thresholds; 32 segments, any flight: thousands of rays go
    # through the warp-parallel march in both solves
    S.set_tuning(long_ray_steps=long_steps, long_ray_flight=-1 if long_steps else 0)
    stream = torch.cuda.current_stream().cuda_stream
    q_ref = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    s_ref = torch.zeros_like(q_ref)
    S.solve_into(S.params(rays=300, seed=5, precision=mcrt.MCRT_FP32), q_ref, s_ref, stream=stream)
    torch.cuda.synchronize()
    st = S.stats()
    assert st["long_overflow"] == 0
    if long_steps:
        assert 0 < st["long_rays"] < 65536
    scale = oracle.solve(grid, kd, T, x, rays=300, seed=5)["scale"]
    outs = [(torch.full(grid.shape, float("nan"), dtype=torch.float64, device="cuda"),
             torch.full(grid.shape, float("nan"), dtype=torch.float64, device="cuda")) for _ in range(2)]
    params = S.params(rays=300, seed=5, precision=mcrt.MCRT_FP32)
    torch.cuda.synchronize()
    for call, (q, s) in enumerate(outs):
        free0 = torch.cuda.mem_get_info()[0]
        rc = L.mcrt_solve_qrad_noalloc(S.ctx, C.byref(params), _ptr(q), _ptr(s), C.c_void_p(stream))
        torch.cuda.synchronize()
        assert rc == mcrt.MCRT_OK, L.mcrt_last_error(S.ctx)
        if call:  # the first call may load the array and the kernels; later ones allocate nothing
            assert torch.cuda.mem_get_info()[0] == free0
        qn, qr = q.cpu().numpy(), q_ref.cpu().numpy()
        assert np.all(np.isfinite(qn)), call
        assert np.array_equal(qn, qr), call
        assert np.all(np.abs(qn - qr) <= 1e-4 * scale), call
        assert np.array_equal(s.cpu().numpy(), s_ref.cpu().numpy()), call
    S.close()


def test_noalloc_chunked_box_with_hand_offs_across_chunks():
    """A solve larger than one fill of the static array runs in several launches
    (about 2,800 cell positions of 5,000 rays each per fill here), with long rays
    handed off in every chunk; it must equal the regular solve (one chunk) bit for
    bit, and the second call must allocate nothing."""
    import torch
    L = mcrt.load()
    grid, kd, T, x = inputs.nongrey_channel(24, 24, 16, seed=23)
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    S.set_tuning(long_ray_steps=256, long_ray_flight=-1)
    rays = 5000
    stream = torch.cuda.current_stream().cuda_stream
    q_ref = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    s_ref = torch.zeros_like(q_ref)
    st_ref = torch.zeros(grid.shape, dtype=torch.int64, device="cuda")
    params = S.params(rays=rays, seed=8, precision=mcrt.MCRT_FP32)
    S.solve_into(params, q_ref, s_ref, st_ref, stream=stream)
    torch.cuda.synchronize()
    st = S.stats()
    assert st["long_overflow"] == 0 and st["long_rays"] > 0
    # chunks of the allocation-free solve: the array less its counters and the
    # 2^16-entry long-ray region, per position the samples and a step sum
    per_pos = rays * 4 + 8
    chunk = ((64 << 20) - 256 - 65536 * 128 - 256) // per_pos  # the documented 64 MiB array
    nchunks = -(-grid.ncells // chunk)
    assert nchunks >= 3
    # every chunk's hand-offs fit the 2^16-entry region (else the bits could differ)
    assert st["long_rays"] / nchunks < 32768
    outs = [(torch.full_like(q_ref, float("nan")), torch.full_like(s_ref, float("nan")),
             torch.full_like(st_ref, -1)) for _ in range(2)]
    torch.cuda.synchronize()
    for call, (q, s, stp) in enumerate(outs):
        p = S.params(rays=rays, seed=8, precision=mcrt.MCRT_FP32)
        p.steps_out = stp.data_ptr()
        free0 = torch.cuda.mem_get_info()[0]
        rc = L.mcrt_solve_qrad_noalloc(S.ctx, C.byref(p), _ptr(q), _ptr(s), C.c_void_p(stream))
        torch.cuda.synchronize()
        assert rc == mcrt.MCRT_OK, L.mcrt_last_error(S.ctx)
        if call:
            assert torch.cuda.mem_get_info()[0] == free0
        assert torch.equal(q, q_ref), call
        assert torch.equal(s, s_ref), call
        assert torch.equal(stp, st_ref), call
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
