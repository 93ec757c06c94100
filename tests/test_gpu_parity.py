"""GPU parity: the CUDA library against the FP64 oracle, draw for draw.

Both sides consume the same Philox draws, so per-cell Q must agree to rounding:
|Q_gpu - Q_oracle| <= rtol * S_i with S_i the oracle's mean absolute tally
(sum of |terms| per ray, weighted): rtol = 1e-10 in FP64 mode and 1e-4 in FP32
mode.  S_i scales the tolerance because Q_i is a difference of terms of both
signs and can vanish where they cancel.  All calls go through the C ABI.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs, mcrt

pytestmark = pytest.mark.gpu

RTOL = {mcrt.MCRT_FP64: 1e-10, mcrt.MCRT_FP32: 1e-4}


def run_pair(grid, kd, T, x, rays, precision, seed=0, tol=1e-4, max_steps=1 << 20, origin=0,
             box=None, ray_offset=0, snapshot=0):
    orc = oracle.solve(grid, kd, T, x, rays=rays, seed=seed, tol=tol, max_steps=max_steps,
                       origin=origin, box=box, ray_offset=ray_offset, snapshot=snapshot)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, s, st = S.solve(box=box, with_steps=True, rays=rays, seed=seed, tol=tol,
                       max_steps=max_steps, origin=origin, precision=precision,
                       ray_offset=ray_offset, snapshot=snapshot)
    stats = S.stats()
    S.close()
    return orc, q, s, st, stats


def assert_parity(orc, q, s, st, precision):
    rtol = RTOL[precision]
    scale = orc["scale"]
    err = np.abs(q - orc["q"])
    bad = err > rtol * scale + 1e-300
    assert not bad.any(), (f"{bad.sum()} cells beyond {rtol} S; worst "
                           f"{np.max(err / np.maximum(scale, 1e-300)):.3e}")
    # Standard errors follow (they come from the same per-ray samples).  sigma^2 =
    # (M2 - Q^2) / (N - 1) with M2 the mean squared sample: an error dM2 in M2 moves
    # sigma by dM2 / (2 (N - 1) sigma^2) relative, so where the samples of a cell are
    # nearly equal (M2 >> (N - 1) sigma^2) the binary32 samples' rounding (a few
    # 1e-7 of each |Y|) is amplified by M2 / ((N - 1) sigma^2).  Over cells with
    # sigma > 1e-3 S that factor reaches about 1e4 at N = 64, hence the 2e-2
    # relative tolerance in FP32, 200 times Q's (binary64: 1e-8).
    srel = 1e-8 if precision == mcrt.MCRT_FP64 else 2e-2
    big = orc["sigma"] > 1e-3 * scale
    assert np.allclose(s[big], orc["sigma"][big], rtol=srel)
    if precision == mcrt.MCRT_FP64:
        assert np.array_equal(st, orc["steps"])
    else:
        assert abs(st.sum() / orc["steps"].sum() - 1.0) < 1e-3


@pytest.mark.parametrize("precision", [mcrt.MCRT_FP64, mcrt.MCRT_FP32])
@pytest.mark.parametrize("kap", [0.1, 1.0, 10.0])
def test_grey_slab_16x32x16_parity(precision, kap):
    grid, kd, T, x = inputs.grey_slab_16x32x16(kap)
    orc, q, s, st, stats = run_pair(grid, kd, T, x, 32, precision, seed=0, tol=1e-6)
    assert_parity(orc, q, s, st, precision)
    assert stats["rays"] == grid.ncells * 32
    assert stats["steps"] == st.sum()


@pytest.mark.parametrize("precision", [mcrt.MCRT_FP64, mcrt.MCRT_FP32])
def test_nongrey_channel_parity(precision):
    grid, kd, T, x = inputs.nongrey_channel(16, 16, 16, seed=3)
    orc, q, s, st, _ = run_pair(grid, kd, T, x, 64, precision, seed=5)
    assert_parity(orc, q, s, st, precision)


@pytest.mark.parametrize("precision", [mcrt.MCRT_FP64, mcrt.MCRT_FP32])
@pytest.mark.parametrize("reflect", [0, 1])
def test_grey_walls_x_field_parity(precision, reflect):
    grid, kd, T, x = inputs.nongrey_channel(12, 16, 10, seed=4, eps_wall=0.8, x_mode="field")
    grid.reflect = reflect
    orc, q, s, st, stats = run_pair(grid, kd, T, x, 48, precision, seed=6)
    assert_parity(orc, q, s, st, precision)
    assert stats["wall_hits"] > 0


@pytest.mark.parametrize("precision", [mcrt.MCRT_FP64, mcrt.MCRT_FP32])
def test_ragged_box_center_origin_offset(precision):
    """Ragged grid, ragged ray count, a crop box, centre origin, ray offset and a
    snapshot index."""
    grid, kd, T, x = inputs.nongrey_channel(7, 9, 5, seed=7, x_mode="field")
    box = (1, 6, 2, 9, 0, 3)
    orc, q, s, st, _ = run_pair(grid, kd, T, x, 37, precision, seed=(1 << 40) + 9, origin=1,
                                box=box, ray_offset=1000, snapshot=3)
    assert q.shape == (3, 7, 5)
    assert_parity(orc, q, s, st, precision)


def test_single_ray_and_step_cap():
    grid, kd, T, x = inputs.nongrey_channel(8, 8, 8, seed=8)
    orc, q, s, st, stats = run_pair(grid, kd, T, x, 1, mcrt.MCRT_FP64, seed=1, max_steps=3)
    assert np.all(s == 0.0)
    assert_parity(orc, q, s, st, mcrt.MCRT_FP64)
    assert stats["capped"] > 0 and np.all(st <= 3)


def test_empty_box_and_state_errors():
    grid, kd, T, x = inputs.nongrey_channel(8, 8, 8, seed=9)
    S = mcrt.Solver(grid, kd)
    q = np.zeros(1)
    with pytest.raises(mcrt.McrtError) as e:
        S.solve_into(S.params(rays=4), q)
    assert e.value.status == mcrt.MCRT_E_STATE
    S.set_fields(T, x)
    q0, s0 = S.solve(box=(2, 2, 0, 8, 0, 8), rays=4)
    assert q0.size == 0
    with pytest.raises(mcrt.McrtError) as e:
        S.solve(box=(0, 9, 0, 8, 0, 8), rays=4)
    assert e.value.status == mcrt.MCRT_E_ARG
    with pytest.raises(mcrt.McrtError) as e:
        S.solve(rays=4, tol=1.5)
    assert e.value.status == mcrt.MCRT_E_ARG
    with pytest.raises(mcrt.McrtError) as e:
        S.solve(rays=4, proposal=mcrt.MCRT_PROPOSAL_CELL)
    assert e.value.status == mcrt.MCRT_E_STATE
    Tbad = T.copy()
    Tbad[1, 2, 3] = np.nan
    with pytest.raises(mcrt.McrtError) as e:
        S.set_fields(Tbad, x)
    assert e.value.status == mcrt.MCRT_E_RANGE
    with pytest.raises(mcrt.McrtError) as e:  # the rejected field is forgotten
        S.solve(rays=4)
    assert e.value.status == mcrt.MCRT_E_STATE
    S.close()


def test_device_and_host_memory_paths_agree_bitwise():
    import torch
    grid, kd, T, x = inputs.nongrey_channel(16, 12, 8, seed=10)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    qh, sh = S.solve(rays=64, seed=2)
    Td = torch.tensor(T, device="cuda")
    xd = torch.tensor(x, device="cuda")
    S.set_fields(Td, xd)
    qd = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    sd = torch.zeros_like(qd)
    stream = torch.cuda.current_stream().cuda_stream
    S.solve_into(S.params(rays=64, seed=2), qd, sd, stream=stream)
    torch.cuda.synchronize()
    assert np.array_equal(qd.cpu().numpy(), qh) and np.array_equal(sd.cpu().numpy(), sh)
    # float32 inputs give the same FP32-mode result as float64 inputs rounded
    S.set_fields(T.astype(np.float32), x.astype(np.float32))
    q32a, _ = S.solve(rays=16, seed=3)
    S.set_fields(T.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64))
    q32b, _ = S.solve(rays=16, seed=3)
    assert np.array_equal(q32a, q32b)
    S.close()


def test_shards_union_equals_full_solve_bitwise():
    """Q_i depends only on cell i's rays (Section 3): disjoint boxes solved
    separately give the full solve bit for bit, so slabs shard across GPUs."""
    grid, kd, T, x = inputs.nongrey_channel(16, 16, 12, seed=11)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    full, fs = S.solve(rays=40, seed=4)
    parts = [S.solve(box=(0, 16, 0, 16, k0, k1), rays=40, seed=4) for k0, k1 in ((0, 5), (5, 12))]
    assert np.array_equal(np.concatenate([p[0] for p in parts], axis=0), full)
    assert np.array_equal(np.concatenate([p[1] for p in parts], axis=0), fs)
    S.close()


def test_fp32_matches_E3_closed_form():
    """FP32 mode on the 16x32x16 grey slab (kappa = 1, 128 rays) against the
    exponential-integral cell averages, within the sampled error."""
    from scipy.special import expn
    grid, kd, T, x = inputs.grey_slab_16x32x16(1.0)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, s = S.solve(rays=128, seed=0, tol=1e-6, precision=mcrt.MCRT_FP32)
    S.close()
    L, dy = 2.0, 2.0 / 32
    y0 = np.arange(32) * dy
    y1 = y0 + dy
    ref = 2 * inputs.SIGMA_SB * 1e12 / dy * (expn(3, y0) - expn(3, y1) + expn(3, L - y1) - expn(3, L - y0))
    row = q.mean(axis=(0, 2))
    se = np.sqrt((s**2).sum(axis=(0, 2))) / 256
    z = (row - ref) / se
    assert np.max(np.abs(z)) < 4 and np.sqrt(np.mean(z**2)) < 1.6


def test_full_size_channel_64cubed_sampled_cells():
    """The benchmark workload (64^3 channel, 40x8 k-distribution, 1000 rays,
    FP32, whole-grid launch) against the oracle on sampled cells."""
    grid, kd, T, x = inputs.nongrey_channel(64, 64, 64, seed=0)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, s = S.solve(rays=1000, seed=0, tol=1e-4, max_steps=1 << 20, precision=mcrt.MCRT_FP32)
    S.close()
    rng = np.random.default_rng(0)
    cells = [tuple(rng.integers(0, 64, 3)) for _ in range(12)] + [(0, 0, 0), (63, 63, 63), (5, 0, 9), (7, 63, 2)]
    for (i, j, k) in cells:
        o = oracle.solve(grid, kd, T, x, rays=1000, seed=0, tol=1e-4, max_steps=1 << 20,
                         box=(i, i + 1, j, j + 1, k, k + 1))
        assert abs(q[k, j, i] - o["q"][0, 0, 0]) <= 1e-4 * o["scale"][0, 0, 0], (i, j, k)


@pytest.mark.parametrize("rays", [255, 256, 257, 600])
def test_fp32_multi_block_cells_parity(rays):
    """Cells whose rays span several ray blocks of the FP32 kernel (and ragged
    last blocks) against the oracle."""
    grid, kd, T, x = inputs.nongrey_channel(6, 8, 5, seed=12, eps_wall=0.9)
    orc, q, s, st, stats = run_pair(grid, kd, T, x, rays, mcrt.MCRT_FP32, seed=13)
    assert_parity(orc, q, s, st, mcrt.MCRT_FP32)
    assert stats["rays"] == grid.ncells * rays


def test_fp32_results_independent_of_launch_shape():
    """The FP32 kernel reduces every cell's samples in a fixed order, so the
    occupancy target does not change a single bit."""
    grid, kd, T, x = inputs.nongrey_channel(20, 16, 12, seed=14, eps_wall=0.8)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q0, s0, st0 = S.solve(rays=300, seed=3, with_steps=True)
    # occupancy target, steps per round and the scratch cap (1 MiB forces many
    # chunks here) change nothing
    for mb, k, mib in ((1, 1, 0), (3, 2, 0), (2, 4, 1), (4, 4, 0), (1, 4, 3), (2, 1, 0)):
        S.set_tuning(mb, k, mib)
        assert S.tuning() == {"min_blocks_per_sm": mb, "steps_per_round": k,
                              "scratch_mib": mib if mib else 4096, "long_ray_steps": 1024,
                              "long_ray_flight": 32, "tally_binary32": 0, "tally_plain_loads": 0,
                              "claim_rays": 1024, "batch_per_snapshot": 0}
        q, s, st = S.solve(rays=300, seed=3, with_steps=True)
        assert np.array_equal(q, q0) and np.array_equal(s, s0) and np.array_equal(st, st0)
    # the claimed runs: one cell at a time, or as long as the solve allows
    for cr in (32, 1 << 20):
        S.set_tuning(claim_rays=cr)
        assert S.tuning()["claim_rays"] == cr
        q, s, st = S.solve(rays=300, seed=3, with_steps=True)
        assert np.array_equal(q, q0) and np.array_equal(s, s0) and np.array_equal(st, st0)
    with pytest.raises(mcrt.McrtError):
        S.set_tuning(9)
    with pytest.raises(mcrt.McrtError):
        S.set_tuning(claim_rays=5)
    S.close()


@pytest.mark.parametrize("stretched,levels", [(False, 1), (True, 1), (False, 6)])
def test_dns_size_256x192x128_crop_against_oracle(stretched, levels):
    """The DNS-size channel (256 x 192 x 128, 40x8 k-distribution, x_H2O field,
    grey walls eps = 0.8, 512 rays, FP32 march with FP64 tallies): the whole field
    is solved on the GPU and its central 32^3 crop is checked cell by cell against
    the FP64 oracle on the same draws (rays cross the full field).  Also on a
    wall-refined grid and with the multigrid march on 6 grids."""
    grid, kd, T, x = inputs.nongrey_channel(256, 192, 128, seed=3, eps_wall=0.8, x_mode="field")
    if stretched:
        grid.yf = inputs.channel_faces(192, grid.ly, 1.5)
        T, x = inputs.channel_fields(grid, 3, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    q, s = S.solve(rays=512, seed=0, tol=1e-4, max_steps=1 << 20, precision=mcrt.MCRT_FP32,
                   mg_levels=levels, mg_steps=5)
    st = S.stats()
    S.close()
    assert st["rays"] == grid.ncells * 512 and st["wall_hits"] > 0
    box = (112, 144, 80, 112, 48, 80)
    o = oracle.solve(grid, kd, T, x, rays=512, seed=0, tol=1e-4, max_steps=1 << 20, box=box,
                     mg_levels=levels, mg_steps=5)
    crop = q[48:80, 80:112, 112:144]
    err = np.abs(crop - o["q"])
    assert np.all(err <= 1e-4 * o["scale"]), np.max(err / o["scale"])
    big = o["sigma"] > 1e-3 * o["scale"]
    assert np.allclose(s[48:80, 80:112, 112:144][big], o["sigma"][big], rtol=2e-2)


def test_binary64_tally_against_binary32_tally_and_oracle():
    """The per-cell tallies (Eq. 8) of the FP32 path: binary64 by default (each run
    of 32 samples summed exactly, the runs added with Neumaier's compensated
    binary64 sum: within about 2^-51 of sum |Y| of the exact sum of the samples),
    compensated binary32 pairs on request (within about 2e-7 of sum |Y|).  Same
    draws, same samples: the two tallies differ by at most the binary32 bound,
    sum |Y| / N <= S_i, and both stay within the FP32 tolerance of the oracle.
    A ragged ray count (not a multiple of 32) exercises the last, partial run."""
    import torch
    grid, kd, T, x = inputs.nongrey_channel(16, 16, 16, seed=3)
    rays = 203
    orc = oracle.solve(grid, kd, T, x, rays=rays, seed=5)
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    res = {}
    for mode in (0, 1):
        S.set_tuning(tally_binary32=mode)
        assert S.tuning()["tally_binary32"] == mode
        q, s = S.solve(rays=rays, seed=5, precision=mcrt.MCRT_FP32)
        res[mode] = (q, s)
    S.close()
    scale = orc["scale"]
    for mode in (0, 1):
        err = np.abs(res[mode][0] - orc["q"]) / scale
        assert err.max() <= 1e-4, (mode, err.max())
    d = np.abs(res[0][0] - res[1][0]) / scale
    assert d.max() <= 3e-7, d.max()
    assert np.any(res[0][0] != res[1][0])  # the two tallies are different arithmetic


def test_tma_fed_tally_equals_plain_loads_bitwise():
    """The binary64 tally reads the samples through the tensor memory accelerator
    (tiled bulk copies with the 128-byte swizzle, two buffers per warp) when the
    ray count is a multiple of 4, else by plain loads; both run the same exact
    32-sample runs in the same order, so Q, sigma and the step counts agree bit
    for bit.  Ragged grids (positions outside the box in the last bricks, a chunk
    not a multiple of 32 positions), a sub-box, ray counts below, at and across
    one 32-sample run, and one that forces several solve chunks."""
    import torch
    grid, kd, T, x = inputs.nongrey_channel(13, 11, 9, seed=21, eps_wall=0.8, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    cases = [dict(rays=4), dict(rays=32), dict(rays=36), dict(rays=100), dict(rays=1000),
             dict(rays=64, box=(2, 11, 1, 10, 3, 8))]
    for kw in cases:
        res = []
        for plain in (0, 1):
            S.set_tuning(tally_plain_loads=plain)
            assert S.tuning()["tally_plain_loads"] == plain
            res.append(S.solve(seed=8, precision=mcrt.MCRT_FP32, with_steps=True, **kw))
        for a, b in zip(*res):
            assert np.array_equal(a, b), kw
    # several chunks (1 MiB of scratch) with both readers
    res = []
    for plain in (0, 1):
        S.set_tuning(scratch_mib=1, tally_plain_loads=plain)
        res.append(S.solve(rays=400, seed=9, precision=mcrt.MCRT_FP32, with_steps=True))
    for a, b in zip(*res):
        assert np.array_equal(a, b)
    S.set_tuning()
    # and the default reader against the oracle
    orc = oracle.solve(grid, kd, T, x, rays=100, seed=8)
    q, s = S.solve(rays=100, seed=8, precision=mcrt.MCRT_FP32)
    assert np.all(np.abs(q - orc["q"]) <= 1e-4 * orc["scale"])
    with pytest.raises(mcrt.McrtError):
        S.set_tuning(tally_plain_loads=2)
    S.close()


def test_claimed_blocks_of_rays_bitwise():
    """A cell with more rays than a claim (mcrt_tuning.claim_rays) is traced in
    blocks of rays claimed one at a time, by whichever warps take them; every
    sample depends only on its cell and ray index, so Q, sigma and the step
    counts equal those of whole-cell claims bit for bit: the plain proposal and a
    per-cell proposal (staged per warp for each claim), blocks of 32 and 64 rays
    (300 rays: a ragged last block), with long rays handed off."""
    import torch
    grid, kd, T, x = inputs.nongrey_channel(10, 9, 7, seed=31, eps_wall=0.8, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    nb, ng, nc = kd.n_bands, kd.n_g, grid.ncells
    rng = np.random.default_rng(5)

    def cum(rows, k):
        c = rng.integers(1, 2**26, size=(rows, k)).astype(np.int64)
        c[:, -1] += 2**32 - c.sum(axis=1)
        return np.cumsum(c, axis=1).astype(np.uint64)

    S.set_cell_proposal(cum(nc, nb), cum(nc * nb, ng).reshape(nc, nb, ng),
                        rng.integers(1, 2**23, size=nc).astype(np.uint32))
    for proposal in (mcrt.MCRT_PROPOSAL_PLANCK_TMAX, mcrt.MCRT_PROPOSAL_CELL):
        kw = dict(rays=300, seed=7, precision=mcrt.MCRT_FP32, proposal=proposal, with_steps=True)
        S.set_tuning(claim_rays=4096, long_ray_steps=8, long_ray_flight=-1)
        ref = S.solve(**kw)
        assert S.stats()["long_rays"] > 0
        for cr in (32, 50):
            S.set_tuning(claim_rays=cr, long_ray_steps=8, long_ray_flight=-1)
            got = S.solve(**kw)
            for a, b in zip(ref, got):
                assert np.array_equal(a, b), (proposal, cr)
    S.close()


def test_segmented_tally_split_and_in_order_agree_bitwise():
    """More than 64 runs of 32 samples per cell (N > 2048): the runs form segments
    of equal length (the last one shorter) whose compensated sums are added in
    order.  The TMA-fed tally sums every segment with a warp of its own and a
    second kernel adds them; the plain-load tally and the allocation-free solve
    add a cell's segments in one warp.  All give the same Q, sigma and step counts
    bit for bit: one segment (2048 rays), two (2052: 65 runs, the last sample run
    ragged), three (4100), several solve chunks, a ray count that only the
    plain-load reader takes (2049); and the oracle at the FP32 tolerance."""
    import ctypes as C
    import torch
    grid, kd, T, x = inputs.nongrey_channel(7, 6, 5, seed=23, eps_wall=0.8, x_mode="field")
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    for rays in (2048, 2052, 4100, 2049):
        res = []
        for plain in (0, 1):
            S.set_tuning(tally_plain_loads=plain)
            res.append(S.solve(rays=rays, seed=12, precision=mcrt.MCRT_FP32, with_steps=True))
            if plain == 0 and rays in (2052, 4100):
                # trace, long-ray march, the segments' sums, their combination
                assert S.stats()["launches"] == 4, rays
        for a, b in zip(*res):
            assert np.array_equal(a, b), rays
        # several chunks (1 MiB of scratch: about 60 positions each)
        S.set_tuning(scratch_mib=1)
        q, s, st = S.solve(rays=rays, seed=12, precision=mcrt.MCRT_FP32, with_steps=True)
        S.set_tuning()
        assert np.array_equal(q, res[0][0]) and np.array_equal(s, res[0][1]) and np.array_equal(st, res[0][2])
    # the allocation-free solve adds the segments in one warp
    stream = torch.cuda.current_stream().cuda_stream
    qn = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    sn = torch.zeros_like(qn)
    mcrt.mcrt_solve_qrad_noalloc(S.ctx, S.params(rays=4100, seed=12, precision=mcrt.MCRT_FP32),
                                 C.c_void_p(qn.data_ptr()), C.c_void_p(sn.data_ptr()), stream)
    torch.cuda.synchronize()
    q, s = S.solve(rays=4100, seed=12, precision=mcrt.MCRT_FP32)
    assert np.array_equal(qn.cpu().numpy(), q) and np.array_equal(sn.cpu().numpy(), s)
    orc = oracle.solve(grid, kd, T, x, rays=2052, seed=12)
    q, s = S.solve(rays=2052, seed=12, precision=mcrt.MCRT_FP32)
    assert np.all(np.abs(q - orc["q"]) <= 1e-4 * orc["scale"])
    S.close()


def test_binary64_tally_sign_mix_and_launch_independence():
    """Grey walls at both temperatures give cells whose samples take both signs
    (Q_i a difference of large terms); the binary64 tally is reproduced bit for
    bit under other launch shapes and agrees with the oracle."""
    import torch
    grid, kd, T, x = inputs.nongrey_channel(12, 16, 10, seed=4, eps_wall=0.8, x_mode="field")
    orc = oracle.solve(grid, kd, T, x, rays=97, seed=6)
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    outs = []
    for shape in ((0, 0), (1, 1), (2, 2)):
        S.set_tuning(*shape)
        outs.append(S.solve(rays=97, seed=6, precision=mcrt.MCRT_FP32))
    S.close()
    for q, s in outs[1:]:
        assert np.array_equal(q, outs[0][0]) and np.array_equal(s, outs[0][1])
    err = np.abs(outs[0][0] - orc["q"]) / orc["scale"]
    assert err.max() <= 1e-4
