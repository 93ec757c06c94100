#!/usr/bin/env python3
"""Benchmark of the ERMC Q_rad solve on GB300.

Workload (one "step" = one full solve): the non-grey turbulent channel on a
64^3 grid (4 pi x 2 x 2 pi m), 40 narrow bands x 8 g-points of synthetic
correlated-k tables, black walls at 500 / 1000 K, 1000 rays per cell, FP32
traversal with FP64 tallies.  Each step traces a fresh block of ray indices
(ray_offset advances), so no result is reused.  Under torchrun every rank solves
its own snapshot (field seed = rank): weak scaling with no data-path collective.
``--scaling strong`` instead splits one snapshot into z-slabs: the field is
broadcast once before timing, and every timed step solves each rank's slab and
gathers Q and sigma on rank 0.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-cell steps/s"
UNIT = "steps/s"
LANES_PER_SM = 128            # FP32/INT lanes per SM (one op per lane per clock)
# Algorithmic FP32/INT operations of the estimator, counted from the source:
OPS_PER_STEP = 44             # axis choice, table position, two interpolations,
                              # absorption, tally, DDA advance
OPS_PER_RAY = 260             # 2 Philox4x32-10 blocks (2 x 80), sampling, direction,
                              # origin, DDA set-up, sample store
GATHER_BYTES_PER_STEP = 8     # algorithmic bytes of a step: the FP32 {T, x} entry of the traversed
                              # cell (the kappa and B nodes are table reads, amortised)
EXP_PER_STEP = 1              # one exponential per step (Eq. 2)
# DRAM bytes of one trace launch of the default workload (64^3, 1000 rays):
# dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture of the current
# trace kernel (profiles/dram_nongrey_64cubed_1000rays.md)
TRACE_DRAM_BYTES_64_1000 = 16984064 + 1001364992


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", "--n", dest="n", type=int, default=64, help="grid is n^3")
    ap.add_argument("--rays", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--long-ray-steps", type=int, default=0,
                    help="hand-off threshold in segments (0: the library default, < 0: off)")
    ap.add_argument("--long-ray-flight", type=int, default=0,
                    help="x/z crossings left for a hand-off (0: the library default, < 0: any)")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: one snapshot per rank; strong: one snapshot split over the ranks")
    return ap.parse_args()


def workload_config(a):
    return {"workload": f"nongrey_channel_{a.n}x{a.n}x{a.n}_40x8kdist_{a.rays}rays",
            "grid": [a.n, a.n, a.n], "box_m": [4 * math.pi, 2.0, 2 * math.pi],
            "rays_per_cell": a.rays, "bands": 40, "g_points": 8, "tol": 1e-4,
            "walls": "black, 500 K / 1000 K", "x_h2o": 0.1,
            "T_field": "linear 500->1000 K + 5% k^-5/3 Gaussian random field",
            "precision": "fp32 traversal and per-ray samples; per-cell tallies in binary64 (Neumaier-compensated sums of exact 32-sample runs)",
            "l2": "flushed between timed steps (256 MiB write)", "seed": 0,
            "long_ray_hand_off": {"steps": a.long_ray_steps or 1024, "flight": a.long_ray_flight or 32}}


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def sm_count(device):
    import torch
    return torch.cuda.get_device_properties(device).multi_processor_count


def ceilings(device, field_bytes, full=True):
    """Measured rates of the two operations a march step repeats: the exponential
    and a random 8-byte gather (library probes, one timed launch each); the
    gather from a buffer of the field's size, and (full) from 32 MiB and 4 GiB."""
    from paper_1810_00188_gb300 import mcrt
    ex2, mhz = mcrt.mcrt_probe_ex2(device)
    sizes = {"field": 1 << max(12, int(field_bytes - 1).bit_length())}
    if full:
        sizes.update({"32MiB": 32 << 20, "4GiB": 4 << 30})
    g = {k: mcrt.mcrt_probe_gather(device, v) for k, v in sizes.items()}
    return {"ex2_per_s": ex2, "ex2_per_clk_per_sm": ex2 / (sm_count(device) * mhz * 1e6), "probe_sm_mhz": mhz,
            "gather8_per_s": g, "gather_buffer_bytes": sizes,
            "note": "random 8-byte loads, 8 in flight per thread, full occupancy; "
                    "ex2.approx chains, 8 per thread"}


def cpu_baseline(a, target_s=12.0):
    """The FP64 oracle on the host cores on z-slabs of the same workload."""
    import oracle
    from paper_1810_00188_gb300 import inputs
    grid, kd, T, x = inputs.nongrey_channel(a.n, a.n, a.n, seed=0)
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    r = oracle.solve(grid, kd, T, x, rays=a.rays, seed=0, tol=1e-4, max_steps=1 << 20,
                     box=(0, a.n, 0, a.n, 0, 1), nthreads=threads)
    t1 = time.perf_counter() - t0
    planes = max(1, min(a.n, int(round(target_s / max(t1, 1e-3)))))
    t0 = time.perf_counter()
    r = oracle.solve(grid, kd, T, x, rays=a.rays, seed=0, tol=1e-4, max_steps=1 << 20,
                     box=(0, a.n, 0, a.n, 1, 1 + min(planes, a.n - 1)), nthreads=threads)
    dt = time.perf_counter() - t0
    steps = float(r["steps"].sum())
    return {"value": steps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{min(planes, a.n - 1)} z-planes ({a.n}x{a.n} cells each) x {a.rays} rays, "
                      f"{steps:.3g} steps in {dt:.1f} s"}


def field_error(grid, kd, T, x, rays, snapshot, qs, box=None, crop=None, tol=1e-4, ray_offset=0,
                max_steps=1 << 20):
    """|Q_gpu - Q_oracle| / S_i over the cells of `box` (the whole grid when None)
    for each GPU result in qs; crop maps a whole-field result onto the box."""
    import numpy as np

    import oracle
    ref = oracle.solve(grid, kd, T, x, rays=rays, seed=0, snapshot=snapshot, tol=tol,
                       ray_offset=ray_offset, max_steps=max_steps, box=box,
                       nthreads=oracle.default_threads())
    out = {"rays": rays, "cells": int(ref["q"].size), "tolerance": {"fp32": 1e-4, "fp64": 1e-10}}
    for name, qg in qs.items():
        qc = qg if crop is None else qg[crop]
        e = np.abs(qc - ref["q"]) / np.maximum(ref["scale"], 1e-300)
        out[name] = {"max": float(e.max()), "p99": float(np.percentile(e, 99)),
                     "mean": float(e.mean())}
    return out


def configs_extra(sp):
    """The other configurations, GPU beside the FP64 oracle on the host cores (all
    cores and one core, bounded samples): the grey slab 16x32x16 x 128 rays (FP64
    and FP32), the 64^3 x 1000-ray channel (oracle only: the main line times the
    GPU), and the DNS-size 256x192x128 channel x 512 rays with grey walls (GPU:
    the whole field; oracle: z-planes of the central 32^3 crop, rays through the
    whole field)."""
    import numpy as np
    import torch

    import oracle
    from paper_1810_00188_gb300 import inputs, mcrt
    allc = oracle.default_threads()
    out = {"oracle_cores": allc}

    def gpu(grid, kd, T, x, rays, prec, seed, tol, reps=2, keep=None):
        S = mcrt.Solver(grid, kd)
        S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"), stream=sp)
        q = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
        sg = torch.empty_like(q)
        best = None
        for k in range(reps + 1):
            S.solve_into(S.params(rays=rays, seed=seed, tol=tol, max_steps=1 << 20, precision=prec,
                                  ray_offset=k * rays), q, sg, stream=sp)
            st = S.stats()
            if k and (best is None or st["kernel_ms"] < best["kernel_ms"]):
                best = st
        if keep is not None:  # one more solve on the first ray block, for the error check
            S.solve_into(S.params(rays=rays, seed=seed, tol=tol, max_steps=1 << 20, precision=prec),
                         q, sg, stream=sp)
            keep.append(q.cpu().numpy())
        S.close()
        return {"ms": best["kernel_ms"], "steps_per_s": best["steps"] / (best["kernel_ms"] / 1e3),
                "rays_per_s": best["rays"] / (best["kernel_ms"] / 1e3)}

    def cpu(grid, kd, T, x, rays, seed, tol, box, threads):
        t0 = time.perf_counter()
        r = oracle.solve(grid, kd, T, x, rays=rays, seed=seed, tol=tol, max_steps=1 << 20, box=box,
                         nthreads=threads)
        dt = time.perf_counter() - t0
        steps = float(np.asarray(r["steps"]).sum())
        return {"steps_per_s": steps / dt, "s": dt, "box": list(box) if box else None}

    # grey slab (E3 case)
    grid, kd, T, x = inputs.grey_slab_16x32x16(1.0)
    k64, k32 = [], []
    out["grey_slab_16x32x16_128rays"] = {
        "gpu_fp64": gpu(grid, kd, T, x, 128, mcrt.MCRT_FP64, 0, 1e-6, keep=k64),
        "gpu_fp32": gpu(grid, kd, T, x, 128, mcrt.MCRT_FP32, 0, 1e-6, keep=k32),
        "oracle_all_cores": cpu(grid, kd, T, x, 128, 0, 1e-6, None, allc),
        "oracle_1_core": cpu(grid, kd, T, x, 128, 0, 1e-6, (0, 16, 0, 32, 0, 2), 1)}
    out["grey_slab_16x32x16_128rays"]["error_vs_oracle"] = field_error(
        grid, kd, T, x, 128, 0, {"fp64": k64[0], "fp32": k32[0]}, tol=1e-6)
    # 64^3 channel, one core (the all-core figure is the main line's cpu_baseline)
    grid, kd, T, x = inputs.nongrey_channel(64, 64, 64, seed=0)
    out["nongrey_channel_64x64x64_1000rays"] = {
        "oracle_1_core": cpu(grid, kd, T, x, 1000, 0, 1e-4, (0, 64, 0, 64, 0, 1), 1)}
    # DNS-size field
    grid, kd, T, x = inputs.nongrey_channel(256, 192, 128, seed=3, eps_wall=0.8, x_mode="field")
    kept = []
    out["dns_256x192x128_512rays_grey_walls"] = {
        "gpu_fp32": gpu(grid, kd, T, x, 512, mcrt.MCRT_FP32, 0, 1e-4, reps=1, keep=kept),
        "oracle_all_cores": cpu(grid, kd, T, x, 512, 0, 1e-4, (112, 144, 80, 112, 48, 56), allc),
        "oracle_1_core": cpu(grid, kd, T, x, 512, 0, 1e-4, (112, 144, 80, 112, 48, 49), 1)}
    # the central 32^3 crop against the oracle, rays through the whole field
    out["dns_256x192x128_512rays_grey_walls"]["error_vs_oracle_32cubed_crop"] = field_error(
        grid, kd, T, x, 512, 0, {"fp32": kept[0]}, box=(112, 144, 80, 112, 48, 80),
        crop=(slice(48, 80), slice(80, 112), slice(112, 144)))
    return out


def batch_extra(sp, rays=256, n=32, seed=0):
    """32 snapshots of uneven grid sizes (32^3, 48x64x48, 96^3, 128^3), 256 rays
    per cell, sharing the k-distribution, in one graph launch.  The tuner picks
    the form (a single persistent trace kernel over all snapshots and one
    reduction, or per-snapshot launches in 1, 2, 4 or 8 graph branches, with the
    default or a 1 GiB cap of each snapshot's sample scratch: a 128^3 snapshot then
    runs as two chunks) and the launch shape (CTAs per SM, march steps per round);
    compared with the same
    snapshots solved one after another (the sum of their device times)."""
    import torch

    from paper_1810_00188_gb300 import autotune, inputs, mcrt
    kd, snaps = inputs.snapshot_batch(n, seed)
    solvers, outs, items = [], [], []
    for k, (grid, T, x) in enumerate(snaps):
        S = mcrt.Solver(grid, kd)
        S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
        q = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
        sg = torch.empty_like(q)
        solvers.append(S)
        outs.append((q, sg))
        items.append((S.ctx, q.data_ptr(), sg.data_ptr(), k))
    params = mcrt.Solver.params(rays=rays, seed=seed, precision=mcrt.MCRT_FP32)

    def make(shape):  # (CTAs per SM, steps per round, per-item launches, graph branches, scratch MiB)
        mb, k, per_item, streams, mib = shape
        solvers[0].set_tuning(mb, k, mib, batch_per_snapshot=per_item)
        return mcrt.mcrt_batch_create(items, params, streams=streams)

    def run(b):
        mcrt.mcrt_batch_run(b, rays, sp)
        return mcrt.mcrt_batch_get_stats(b)["kernel_ms"]

    shapes = ((3, 1, 0, 1, 0), (3, 2, 0, 1, 0), (2, 1, 0, 1, 0), (2, 2, 0, 1, 0), (3, 1, 1, 1, 0), (3, 1, 1, 2, 0),
              (3, 1, 1, 4, 0), (3, 1, 1, 8, 0), (3, 1, 1, 4, 1024), (3, 1, 1, 8, 1024))
    best, table = autotune.tune_batch(make, run, shapes=shapes, reps=1)
    b = make(best)
    try:
        mcrt.mcrt_batch_run(b, 0, sp)
        mcrt.mcrt_batch_get_stats(b)
        times, st = [], None
        for k in range(3):
            mcrt.mcrt_batch_run(b, (k + 1) * rays, sp)
            st = mcrt.mcrt_batch_get_stats(b)
            times.append(st["kernel_ms"])
        # the smallest snapshot of the last run against the FP64 oracle, cell by cell
        ks = min(range(n), key=lambda k: snaps[k][0].ncells)
        torch.cuda.synchronize()
        qk = outs[ks][0].cpu().numpy()
    finally:
        mcrt.mcrt_batch_destroy(b)
    solvers[0].set_tuning()
    seq = 0.0
    for S, (q, sg) in zip(solvers, outs):
        S.solve_into(S.params(rays=rays, seed=seed, ray_offset=rays, precision=mcrt.MCRT_FP32), q, sg,
                     stream=sp)
        seq += S.stats()["kernel_ms"]
    for S in solvers:
        S.close()
    t = statistics.median(times) / 1e3
    cells = sum(g.ncells for g, _, _ in snaps)
    return {"workload": f"{n} snapshots {{32^3, 48x64x48, 96^3, 128^3}}, {rays} rays/cell",
            "cells": cells, "graph_ms": t * 1e3, "rays_per_s": cells * rays / t,
            "steps_per_s": st["steps"] / t, "launches_in_graph": st["launches"],
            "sequential_ms": seq, "speedup_vs_sequential": seq / (t * 1e3),
            "tuned": {"min_blocks_per_sm": best[0], "steps_per_round": best[1],
                      "form": "per-item launches" if best[2] else "one persistent launch",
                      "graph_branches": best[3], "scratch_mib": best[4] or "default"},
            "tuning_ms": {(f"{k[0]}x{k[1]} per-item x{k[3]}" if k[2] else f"{k[0]}x{k[1]} one launch")
                          + (f" scratch {k[4]} MiB" if k[4] else ""): v for k, v in table.items()},
            "error_vs_oracle": dict(field_error(snaps[ks][0], kd, snaps[ks][1], snaps[ks][2], rays, ks,
                                                {"fp32": qk}, ray_offset=3 * rays, max_steps=1 << 30),
                                    snapshot=ks, grid=list(snaps[ks][0].shape))}


# The paper's own timing table (64^3 cells, 6e4 rays per cell, 119 narrow bands x
# 16 g-points, one Tesla K40M; Section 6): seconds per solve, context only
PAPER_64CUBED_6E4_S = {"gpu_nb_sorting_exact": 573.0, "gpu_optimized_multigrid": 132.8, "cpu_serial": 39313.3}


def paper_scale_extra(sp, rays=60000, scratch_mib=0):
    """The size of the paper's timing runs, on synthetic inputs of that shape: a
    64^3 slab of 1 m between black walls at 400 K, periodic in x and z, a
    parabolic temperature profile (400 K at the walls, 1400 K at mid-height) with
    a 5% random part, 119 bands x 16 g-points of synthetic correlated-k tables,
    6e4 rays per cell (1.57e10 rays: the sample scratch runs in chunks).  The
    exact FP32 march and the multigrid march (5 grids, 5 segments per grid, the
    paper's optimized setting), one solve each, beside the paper's K40M times for
    the same sizes (context, another machine and other spectra).  scratch_mib 0:
    the library's default cap of the sample scratch (the solve runs in chunks)."""
    import numpy as np
    import torch

    from paper_1810_00188_gb300 import inputs, mcrt
    kd = inputs.make_kdist(seed=7, n_bands=119, n_g=16, nT=80, nu0_cm=150.0, dnu_cm=25.0)  # 300..1880 K
    grid = inputs.Grid(64, 64, 64, 1.0, 1.0, 1.0, T_wall=(400.0, 400.0))
    yc = (np.arange(64) + 0.5) / 64.0
    prof = 400.0 + 1000.0 * 4.0 * yc * (1.0 - yc)
    G = inputs.gaussian_random_field(grid.shape, (grid.lz, grid.ly, grid.lx), 11)
    T = np.ascontiguousarray(prof[None, :, None] * (1.0 + 0.05 * np.clip(G, -4.0, 4.0)))
    x = np.full(grid.shape, kd.x_ref)
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    S.set_tuning(scratch_mib=scratch_mib)
    q = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
    sg = torch.empty_like(q)
    out = {"scratch_mib": S.tuning()["scratch_mib"], "workload": "64^3 slab 1 m, 119 x 16 k-distribution (synthetic), 6e4 rays/cell, black walls 400 K, "
                       "parabolic T 400 -> 1400 K",
           "paper_k40m_s": PAPER_64CUBED_6E4_S}
    for name, mg in (("exact", 1), ("multigrid", 5)):
        S.solve_into(S.params(rays=256, seed=0, precision=mcrt.MCRT_FP32, mg_levels=mg, mg_steps=5), q, sg,
                     stream=sp)  # warm-up
        S.solve_into(S.params(rays=rays, seed=0, ray_offset=256, precision=mcrt.MCRT_FP32, mg_levels=mg,
                              mg_steps=5), q, sg, stream=sp)
        st = S.stats()
        out[name] = {"s": st["kernel_ms"] / 1e3, "steps": st["steps"], "rays": st["rays"],
                     "steps_per_s": st["steps"] / (st["kernel_ms"] / 1e3), "launches": st["launches"],
                     "trace_ms": st["trace_ms"], "long_rays_ms": st["long_ms"], "reduce_ms": st["reduce_ms"],
                     "rays_handed_off": st["long_rays"]}
    S.close()
    out["speedup_vs_paper"] = {"exact_vs_nb_sorting": PAPER_64CUBED_6E4_S["gpu_nb_sorting_exact"] / out["exact"]["s"],
                               "multigrid_vs_optimized": PAPER_64CUBED_6E4_S["gpu_optimized_multigrid"]
                               / out["multigrid"]["s"]}
    return out


def multigrid_extra(S, params, q, s, sp, rays, steps_per_grid=5):
    """The multigrid march (Section 4.3) on the benchmark workload: every grid
    the field allows, `steps_per_grid` segments per grid; time against the
    exact march on the same draws, and the paired difference of the two
    estimates (an approximation, so its bias is reported, not hidden)."""
    import numpy as np

    from paper_1810_00188_gb300 import mcrt
    g = S.grid
    L = mcrt.mcrt_multigrid_levels(g.nx, g.ny, g.nz)
    out = {"grids": L, "steps_per_grid": steps_per_grid}
    res = {}
    for name, lv in (("exact", 1), ("multigrid", L)):
        ts = []
        for k in range(3):
            S.solve_into(params(k, rays=rays, mg_levels=lv, mg_steps=steps_per_grid), q, s, stream=sp)
            st = S.stats()
            ts.append(st["kernel_ms"])
        res[name] = (q.cpu().numpy(), s.cpu().numpy(), statistics.median(ts), st)
        out[name] = {"kernel_ms": statistics.median(ts), "steps_per_ray": st["steps"] / st["rays"],
                     "max_ray_steps": st["max_ray_steps"]}
    q0, s0, _, _ = res["exact"]
    q1, s1, _, _ = res["multigrid"]
    d = q1 - q0
    out["speedup"] = out["exact"]["kernel_ms"] / out["multigrid"]["kernel_ms"]
    out["paired_rel_l1_diff"] = float(np.abs(d).sum() / np.abs(q0).sum())
    out["mean_diff_over_mean_abs_q"] = float(d.mean() / np.abs(q0).mean())
    out["frac_cells_beyond_3_sigma"] = float(np.mean(np.abs(d) > 3 * np.sqrt(s0**2 + s1**2)))
    return out


def spectral_extra(S, T, params, q, s, sp, rays=256, reps=3):
    """Spectral proposals on the benchmark field: Zhang's T_max pdf (the
    paper's, Eq. 13), the classic ERMC pdf at each cell's own temperature, and
    their temperature-weighted mix.  For each: kernel time, p95 relative sigma
    over cells, median relative sigma in the coldest and hottest tenths of the
    cells, and the projected GPU time to 1% p95 relative sigma."""
    import numpy as np

    from paper_1810_00188_gb300 import mcrt
    Tf = np.asarray(T).reshape(-1)
    cold = Tf <= np.percentile(Tf, 10)
    hot = Tf >= np.percentile(Tf, 90)
    out = {"rays_per_cell": rays}
    for name, mode in (("T_max", None), ("local", mcrt.MCRT_SPECTRAL_LOCAL),
                       ("hybrid", mcrt.MCRT_SPECTRAL_HYBRID)):
        prop = mcrt.MCRT_PROPOSAL_PLANCK_TMAX
        if mode is not None:
            S.set_spectral_proposal(mode, stream=sp)
            prop = mcrt.MCRT_PROPOSAL_CELL
        ts, p95, rc, rh = [], [], [], []
        for k in range(reps):
            pk = params(k, rays=rays)
            pk.proposal = prop
            S.solve_into(pk, q, s, stream=sp)
            ts.append(S.stats()["kernel_ms"])
            qn, sn = q.cpu().numpy().reshape(-1), s.cpu().numpy().reshape(-1)
            rel = sn / np.maximum(np.abs(qn), 0.05 * np.mean(np.abs(qn)))
            p95.append(float(np.percentile(rel, 95)))
            rc.append(float(np.median(rel[cold])))
            rh.append(float(np.median(rel[hot])))
        t, pr = statistics.median(ts), statistics.median(p95)
        out[name] = {"kernel_ms": t, "p95_rel_sigma": pr, "cold_median_rel_sigma": statistics.median(rc),
                     "hot_median_rel_sigma": statistics.median(rh), "ms_to_1pct": t * (pr / 0.01) ** 2}
    for name in ("local", "hybrid"):
        out[name]["speedup_vs_T_max"] = out["T_max"]["ms_to_1pct"] / out[name]["ms_to_1pct"]
    return out


def estimators_extra(S, T, params, q, s, sp, rays=256, reps=3):
    """The reciprocal estimators of Section 2 on the benchmark field, all at the
    same rays per cell: the emission-based estimate with Zhang's T_max pdf (the
    paper's), with each cell's own emission spectrum (classic ERMC), the
    absorption-based estimate (ARMC, T_max pdf), and their temperature-weighted
    combination.  For each: kernel time, and over cells the p95 relative sigma and
    the median relative sigma of the coldest and hottest tenths."""
    import numpy as np

    from paper_1810_00188_gb300 import mcrt
    Tf = np.asarray(T).reshape(-1)
    cold = Tf <= np.percentile(Tf, 10)
    hot = Tf >= np.percentile(Tf, 90)
    out = {"rays_per_cell": rays,
           "criterion": "relative sigma_i / max(|Q_i|, 0.05 mean |Q|); ARMC and hybrid sigma from batch means"}
    arms = (("ermc_T_max", mcrt.MCRT_EST_ERMC, None), ("ermc_local", mcrt.MCRT_EST_ERMC, mcrt.MCRT_SPECTRAL_LOCAL),
            ("armc_T_max", mcrt.MCRT_EST_ARMC, None), ("hybrid_T_max", mcrt.MCRT_EST_HYBRID, None))
    for name, est, spec in arms:
        prop = mcrt.MCRT_PROPOSAL_PLANCK_TMAX
        if spec is not None:
            S.set_spectral_proposal(spec, stream=sp)
            prop = mcrt.MCRT_PROPOSAL_CELL
        ts, p95, rc, rh = [], [], [], []
        for k in range(reps):
            pk = params(k, rays=rays)
            pk.proposal = prop
            pk.estimator = est
            S.solve_into(pk, q, s, stream=sp)
            ts.append(S.stats()["kernel_ms"])
            qn, sn = q.cpu().numpy().reshape(-1), s.cpu().numpy().reshape(-1)
            rel = sn / np.maximum(np.abs(qn), 0.05 * np.mean(np.abs(qn)))
            p95.append(float(np.percentile(rel, 95)))
            rc.append(float(np.median(rel[cold])))
            rh.append(float(np.median(rel[hot])))
        out[name] = {"kernel_ms": statistics.median(ts), "p95_rel_sigma": statistics.median(p95),
                     "cold_tenth_median_rel_sigma": statistics.median(rc),
                     "hot_tenth_median_rel_sigma": statistics.median(rh)}
    base = out["ermc_T_max"]["cold_tenth_median_rel_sigma"]
    for name, _, _ in arms:
        out[name]["cold_sigma_vs_ermc_T_max"] = out[name]["cold_tenth_median_rel_sigma"] / base
    return out


def learned_extra(sp, n_train=200, train_grid=64, eval_grid=128, rays_tally=512, rays_eval=256,
                  steps=1500, seed=0, eval_seeds=(1000, 1001, 1002)):
    """Learned proposal: tallies of `n_train` seeded 64^3 fields, training on the
    GPU, then plain and learned FP32 solves of held-out 128^3 fields (seeds
    1000-1002) given the SAME measured GPU time: the plain arm runs 256 rays per
    cell, the learned arm the ray count that fills the same kernel time (from a
    pilot solve); both arms' achieved p95 relative sigma is measured.  Two forms,
    each against plain sampling on the same march: the multigrid march (every
    grid, 5 segments per grid; tallies from multigrid solves, cost constant
    c0 = 12 steps) and the exact march (tallies from exact solves, c0 = 3)."""
    import torch

    from paper_1810_00188_gb300 import inputs, learn, mcrt
    n = eval_grid
    out = {"workload": f"train {n_train} x {train_grid}^3 fields (4096 cells each, {rays_tally} rays), "
                       f"held-out {n}^3 fields (seeds {', '.join(map(str, eval_seeds))}); plain arm "
                       f"{rays_eval} rays/cell, learned arm the rays that fill the same GPU time",
           "criterion": "p95 over cells of sigma_i / max(|Q_i|, 0.05 mean |Q|), measured at equal "
                        "kernel time (no projection)"}
    fields = []
    for sd in eval_seeds:
        grid, kd, T, x = inputs.nongrey_channel(n, n, n, seed=sd, x_mode="field")
        fields.append((sd, grid, kd, T, x))
    for name, mg, c0 in (("multigrid", 1, 12.0), ("exact", 0, 3.0)):
        t0 = time.perf_counter()
        ds = learn.build_dataset(grid_shape=(train_grid,) * 3, seeds=range(n_train), rays=rays_tally,
                                 cells_per_field=4096, stream=sp, mg=mg)
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t0
        net = mcrt.Mlp(ds.K)
        mean, inv = learn.feature_norm(ds)
        net.set_params(learn.init_theta(ds.K, ds.p0.mean(0).cpu().numpy(), seed=seed), mean, inv)
        l0 = learn.mean_loss(net, ds, c0=c0, stream=sp)
        t0 = time.perf_counter()
        losses = learn.train(net, ds, steps=steps, c0=c0, stream=sp, seed=seed)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        l1 = learn.mean_loss(net, ds, c0=c0, stream=sp)
        del ds
        torch.cuda.empty_cache()
        L = mcrt.mcrt_multigrid_levels(n, n, n) if mg else 1
        per_seed = {}
        for sd, grid, kd, T, x in fields:
            S = mcrt.Solver(grid, kd)
            S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"), stream=sp)
            per_seed[str(sd)] = learn.compare_equal_budget(S, net, rays=rays_eval, seed=seed + 7, stream=sp,
                                                           mg_levels=L, mg_steps=5)
            S.close()
        net.close()
        ratios = [v["p95_sigma_ratio_plain_over_learned"] for v in per_seed.values()]
        out[name] = {"grids": L, "c0": c0, "dataset_s": t_data, "train_s": t_train, "train_steps": steps,
                     "loss_before": l0, "loss_after": l1, "loss_last_batch": losses[-1][1],
                     "fields": per_seed,
                     "p95_sigma_ratio_plain_over_learned": {"min": min(ratios), "median": statistics.median(ratios),
                                                            "max": max(ratios)}}
    return out


def solves_at_1pct(sp):
    """Q_rad solves per second at 1% cell sigma (the p95 over cells of
    sigma_i / max(|Q_i|, 0.05 mean |Q|) at most 1%), MEASURED where one solve can
    reach it: the grey slab 16x32x16 (kappa = 0.1, 1, 10; T = 1000 K, cold black
    walls; FP32 and FP64): from a 128-ray solve the rays N* that the 1/N law asks
    for are run, the achieved p95 is checked, and N* is raised until it holds.
    For the non-grey 32^3 channel the p95 curve is measured up to 65,536 rays per
    cell (2.1e9 rays in one solve); N* lies beyond one solve there and its
    projection from the largest measured point is labelled as one."""
    import numpy as np
    import torch

    from paper_1810_00188_gb300 import inputs, learn, mcrt
    out = {"criterion": "p95 over cells of sigma_i / max(|Q_i|, 0.05 mean |Q|) <= 0.01"}

    def solve(S, rays, prec, q, s, tol):
        S.solve_into(S.params(rays=rays, seed=0, tol=tol, max_steps=1 << 20, precision=prec), q, s, stream=sp)
        st = S.stats()
        return st["kernel_ms"], learn.rel_sigma_p95(q.cpu().numpy(), s.cpu().numpy())

    for kap in (0.1, 1.0, 10.0):
        grid, kd, T, x = inputs.grey_slab_16x32x16(kap)
        S = mcrt.Solver(grid, kd)
        S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"), stream=sp)
        q = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
        s = torch.empty_like(q)
        for prec, pname in ((mcrt.MCRT_FP32, "fp32"), (mcrt.MCRT_FP64, "fp64")):
            _, p0 = solve(S, 128, prec, q, s, 1e-6)
            n = int(math.ceil(128 * (p0 / 0.01) ** 2))
            tries = []
            for _ in range(4):
                if prec == mcrt.MCRT_FP32:
                    solve(S, n, prec, q, s, 1e-6)  # warm-up at this size (scratch allocation)
                ms, pn = solve(S, n, prec, q, s, 1e-6)
                tries.append({"rays": n, "kernel_ms": ms, "p95_rel_sigma": pn})
                if pn <= 0.01:
                    break
                n = int(math.ceil(n * (pn / 0.01) ** 2 * 1.02))
            last = tries[-1]
            out[f"grey_slab_16x32x16_kappa{kap:g}_{pname}"] = {
                "p95_rel_sigma_at_128_rays": p0, "rays_needed": last["rays"], "tries": tries,
                "verified": last["p95_rel_sigma"] <= 0.01, "solve_ms": last["kernel_ms"],
                "solves_per_s": 1e3 / last["kernel_ms"], "measured": True}
        S.close()
    # non-grey 32^3 channel: the curve
    grid, kd, T, x = inputs.nongrey_channel(32, 32, 32, seed=0)
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"), stream=sp)
    q = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
    s = torch.empty_like(q)
    curve = []
    for rays in (1000, 4000, 16000, 65536):
        ms, pn = solve(S, rays, mcrt.MCRT_FP32, q, s, 1e-4)
        curve.append({"rays": rays, "kernel_ms": ms, "p95_rel_sigma": pn,
                      "rays_needed_by_1_over_N_from_here": int(math.ceil(rays * (pn / 0.01) ** 2))})
    S.close()
    big = curve[-1]
    out["nongrey_channel_32cubed_fp32"] = {
        "curve": curve, "measured": False,
        "projected": {"from_rays": big["rays"], "rays_needed": big["rays_needed_by_1_over_N_from_here"],
                      "solve_s": big["kernel_ms"] / 1e3 * big["rays_needed_by_1_over_N_from_here"] / big["rays"],
                      "note": "projection with the 1/N law from the largest measured ray count; the measured "
                              "curve falls more slowly than the law between 1,000 and 16,000 rays"}}
    return out


def parallelism(a, world):
    if a.scaling == "strong" and world > 1:
        return f"strong: one snapshot in {world} z-slabs, field broadcast once, Q/sigma gathered each step"
    return f"weak: one snapshot per rank ({world}), no data-path collective"


def launch_ranks(a):
    """With --gpus N > 1 outside a launcher, start N ranks on this node (one per
    GPU) with torch's launcher and return its exit status; under a launcher, the
    world size must equal --gpus."""
    world = int(os.environ.get("WORLD_SIZE", "0") or 0)
    if world == 0 and a.gpus > 1:
        import socket
        with socket.socket() as so:
            so.bind(("127.0.0.1", 0))
            port = so.getsockname()[1]
        env = dict(os.environ)
        env.setdefault("NCCL_DEBUG", "INFO")
        env.setdefault("NCCL_DEBUG_SUBSYS", "INIT")
        # "--n" would read as an abbreviation of the launcher's own options
        args = ["--grid" if v == "--n" else v for v in sys.argv[1:]]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={a.gpus}",
               "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *args]
        return subprocess.call(cmd, env=env)
    if world and world != a.gpus:
        raise SystemExit(f"bench.py: --gpus {a.gpus} but the launcher started {world} ranks")
    return None


def run_reference(a):
    """Reference arm: the FP64 CPU oracle, timed as it stands on the host cores
    (rank 0 only; other ranks exit without work)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1") or 1)
    if rank != 0:
        return
    import oracle
    from paper_1810_00188_gb300 import inputs
    grid, kd, T, x = inputs.nongrey_channel(a.n, a.n, a.n, seed=0)
    threads = oracle.default_threads()

    def one(k):
        z = k % a.n
        t0 = time.perf_counter()
        r = oracle.solve(grid, kd, T, x, rays=a.rays, seed=0, tol=1e-4, max_steps=1 << 20,
                         box=(0, a.n, 0, a.n, z, z + 1), nthreads=threads, ray_offset=0)
        return float(r["steps"].sum()), time.perf_counter() - t0

    for k in range(a.warmup):
        one(k)
    tot_s, tot_t = 0.0, 0.0
    for k in range(a.steps):
        s, t = one(a.warmup + k)
        tot_s += s
        tot_t += t
    v = tot_s / tot_t
    cfg = workload_config(a)
    cfg["parallelism"] = parallelism(a, world)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot_t / a.steps,
            "higher_is_better": True, "scaling": a.scaling, "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"one z-plane ({a.n}x{a.n} cells) x {a.rays} rays per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    rc = launch_ranks(a)
    if rc is not None:
        sys.exit(rc)
    if a.impl == "reference":
        run_reference(a)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1810_00188_gb300 import dist as pdist
    from paper_1810_00188_gb300 import inputs, mcrt

    world = int(os.environ.get("WORLD_SIZE", "1") or 1)
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        os.environ.setdefault("NCCL_DEBUG", "INFO")
        os.environ.setdefault("NCCL_DEBUG_SUBSYS", "INIT")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    strong = a.scaling == "strong" and world > 1
    snap = 0 if a.scaling == "strong" else rank
    grid, kd, T, x = inputs.nongrey_channel(a.n, a.n, a.n, seed=snap)
    S = mcrt.Solver(grid, kd, device=local)
    if a.long_ray_steps or a.long_ray_flight:
        S.set_tuning(long_ray_steps=a.long_ray_steps, long_ray_flight=a.long_ray_flight)
    Td = torch.tensor(T, device="cuda")
    xd = torch.tensor(x, device="cuda")
    boxes = pdist.shard_boxes(grid.nx, grid.ny, grid.nz, world)
    box = boxes[rank] if strong else None
    if strong:
        if rank != 0:
            Td.zero_()
            xd.zero_()
        pdist.broadcast_fields(Td, xd, src=0)  # rank 0's field on every rank
    S.set_fields(Td, xd)
    q = torch.empty(S.box_shape(box), dtype=torch.float64, device="cuda")
    s = torch.empty_like(q)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def params(k, prec=mcrt.MCRT_FP32, rays=a.rays, mg_levels=1, mg_steps=5):
        return S.params(rays=rays, seed=0, snapshot=snap, ray_offset=k * rays, tol=1e-4,
                        max_steps=1 << 20, precision=prec, mg_levels=mg_levels, mg_steps=mg_steps,
                        box=box)

    for k in range(a.warmup):
        S.solve_into(params(k), q, s, stream=sp)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    steps_total, kern_ms, trace_ms, long_ms, red_ms, launches = 0, [], [], [], [], 0
    for k in range(a.steps):
        flush.zero_()
        ev[k][0].record(stream)
        S.solve_into(params(a.warmup + k), q, s, stream=sp)
        if strong:
            pdist.gather_slabs([q, s], boxes, grid.shape, dst=0)
        ev[k][1].record(stream)
        st = S.stats()  # waits for this solve
        steps_total += st["steps"]
        kern_ms.append(st["kernel_ms"])
        trace_ms.append(st["trace_ms"])
        long_ms.append(st["long_ms"])
        red_ms.append(st["reduce_ms"])
        launches += st["launches"]
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    t_local = sum(step_ms) / 1e3
    steps_all, t_max = pdist.aggregate(float(steps_total), t_local, device="cuda")
    value = steps_all / t_max
    rays_all = float((1 if strong else world) * a.steps) * grid.ncells * a.rays

    result = None
    if rank == 0:
        peaks = measured_peaks()
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        nsm = sm_count(local)
        alu_peak = nsm * LANES_PER_SM * sm_max * 1e6        # op/s
        hbm = float(peaks.get("hbm_gbs", 6800.0)) * 1e9       # B/s
        hbm_note = "of measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "of fallback (6.8 TB/s)"
        trace_s = statistics.mean(trace_ms) / 1e3             # the trace kernel alone, CUDA events
        steps_per_launch = steps_total / a.steps
        bs = S.box_shape(box)
        rays_per_launch = bs[0] * bs[1] * bs[2] * a.rays
        steps_rate = steps_per_launch / trace_s
        gather = steps_rate * GATHER_BYTES_PER_STEP            # algorithmic B/s of the trace kernel
        c = ceilings(local, grid.ncells * 8, full=not a.no_extras)
        ex2 = c["ex2_per_s"]
        l2g = c["gather8_per_s"]["field"] * GATHER_BYTES_PER_STEP  # useful B/s of random 8-B gathers
        hbm_bound = hbm / GATHER_BYTES_PER_STEP
        exp_bound = ex2 / EXP_PER_STEP
        ops = OPS_PER_STEP * steps_per_launch + OPS_PER_RAY * rays_per_launch
        result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                  "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t_max / a.steps,
                  "higher_is_better": True, "scaling": a.scaling, "vs_baseline": None,
                  "dtype": "f32", "data": "synthetic", "config": workload_config(a),
                  "rays_per_s": rays_all / t_max,
                  "steps_per_ray": steps_total / (a.steps * rays_per_launch),
                  "roofline": {
                      "kernel": "trace_fp32_kernel",
                      "bound": "hbm" if hbm_bound <= exp_bound else "mufu",
                      "achieved": gather / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                      "frac": gather / hbm, "peak_basis": hbm_note,
                      "traffic": (TRACE_DRAM_BYTES_64_1000 if (a.n, a.rays) == (64, 1000) else None),
                      "traffic_note": "dram read+write bytes of one trace launch (ncu) of the kernel as it "
                                      "stands, else null; the kernel writes 4 B per ray of samples",
                      "definition": "steps/s <= min(bytes/s of the level holding the field / 8 B per step, "
                                    "ex2/s / 1 exp per step); achieved = 8 B x steps per launch / the trace "
                                    "kernel's mean CUDA-event time in the timed region",
                      "trace_kernel_ms": trace_s * 1e3, "steps_per_s_trace_kernel": steps_rate,
                      "l2_gather": {"peak": l2g / 1e9, "unit": "GB/s", "frac": gather / l2g,
                                    "basis": "the library's random 8-byte gather probe on a buffer of the "
                                             "field's size (the field is L2-resident), useful bytes"},
                      "mufu": {"peak_ex2_per_s": ex2, "frac": steps_rate * EXP_PER_STEP / ex2,
                               "basis": "the library's ex2.approx probe"},
                      "alu": {"achieved": ops / trace_s / 1e12, "peak": alu_peak / 1e12, "unit": "Top/s",
                              "frac": ops / trace_s / alu_peak, "ops_per_step": OPS_PER_STEP,
                              "ops_per_ray": OPS_PER_RAY,
                              "basis": f"{nsm} SM x {LANES_PER_SM} lanes x {sm_max:.0f} MHz, 1 op/lane/clk"}},
                  "kernel_ms": {"solve": statistics.mean(kern_ms), "trace": statistics.mean(trace_ms),
                                "long_rays": statistics.mean(long_ms), "reduce": statistics.mean(red_ms)},
                  "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms),
                              "max": max(step_ms)},
                  "ceilings": c, "gpu_launches": launches, "clocks": clk}
        result["config"]["parallelism"] = parallelism(a, world)
    # --- extras on rank 0: e2e through host buffers, FP64, solves/s at 1% sigma
    if rank == 0:
        Tp = torch.tensor(T).pin_memory()
        xp = torch.tensor(x).pin_memory()
        qh = torch.empty(S.box_shape(box), dtype=torch.float64).pin_memory()
        sh = torch.empty_like(qh).pin_memory()
        ke = max(1, min(a.steps, 5))
        torch.cuda.synchronize()
        e_steps, t0 = 0, time.perf_counter()
        for k in range(ke):
            S.set_fields(Tp.numpy(), xp.numpy())
            S.solve_into(params(a.warmup + k), qh.numpy(), sh.numpy())
            e_steps += S.stats()["steps"]
        te = time.perf_counter() - t0
        result["e2e"] = {"value": e_steps / te, "unit": UNIT,
                         "scope": "rank 0's slab" if strong else "rank 0's snapshot",
                         "h2d_bytes_per_step": int(Tp.numel() * 8 + xp.numel() * 8),
                         "d2h_bytes_per_step": int(qh.numel() * 8 + sh.numel() * 8)}
        if not a.no_extras and not strong:
            S.set_fields(Td, xd)
            # FP64 traversal throughput on a tenth of the rays
            r64 = max(32, a.rays // 10)
            S.solve_into(params(0, mcrt.MCRT_FP64, r64), q, s, stream=sp)
            st = S.stats()
            result["fp64_steps_per_s"] = st["steps"] / (st["kernel_ms"] / 1e3)
            # per-field error of both precisions against the FP64 oracle, draw for draw
            # (the same rays; |dQ| / S_i with S_i the oracle's mean absolute tally)
            q64 = q.cpu().numpy()
            S.solve_into(params(0, mcrt.MCRT_FP32, r64), q, s, stream=sp)
            q32 = q.cpu().numpy()
            result["error_vs_oracle"] = field_error(grid, kd, T, x, r64, snap, {"fp64": q64, "fp32": q32})
            # Q_rad solves/s at 1% cell sigma on this workload: the p95 curve to 16x the
            # base rays (the 1/N law's N* is out of reach of one solve here)
            curve = []
            for m in (1, 4, 16):
                S.solve_into(params(0, rays=m * a.rays), q, s, stream=sp)
                st = S.stats()
                qn, sn = q.cpu().numpy(), s.cpu().numpy()
                ref = np.maximum(np.abs(qn), 0.05 * np.mean(np.abs(qn)))
                pm = float(np.percentile(sn / ref, 95))
                curve.append({"rays": m * a.rays, "p95_rel_sigma": pm, "kernel_ms": st["kernel_ms"],
                              "rays_needed_by_1_over_N_from_here": int(math.ceil(m * a.rays * (pm / 0.01) ** 2))})
            big = curve[-1]
            sol = {"this_workload": {
                "curve": curve, "measured": False,
                "projected": {"from_rays": big["rays"], "rays_needed": big["rays_needed_by_1_over_N_from_here"],
                              "solves_per_s": 1e3 / (big["kernel_ms"] * big["rays_needed_by_1_over_N_from_here"]
                                                     / big["rays"]),
                              "note": "1/N-law projection from the largest measured ray count, labelled as one"}}}
            sol.update(solves_at_1pct(sp))
            result["qrad_solves_per_s_at_1pct_sigma"] = sol
            result["multigrid"] = multigrid_extra(S, params, q, s, sp, a.rays)
            result["spectral_proposals"] = spectral_extra(S, T, params, q, s, sp)
            result["estimators"] = estimators_extra(S, T, params, q, s, sp)
            if world == 1:
                result["configs"] = configs_extra(sp)
                result["paper_scale"] = paper_scale_extra(sp)
                # before the learned-proposal leg, whose datasets stay in torch's cache
                result["batched_snapshots"] = batch_extra(sp)
                torch.cuda.empty_cache()
            result["learned_vs_plain"] = learned_extra(sp)
        if not a.no_cpu_baseline and world == 1:
            result["cpu_baseline"] = cpu_baseline(a)
        print(json.dumps(result), flush=True)
    barrier()
    S.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
