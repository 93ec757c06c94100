"""Autotuner of the FP32 solve's launch shape and of batch partitions.

The knobs are the library's `mcrt_tuning` (CTAs per SM, march steps per refill
round, sample-scratch cap: the ray batch of one launch) and, for batches, the
launch shape, the number of concurrent graph branches and the share of the
GPU's persistent CTAs given to each snapshot.  Q, sigma and the step counts are bitwise
independent of all of them (every cell's samples are reduced in a fixed order),
so the tuner only measures time: the library's own CUDA events around each
solve's launches.
"""
from __future__ import annotations

import statistics

from . import mcrt

SHAPES = ((2, 1), (2, 2), (3, 1), (3, 2), (4, 2))


def time_solve(S, params, q, s, stream=0, reps=3):
    """Median device time [ms] of `reps` solves into device buffers q, s."""
    times = []
    for _ in range(reps):
        S.solve_into(params, q, s, stream=stream)
        times.append(S.stats()["kernel_ms"])
    return statistics.median(times)


SCRATCH_MIB = (256, 1024, 4096)


def tune_solver(S, params, q, s, stream=0, shapes=SHAPES, reps=3, scratch_mib=None):
    """Tries each (CTAs per SM, steps per round), then, at the fastest, each cap of
    the per-ray sample scratch in MiB (the ray batch of one launch: a smaller cap
    runs the solve in more chunks), and keeps the fastest on S.  The long-ray
    thresholds and the tally precision are part of the estimator's arithmetic, not
    knobs: they are left as set.  Returns (best (mb, k) or (mb, k, mib), {knobs: ms})."""
    table = {}
    for mb, k in shapes:
        S.set_tuning(mb, k)
        time_solve(S, params, q, s, stream, reps=1)  # first launch configures the variant
        table[(mb, k)] = time_solve(S, params, q, s, stream, reps)
    best = min(table, key=table.get)
    if scratch_mib:
        base = table[best]
        for mib in scratch_mib:
            S.set_tuning(best[0], best[1], mib)
            time_solve(S, params, q, s, stream, reps=1)
            table[best + (mib,)] = time_solve(S, params, q, s, stream, reps)
        b3 = min((kk for kk in table if len(kk) == 3), key=table.get)
        if table[b3] < base:
            best = b3
    S.set_tuning(*best)
    return best, table


def batch_weights(solvers, outs, rays_probe=16, stream=0, seed=0):
    """Relative cost of each snapshot from a short probe solve (few rays per
    cell): the batch gives each snapshot a share of the persistent CTAs in
    proportion to it."""
    w = []
    for S, (q, s) in zip(solvers, outs):
        p = S.params(rays=rays_probe, seed=seed, precision=mcrt.MCRT_FP32)
        S.solve_into(p, q, s, stream=stream)
        st = S.stats()
        w.append(max(st["kernel_ms"], 1e-3))
    return w


def tune_batch(make_batch, run, shapes=SHAPES, reps=2):
    """make_batch(shape) -> batch handle built with that launch shape;
    run(batch) -> device ms.  Returns (best shape, {shape: ms})."""
    table = {}
    for shape in shapes:
        b = make_batch(shape)
        try:
            run(b)
            table[shape] = statistics.median(run(b) for _ in range(reps))
        finally:
            mcrt.mcrt_batch_destroy(b)
    best = min(table, key=table.get)
    return best, table
