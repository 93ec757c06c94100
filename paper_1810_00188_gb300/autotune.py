"""Autotuner of the FP32 solve's launch shape and of batch partitions.

The knobs are the library's `mcrt_tuning` (CTAs per SM, march steps per refill
round, sample-scratch cap: the ray batch of one launch, rays per claimed run of
cells: the work tile) and, for batches, the form (one persistent launch or
per-snapshot launches), the launch shape, the number of concurrent graph
branches and the share of the GPU's persistent CTAs given to each snapshot.  Q, sigma and the step counts are bitwise
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
CLAIM_RAYS = (1024, 4096, 16384)


def _set(S, key, keep):
    """Applies the knobs key = (CTAs per SM, steps per round, scratch MiB, claim
    rays; 0: the library default), keeping the other tuning fields as set."""
    mb, k, mib, claim = key
    S.set_tuning(mb, k, mib, keep["long_ray_steps"], keep["long_ray_flight"], keep["tally_binary32"],
                 tally_plain_loads=keep["tally_plain_loads"],
                 batch_per_snapshot=keep["batch_per_snapshot"], claim_rays=claim)


def tune_solver(S, params, q, s, stream=0, shapes=SHAPES, reps=3, scratch_mib=None, claim_rays=None):
    """Coordinate search on S: each (CTAs per SM, steps per round) of `shapes`;
    then, at the fastest, each cap of the per-ray sample scratch in MiB (the ray
    batch of one launch: a smaller cap runs the solve in more chunks); then each
    number of rays per run of cells a warp claims (the work tile).  The long-ray
    thresholds, the tally precision and the batch form are part of the
    estimator's arithmetic or of batches, not knobs here: they are kept as set.
    Keys are (mb, k, mib, claim) with 0 for a default; returns (best key,
    {key: ms}) and leaves S tuned to the best key."""
    keep = S.tuning()
    table = {}

    def trial(key):
        _set(S, key, keep)
        time_solve(S, params, q, s, stream, reps=1)  # the first launch configures the variant
        table[key] = time_solve(S, params, q, s, stream, reps)

    for mb, k in shapes:
        trial((mb, k, 0, 0))
    best = min(table, key=table.get)
    for mib in scratch_mib or ():
        trial((best[0], best[1], mib, 0))
    best = min(table, key=table.get)
    for claim in claim_rays or ():
        trial((best[0], best[1], best[2], claim))
    best = min(table, key=table.get)
    _set(S, best, keep)
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
