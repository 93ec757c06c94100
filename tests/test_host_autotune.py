"""The autotuner's search logic on the host, against a stand-in solver whose
device time is a known function of the knobs (no GPU).

tune_solver searches (CTAs per SM, steps per round) first, then the sample
scratch cap at the best shape, then the claimed-run size, keeps the fields it
does not tune (long-ray thresholds, tally precision and reader, batch form) as
they were set, and leaves the solver on the best knobs; tune_batch builds,
times and destroys one batch per shape and returns the fastest.
"""
import pytest

from paper_1810_00188_gb300 import autotune, mcrt


class FakeSolver:
    """set_tuning / tuning / solve_into / stats with the library's defaults; the
    'device time' of a solve is a function of the current knobs."""

    DEFAULTS = {"min_blocks_per_sm": 3, "steps_per_round": 1, "scratch_mib": 4096, "long_ray_steps": 1024,
                "long_ray_flight": 32, "tally_binary32": 0, "tally_plain_loads": 0, "claim_rays": 1024,
                "batch_per_snapshot": 0}

    def __init__(self, cost):
        self.t = dict(self.DEFAULTS)
        self.cost = cost
        self.solves = 0

    def set_tuning(self, min_blocks_per_sm=0, steps_per_round=0, scratch_mib=0, long_ray_steps=0,
                   long_ray_flight=0, tally_binary32=0, batch_per_snapshot=0, claim_rays=0,
                   tally_plain_loads=0):
        d = self.DEFAULTS
        self.t = {"min_blocks_per_sm": min_blocks_per_sm or d["min_blocks_per_sm"],
                  "steps_per_round": steps_per_round or d["steps_per_round"],
                  "scratch_mib": scratch_mib or d["scratch_mib"],
                  "long_ray_steps": long_ray_steps or d["long_ray_steps"],
                  "long_ray_flight": long_ray_flight or d["long_ray_flight"],
                  "tally_binary32": tally_binary32, "tally_plain_loads": tally_plain_loads,
                  "claim_rays": claim_rays or d["claim_rays"], "batch_per_snapshot": batch_per_snapshot}

    def tuning(self):
        return dict(self.t)

    def solve_into(self, params, q, s, stream=0):
        self.solves += 1

    def stats(self):
        return {"kernel_ms": self.cost(self.t)}


def _cost(t):
    # best shape (2, 2); at that shape the 256 MiB cap is fastest; then 4096 rays per claim
    ms = 10.0 + abs(t["min_blocks_per_sm"] - 2) + abs(t["steps_per_round"] - 2)
    ms += {256: -0.5, 1024: 0.0, 4096: 0.2}.get(t["scratch_mib"], 1.0)
    ms += {1024: 0.0, 4096: -0.25, 16384: 0.1}.get(t["claim_rays"], 0.5)
    return ms


def test_tune_solver_coordinate_search_and_kept_fields():
    S = FakeSolver(_cost)
    # fields the tuner must not touch
    S.set_tuning(long_ray_steps=256, long_ray_flight=-1, tally_binary32=1, tally_plain_loads=1,
                 batch_per_snapshot=1)
    best, table = autotune.tune_solver(S, None, None, None, reps=1, scratch_mib=autotune.SCRATCH_MIB,
                                       claim_rays=autotune.CLAIM_RAYS)
    assert best == (2, 2, 256, 4096)
    assert best in table and table[best] == min(table.values())
    # every shape tried at the default scratch and claim, then the caps at the best shape,
    # then the claims at the best shape and cap
    assert {k for k in table if k[2:] == (0, 0)} == {(mb, k, 0, 0) for mb, k in autotune.SHAPES}
    assert {k[2] for k in table if k[:2] == (2, 2) and k[3] == 0} == {0, *autotune.SCRATCH_MIB}
    assert {k[3] for k in table if k[:3] == (2, 2, 256)} == {0, *autotune.CLAIM_RAYS}
    t = S.tuning()
    assert (t["min_blocks_per_sm"], t["steps_per_round"], t["scratch_mib"], t["claim_rays"]) == (2, 2, 256, 4096)
    assert (t["long_ray_steps"], t["long_ray_flight"], t["tally_binary32"], t["tally_plain_loads"],
            t["batch_per_snapshot"]) == (256, -1, 1, 1, 1)


def test_tune_solver_keeps_the_shape_when_no_cap_helps():
    S = FakeSolver(lambda t: 5.0 + (0 if t["scratch_mib"] == 4096 else 1.0) + (t["min_blocks_per_sm"] != 3))
    best, table = autotune.tune_solver(S, None, None, None, reps=1, scratch_mib=(256, 1024))
    assert best[:2] in {(3, 1), (3, 2)} and best[2] == 0  # the default cap stays
    assert S.tuning()["scratch_mib"] == 4096


def test_tune_batch_returns_the_fastest_and_destroys_every_batch(monkeypatch):
    destroyed = []
    monkeypatch.setattr(mcrt, "mcrt_batch_destroy", lambda b: destroyed.append(b))
    ms = {(3, 1): 9.0, (2, 2): 7.5, (4, 1): 8.0}
    runs = []

    def make(shape):
        return ("batch", shape)

    def run(b):
        runs.append(b)
        return ms[b[1]]

    best, table = autotune.tune_batch(make, run, shapes=tuple(ms), reps=2)
    assert best == (2, 2) and table == ms
    assert sorted(destroyed) == sorted(("batch", s) for s in ms)
    assert len(runs) == 3 * len(ms)  # one warm-up run and two timed runs per shape


def test_tune_batch_destroys_the_batch_when_a_run_fails(monkeypatch):
    destroyed = []
    monkeypatch.setattr(mcrt, "mcrt_batch_destroy", lambda b: destroyed.append(b))

    def run(b):
        raise RuntimeError("device error")

    with pytest.raises(RuntimeError):
        autotune.tune_batch(lambda shape: ("batch", shape), run, shapes=((3, 1),), reps=1)
    assert destroyed == [("batch", (3, 1))]
