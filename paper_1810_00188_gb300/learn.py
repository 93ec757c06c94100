"""Training driver of the learned proposal.

Host orchestration only: the tallies, features, forward/backward passes, the
gradient reduction and Adam all run in the library's kernels through the C ABI;
this module picks the fields, the cells and the batches (seeded), and keeps the
device tensors the kernels read.

Training data (one sample per tallied cell): the 12 features, the second-moment
tallies m [K][2] and cost tallies c [K][2] of a plain FP32 solve, the plain pdf
p0 [K] of the sample's field, and the weight w = 1 / ref^2 with
ref = max(|Q|, 0.05 mean |Q|) the cell's error scale (the per-cell 1% criterion).
With A(q) = sum m / (q_k q_h) (the second moment of the estimate per ray under q)
and C(q) = c0 + sum c q_k q_h (the ray's cost in steps, c0 its fixed part), the
default loss is the batch estimate of the GPU-time ratio to a given relative
error, (sum w A(q) / sum w A(p0)) (sum C(q) / sum C(p0)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import inputs, mcrt


@dataclasses.dataclass
class Dataset:
    feat: object        # torch [N, 12] float32, cuda
    mom: object         # torch [N, K, 2]
    cost: object        # torch [N, K, 2]
    p0: object          # torch [N, K]
    wgt: object         # torch [N]: 1 / ref^2
    K: int
    fields: int

    @property
    def n(self) -> int:
        return int(self.feat.shape[0])


def tally_field(S, rays, seed, snapshot, cells, stream=0, mg_levels=1, mg_steps=5):
    """Features, tallies, p0 rows and weights 1/ref^2 of `cells` (torch int32
    cuda) of the context's current fields (from a multigrid solve when
    mg_levels > 1)."""
    import torch
    feat = S.features(cells, stream=stream)
    p = S.params(rays=rays, seed=seed, snapshot=snapshot, precision=mcrt.MCRT_FP32,
                 mg_levels=mg_levels, mg_steps=mg_steps)
    q = torch.empty(S.box_shape(None), dtype=torch.float64, device=feat.device)
    mom, cost = S.tally(p, cells, q=q, stream=stream)
    p0 = torch.tensor(S.plain_probs(), device=feat.device)
    qa = q.reshape(-1).abs()
    ref = torch.clamp(qa[cells.long()], min=0.05 * float(qa.mean()))
    wgt = (1.0 / ref**2).float()
    return feat, mom, cost, p0.expand(cells.shape[0], -1), wgt


def build_dataset(grid_shape=(64, 64, 64), seeds=range(200), rays=512, cells_per_field=4096,
                  kdist_seed=0, x_mode="field", sample_seed=0, stream=0, dense=True, mg=0,
                  mg_steps=5):
    """Tallies of `cells_per_field` random cells of each seeded channel field
    (cost tallies replaced by the dataset-wide mean steps per point unless
    dense=False).  mg = 1 tallies multigrid solves on every grid the field
    allows (mg_steps segments per grid)."""
    import concurrent.futures as cf

    import torch
    nx, ny, nz = grid_shape
    feats, moms, costs, p0s, wgts = [], [], [], [], []
    rng = np.random.default_rng(sample_seed)
    S = None
    kd = None
    seeds = [int(s) for s in seeds]

    def make(s):
        return inputs.nongrey_channel(nx, ny, nz, seed=s, kdist_seed=kdist_seed, x_mode=x_mode)

    # the host builds the next fields while the GPU tallies the current one
    pool = cf.ThreadPoolExecutor(max_workers=8)
    futs = [pool.submit(make, s) for s in seeds[:8]]
    for i, s in enumerate(seeds):
        grid, kd_s, T, x = futs[i].result()
        futs[i] = None
        if i + 8 < len(seeds):
            futs.append(pool.submit(make, seeds[i + 8]))
        if S is None:
            kd = kd_s
            S = mcrt.Solver(grid, kd)
        S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"), stream=stream)
        n = min(cells_per_field, grid.ncells)
        cells = torch.tensor(np.sort(rng.choice(grid.ncells, n, replace=False)).astype(np.int32),
                             device="cuda")
        L = mcrt.mcrt_multigrid_levels(nx, ny, nz) if mg else 1
        f, m, c, p, w = tally_field(S, rays, seed=1000 + s, snapshot=s, cells=cells, stream=stream,
                                    mg_levels=L, mg_steps=mg_steps)
        feats.append(f)
        moms.append(m)
        costs.append(c)
        p0s.append(p.contiguous())
        wgts.append(w)
    pool.shutdown()
    S.close()
    K = kd.n_bands * kd.n_g
    w = torch.cat(wgts)
    ds = Dataset(torch.cat(feats), torch.cat(moms), torch.cat(costs), torch.cat(p0s),
                 (w / w.mean()).contiguous(), K, len(feats))
    if dense:
        dense_cost(ds)
    return ds


def dense_cost(ds: Dataset):
    """Replaces the per-cell cost tallies by the mean steps per ray of each
    spectral point over the whole dataset (the same for every cell and both
    hemispheres).  A cell's tallies are zero at the points its rays never drew;
    trained on them, a network learns that those points are free and moves its
    probability there -- typically optically thin bands, whose rays are the
    longest.  The dataset-wide mean is an unbiased ratio estimate of the steps of
    a ray at each point: sum_c sum_h p_k p_h c[c,k,h] / sum_c p_k."""
    import torch
    w = ds.p0.double() * 0.5                                         # [N, K]
    steps = (ds.cost.double() * w[:, :, None]).sum(dim=(0, 2))       # sum_c sum_h p_k p_h c
    norm = ds.p0.double().sum(dim=0)
    drawn = steps > 0  # every drawn ray takes at least one step
    sbar = torch.where(drawn, steps / torch.clamp(norm, min=1e-300), torch.zeros_like(norm))
    # a point never drawn in the whole dataset is an optically thin one (the plain
    # pdf weights points by kappa): it gets the largest mean seen
    sbar = torch.where(drawn, sbar, sbar.max())
    ds.cost = sbar.float()[None, :, None].expand(ds.n, -1, 2).contiguous()
    return sbar


def feature_norm(ds: Dataset):
    """Mean and 1/std of each feature over the dataset (constant features get 1)."""
    f = ds.feat.double().cpu().numpy()
    mean = f.mean(axis=0)
    std = f.std(axis=0)
    inv = np.where(std > 1e-6 * np.maximum(np.abs(mean), 1.0), 1.0 / np.maximum(std, 1e-30), 1.0)
    return mean.astype(np.float32), inv.astype(np.float32)


def init_theta(K, p0_mean, seed=0, scale=1.0):
    """He-style random weights; the spectral biases start at log p0 (so the
    untrained network proposes the mean plain pdf), the hemisphere ones at 0."""
    H, F = mcrt.MCRT_NHIDDEN, mcrt.MCRT_NFEAT
    rng = np.random.default_rng(seed)
    W1 = rng.normal(scale=scale * math.sqrt(2.0 / F), size=(H, F))
    W2 = rng.normal(scale=scale * math.sqrt(2.0 / H), size=(H, H))
    W3 = rng.normal(scale=0.1 * scale * math.sqrt(1.0 / H), size=(K + 2, H))
    b3 = np.zeros(K + 2)
    b3[:K] = np.log(np.maximum(np.asarray(p0_mean, dtype=np.float64), 1e-12))
    b3[:K] -= b3[:K].max()
    theta = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3.ravel(), b3])
    assert theta.size == mcrt.mcrt_mlp_nparams(K)
    return theta.astype(np.float32)


def train(mlp, ds: Dataset, steps=1500, batch=None, lr=2e-3, c0=1.0, mix=0.1, seed=0,
          log_every=0, stream=0, use_cost=True, mode=mcrt.MCRT_LOSS_BATCH):
    """Adam on the loss over random batches.  Returns the losses at the logged
    steps (and the last one)."""
    import torch
    if batch is None:
        batch = 16 * torch.cuda.get_device_properties(0).multi_processor_count * 2
    rng = np.random.default_rng(seed)
    losses = []
    perm = None
    pos = ds.n
    for it in range(steps):
        if pos + batch > ds.n:
            perm = torch.tensor(rng.permutation(ds.n).astype(np.int32), device=ds.feat.device)
            pos = 0
        idx = perm[pos:pos + min(batch, ds.n)]
        pos += batch
        mlp.loss_grad(ds.feat, ds.mom, ds.p0, cost=ds.cost if use_cost else None, c0=c0, idx=idx,
                      mix=mix, wgt=ds.wgt, mode=mode, stream=stream)
        mlp.adam(lr=lr, stream=stream)
        if (log_every and it % log_every == 0) or it == steps - 1:
            losses.append((it, mlp.last_loss()))
    return losses


def mean_loss(mlp, ds: Dataset, c0=1.0, mix=0.1, stream=0, use_cost=True,
              mode=mcrt.MCRT_LOSS_BATCH):
    """Loss over the whole dataset (no update)."""
    mlp.loss_grad(ds.feat, ds.mom, ds.p0, cost=ds.cost if use_cost else None, c0=c0, mix=mix,
                  wgt=ds.wgt, mode=mode, stream=stream)
    return mlp.last_loss()


def rel_sigma_p95(q, s):
    """95th percentile over cells of sigma / max(|Q|, 0.05 mean |Q|) (the
    per-cell 1% criterion)."""
    q = np.asarray(q).reshape(-1)
    s = np.asarray(s).reshape(-1)
    ref = np.maximum(np.abs(q), 0.05 * np.mean(np.abs(q)))
    return float(np.percentile(s / ref, 95))


def compare_on_field(S, mlp, rays, seed=0, mix=0.1, reps=3, stream=0, mg_levels=1, mg_steps=5):
    """Plain and learned FP32 solves of the context's fields at `rays` per cell
    (both on mg_levels grids): kernel time, p95 relative sigma, and the
    projected GPU time to reach 1% (time x (p95 / 0.01)^2, the estimator's 1/N
    law)."""
    import torch
    shape = S.box_shape(None)
    dev = f"cuda:{S.device}"
    q = torch.empty(shape, dtype=torch.float64, device=dev)
    s = torch.empty_like(q)
    out = {}
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    S.set_learned_proposal(mlp, mix=mix, stream=stream)
    t1.record()
    torch.cuda.synchronize()
    out["proposal_ms"] = t0.elapsed_time(t1)
    for name, prop in (("plain", mcrt.MCRT_PROPOSAL_PLANCK_TMAX), ("learned", mcrt.MCRT_PROPOSAL_CELL)):
        times, p95 = [], []
        steps = 0
        for r in range(reps):
            p = S.params(rays=rays, seed=seed, ray_offset=r * rays, precision=mcrt.MCRT_FP32,
                         proposal=prop, mg_levels=mg_levels, mg_steps=mg_steps)
            S.solve_into(p, q, s, stream=stream)
            st = S.stats()
            times.append(st["kernel_ms"])
            steps += st["steps"]
            p95.append(rel_sigma_p95(q.cpu().numpy(), s.cpu().numpy()))
        t = float(np.median(times))
        pr = float(np.median(p95))
        out[name] = {"kernel_ms": t, "p95_rel_sigma": pr,
                     "steps_per_ray": steps / (reps * rays * S.grid.ncells),
                     "ms_to_1pct": t * (pr / 0.01) ** 2}
    out["speedup_to_1pct"] = out["plain"]["ms_to_1pct"] / out["learned"]["ms_to_1pct"]
    out["speedup_to_1pct_incl_proposal"] = out["plain"]["ms_to_1pct"] / (
        out["learned"]["ms_to_1pct"] + out["proposal_ms"])
    return out


def compare_equal_budget(S, mlp, rays, seed=0, mix=0.1, reps=2, stream=0, mg_levels=1, mg_steps=5):
    """Plain and learned FP32 solves of the context's fields given the same
    measured GPU time: the plain arm runs `rays` per cell; a pilot learned solve
    at the same rays gives its time per ray, and the learned arm then runs the
    ray count that fills the plain arm's kernel time.  Reports both arms' measured
    kernel times, rays and achieved p95 relative sigma (medians over `reps`
    solves at different ray offsets) and the sigma ratio at equal time; the time
    to build the proposal is reported separately (it is paid once per field)."""
    import torch
    shape = S.box_shape(None)
    dev = f"cuda:{S.device}"
    q = torch.empty(shape, dtype=torch.float64, device=dev)
    s = torch.empty_like(q)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    S.set_learned_proposal(mlp, mix=mix, stream=stream)
    t1.record()
    torch.cuda.synchronize()
    out = {"proposal_ms": t0.elapsed_time(t1)}

    def arm(prop, n, base):
        times, p95, steps = [], [], 0
        for r in range(reps):
            p = S.params(rays=n, seed=seed, ray_offset=base + r * n, precision=mcrt.MCRT_FP32,
                         proposal=prop, mg_levels=mg_levels, mg_steps=mg_steps)
            S.solve_into(p, q, s, stream=stream)
            st = S.stats()
            times.append(st["kernel_ms"])
            steps += st["steps"]
            p95.append(rel_sigma_p95(q.cpu().numpy(), s.cpu().numpy()))
        return {"rays": n, "kernel_ms": float(np.median(times)), "p95_rel_sigma": float(np.median(p95)),
                "steps_per_ray": steps / (reps * n * S.grid.ncells)}

    plain = arm(mcrt.MCRT_PROPOSAL_PLANCK_TMAX, rays, 0)
    # the learned arm's rays: two pilots (the time per ray falls a little with the
    # ray count, so one pilot at the plain arm's rays overshoots)
    n_l = rays
    for _ in range(2):
        pilot = arm(mcrt.MCRT_PROPOSAL_CELL, n_l, 0)
        n_l = max(1, int(round(n_l * plain["kernel_ms"] / pilot["kernel_ms"])))
    learned = arm(mcrt.MCRT_PROPOSAL_CELL, n_l, 1 << 20)
    out.update({"plain": plain, "learned": learned,
                "time_ratio_learned_over_plain": learned["kernel_ms"] / plain["kernel_ms"],
                "p95_sigma_ratio_plain_over_learned": plain["p95_rel_sigma"] / learned["p95_rel_sigma"]})
    return out
