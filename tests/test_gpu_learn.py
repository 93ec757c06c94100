"""GPU parity of the learned-proposal path against the oracle: cell features,
second-moment and cost tallies (draw for draw), the network's forward pass, its
loss gradient (relative 1e-3, FP16 weights with FP32 arithmetic against FP64),
Adam, the integer quantisation (bit-exact), the per-cell proposal solve (draw
for draw), and what a trained network gains over the plain proposal."""
import numpy as np
import pytest

import oracle
from paper_1810_00188_gb300 import inputs, learn, mcrt

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _solver(grid, kd, T, x):
    torch = _torch()
    S = mcrt.Solver(grid, kd)
    S.set_fields(torch.tensor(T, device="cuda"), torch.tensor(x, device="cuda"))
    return S


def _field(nx=13, ny=10, nz=7, seed=3, eps=(0.7, 0.9)):
    grid, kd, T, x = inputs.nongrey_channel(nx, ny, nz, seed=seed, x_mode="field")
    grid = inputs.Grid(nx, ny, nz, grid.lx, grid.ly, grid.lz, eps_wall=eps, T_wall=grid.T_wall)
    return grid, kd, T, x


# ---- features ---------------------------------------------------------------------

def test_features_match_oracle():
    torch = _torch()
    grid, kd, T, x = _field()
    S = _solver(grid, kd, T, x)
    ref = oracle.features(grid, kd, T, x)
    got = S.features().cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=2e-5, atol=2e-6)
    cells = np.array([0, grid.ncells - 1, 5, 77, 300, 13 * 10 - 1], dtype=np.int32)
    got2 = S.features(torch.tensor(cells, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(got2, ref[cells], rtol=2e-5, atol=2e-6)
    with pytest.raises(mcrt.McrtError) as e:
        S.features(torch.tensor([grid.ncells], dtype=torch.int32, device="cuda"))
    assert e.value.status == mcrt.MCRT_E_ARG
    S.close()


# ---- tallies -----------------------------------------------------------------------

def _random_cell_proposal(nc, nb, ng, seed):
    """Host-generated integer proposals: random counts of 2^32 (every point >= 1)
    and hemisphere counts across [1, 2^23 - 1]."""
    rng = np.random.default_rng(seed)
    def cum(rows, k):
        c = rng.integers(1, 2**26, size=(rows, k)).astype(np.int64)
        c[:, -1] += 2**32 - c.sum(axis=1)
        return np.cumsum(c, axis=1).astype(np.uint64)
    cn = cum(nc, nb)
    cg = cum(nc * nb, ng).reshape(nc, nb, ng)
    hemi = rng.integers(1, 2**23, size=nc).astype(np.uint32)
    return cn, cg, hemi


@pytest.mark.parametrize("cellprop", [False, True])
def test_tally_matches_oracle(cellprop):
    torch = _torch()
    grid, kd, T, x = _field(9, 10, 6, seed=5)
    nb, ng = kd.n_bands, kd.n_g
    K = nb * ng
    S = _solver(grid, kd, T, x)
    prop = None
    if cellprop:
        prop = _random_cell_proposal(grid.ncells, nb, ng, 8)
        S.set_cell_proposal(*prop)
    rays = 300
    cells = np.array([0, 1, 8, 9, 80, 200, 333, grid.ncells - 1], dtype=np.int32)
    p = S.params(rays=rays, seed=4, snapshot=2, ray_offset=17, precision=mcrt.MCRT_FP32,
                 proposal=mcrt.MCRT_PROPOSAL_CELL if cellprop else mcrt.MCRT_PROPOSAL_PLANCK_TMAX)
    q = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
    mom, cost = S.tally(p, torch.tensor(cells, device="cuda"), q=q)
    mom, cost = mom.cpu().numpy(), cost.cpu().numpy()
    orc = oracle.solve(grid, kd, T, x, rays=rays, seed=4, snapshot=2, ray_offset=17, tally=True,
                       proposal=None if not cellprop else
                       (prop[0], prop[1].reshape(grid.ncells, K), prop[2]))
    tm = orc["tally"].reshape(grid.ncells, K, 2)[cells]
    tc = orc["tally_cost"].reshape(grid.ncells, K, 2)[cells]
    # the same rays land in the same bins (integer decisions on the same draws)
    np.testing.assert_array_equal(mom > 0, tm > 0)
    np.testing.assert_array_equal(cost > 0, tc > 0)
    # second moments: FP32 samples against FP64, relative to the cell's total
    tot = tm.sum(axis=(1, 2))[:, None, None]
    assert np.all(np.abs(mom - tm) <= 1e-3 * tot + 1e-30)
    # costs: steps per ray agree (a rare FP32/FP64 step difference is allowed)
    np.testing.assert_allclose(cost.sum(axis=(1, 2)), tc.sum(axis=(1, 2)), rtol=2e-2)
    close = np.isclose(cost, tc, rtol=1e-5, atol=0)
    assert close.mean() > 0.99
    # the solve itself is the regular FP32 solve
    q2, _ = S.solve(rays=rays, seed=4, snapshot=2, ray_offset=17, precision=mcrt.MCRT_FP32,
                    proposal=p.proposal)
    np.testing.assert_array_equal(q.cpu().numpy(), q2)
    S.close()


def test_cell_proposal_solve_parity():
    """Per-cell proposals (host-generated counts, hemisphere splits) through the
    FP32 and FP64 kernels, draw for draw against the oracle."""
    grid, kd, T, x = _field(11, 12, 5, seed=6)
    nb, ng = kd.n_bands, kd.n_g
    prop = _random_cell_proposal(grid.ncells, nb, ng, 9)
    orc = oracle.solve(grid, kd, T, x, rays=96, seed=3,
                       proposal=(prop[0], prop[1].reshape(grid.ncells, nb * ng), prop[2]))
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, x)
    S.set_cell_proposal(*prop)
    for prec, rtol in ((mcrt.MCRT_FP64, 1e-10), (mcrt.MCRT_FP32, 1e-4)):
        q, s = S.solve(rays=96, seed=3, precision=prec, proposal=mcrt.MCRT_PROPOSAL_CELL)
        err = np.abs(q - orc["q"]) / np.maximum(orc["scale"], 1e-300)
        assert err.max() <= rtol, (prec, err.max())
    S.close()


# ---- network ------------------------------------------------------------------------

def _net_problem(K, n, seed):
    rng = np.random.default_rng(seed)
    theta = (rng.normal(scale=0.4, size=mcrt.mcrt_mlp_nparams(K))).astype(np.float16).astype(np.float32)
    feat = rng.normal(size=(n, 12)).astype(np.float32)
    fmean = rng.normal(scale=0.2, size=12).astype(np.float32)
    finv = rng.uniform(0.5, 2.0, size=12).astype(np.float32)
    mom = (rng.exponential(size=(n, K, 2)) * (rng.random((n, K, 2)) < 0.3)).astype(np.float32)
    cost = (rng.exponential(scale=10.0, size=(n, K, 2)) * (mom > 0)).astype(np.float32)
    p0 = rng.dirichlet(np.ones(K), size=n).astype(np.float32)
    return theta, feat, fmean, finv, mom, cost, p0


def test_mlp_forward_matches_oracle():
    torch = _torch()
    K, n = 320, 77
    theta, feat, fmean, finv, _, _, p0 = _net_problem(K, n, 1)
    net = mcrt.Mlp(K)
    net.set_params(theta, fmean, finv)
    _, used = net.params(used=True)
    np.testing.assert_array_equal(used, theta)  # FP16-representable values pass unchanged
    q = net.forward(torch.tensor(feat, device="cuda"), torch.tensor(p0[0], device="cuda"), mix=0.1)
    ref = oracle.mlp_forward(used, K, fmean, finv, feat, p0[0].astype(np.float64), mix=0.1)
    np.testing.assert_allclose(q.cpu().numpy(), ref, rtol=2e-4, atol=1e-9)
    q2 = net.forward(torch.tensor(feat, device="cuda"), torch.tensor(p0, device="cuda"), mix=0.25)
    ref2 = oracle.mlp_forward(used, K, fmean, finv, feat, p0.astype(np.float64), mix=0.25)
    np.testing.assert_allclose(q2.cpu().numpy(), ref2, rtol=2e-4, atol=1e-9)
    net.close()


@pytest.mark.parametrize("with_cost,mode", [(False, 0), (True, 0), (False, 1), (True, 1)])
def test_mlp_gradient_matches_oracle(with_cost, mode):
    torch = _torch()
    K, N = 320, 300
    theta, feat, fmean, finv, mom, cost, p0 = _net_problem(K, N, 2)
    wgt = np.random.default_rng(7).uniform(0.05, 4.0, N).astype(np.float32)
    net = mcrt.Mlp(K)
    net.set_params(theta, fmean, finv)
    idx = np.random.default_rng(3).permutation(N)[:203].astype(np.int32)
    d = {k: torch.tensor(v, device="cuda") for k, v in
         dict(feat=feat, mom=mom, cost=cost, p0=p0, idx=idx, wgt=wgt).items()}
    grad = torch.empty(net.nparams, dtype=torch.float32, device="cuda")
    c0 = 8.0
    kw = dict(cost=d["cost"] if with_cost else None, c0=c0, idx=d["idx"], mix=0.1, wgt=d["wgt"],
              mode=mode)
    net.loss_grad(d["feat"], d["mom"], d["p0"], grad=grad, **kw)
    loss = net.last_loss()
    g = grad.cpu().numpy().astype(np.float64)
    Lr, gr = oracle.mlp_loss_grad(theta, K, fmean, finv, feat[idx], mom[idx], p0[idx], mix=0.1,
                                  cost=cost[idx] if with_cost else None, c0=c0, wgt=wgt[idx],
                                  mode=mode)
    assert loss == pytest.approx(Lr, rel=1e-5)
    assert np.linalg.norm(g - gr) <= 1e-3 * np.linalg.norm(gr)
    assert np.max(np.abs(g - gr)) <= 1e-3 * np.max(np.abs(gr))
    # fixed-order reduction: the same batch gives the same bits
    grad2 = torch.empty_like(grad)
    net.loss_grad(d["feat"], d["mom"], d["p0"], grad=grad2, **kw)
    assert torch.equal(grad, grad2)
    # an index outside the dataset is skipped and reported
    bad = d["idx"].clone()
    bad[5] = N
    net.loss_grad(d["feat"], d["mom"], d["p0"], c0=c0, idx=bad, mix=0.1)
    with pytest.raises(mcrt.McrtError) as e:
        net.last_loss()
    assert e.value.status == mcrt.MCRT_E_ARG
    net.close()


def test_adam_matches_oracle():
    torch = _torch()
    K = 40
    rng = np.random.default_rng(4)
    theta = rng.normal(size=mcrt.mcrt_mlp_nparams(K)).astype(np.float32)
    net = mcrt.Mlp(K)
    net.set_params(theta)
    th, m1, m2 = theta.astype(np.float64), np.zeros(theta.size), np.zeros(theta.size)
    for t in (1, 2, 3):
        g = rng.normal(scale=10.0 ** rng.integers(-4, 2), size=theta.size).astype(np.float32)
        net.adam(torch.tensor(g, device="cuda"), lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
        th, m1, m2 = oracle.adam(th, g, m1, m2, t, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
    got, used = net.params(used=True)
    np.testing.assert_allclose(got, th, rtol=1e-6, atol=1e-6)
    np.testing.assert_array_equal(used, got.astype(np.float16).astype(np.float32))
    net.close()


# ---- quantisation and the learned proposal -------------------------------------------------

def test_quantisation_is_bit_exact():
    torch = _torch()
    grid = inputs.Grid(5, 4, 3, 1.0, 2.0, 1.0)
    kd = inputs.make_kdist(0)
    T = np.full(grid.shape, 800.0)
    S = mcrt.Solver(grid, kd)
    S.set_fields(T, None)
    nb, ng = kd.n_bands, kd.n_g
    K = nb * ng
    rng = np.random.default_rng(5)
    q = np.zeros((grid.ncells, K + 2), dtype=np.float32)
    for c in range(grid.ncells):
        conc = 10.0 ** rng.uniform(-2, 1)
        v = rng.dirichlet(np.ones(K) * conc)
        v[rng.random(K) < 0.05] = 0.0
        if c == 3:
            v[8:16] = 0.0  # a band without weight
        q[c, :K] = v
        q[c, K] = [0.0, 1.0, 0.5, 1e-9][c % 4] if c < 8 else rng.random()
    S.set_cell_proposal_probs(torch.tensor(q, device="cuda"))
    cn, cg, hemi = S.cell_proposal()
    for c in range(grid.ncells):
        a, b, h = oracle.learned_counts(q[c, :K].astype(np.float64), nb, ng, float(q[c, K]))
        np.testing.assert_array_equal(cn[c], a)
        np.testing.assert_array_equal(cg[c], b)
        assert hemi[c] == h
    bad = q.copy()
    bad[2, :K] = 0.0
    with pytest.raises(mcrt.McrtError):
        S.set_cell_proposal_probs(torch.tensor(bad, device="cuda"))
    S.close()


def test_learned_proposal_is_features_forward_quantise():
    torch = _torch()
    grid, kd, T, x = _field(12, 9, 7, seed=7)
    K = kd.n_bands * kd.n_g
    S = _solver(grid, kd, T, x)
    net = mcrt.Mlp(K)
    theta = learn.init_theta(K, S.plain_probs(), seed=1, scale=2.0)
    net.set_params(theta, np.zeros(12, np.float32), np.ones(12, np.float32))
    S.set_learned_proposal(net, mix=0.1)
    a = S.cell_proposal()
    f = S.features()
    q = net.forward(f, torch.tensor(S.plain_probs(), device="cuda"), mix=0.1)
    S.set_cell_proposal_probs(q)
    b = S.cell_proposal()
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    net.close()
    S.close()


def test_learned_solve_is_unbiased():
    """A strongly skewed network proposal and the plain one estimate the same
    Q: per-cell z-scores of the difference are standard normal."""
    torch = _torch()
    grid, kd, T, x = _field(8, 16, 8, seed=8, eps=(1.0, 1.0))
    K = kd.n_bands * kd.n_g
    S = _solver(grid, kd, T, x)
    net = mcrt.Mlp(K)
    rng = np.random.default_rng(6)
    p0 = S.plain_probs()
    theta = learn.init_theta(K, np.sqrt(p0) * rng.uniform(0.2, 5.0, K), seed=2, scale=3.0)
    f = S.features().cpu().numpy()
    net.set_params(theta, f.mean(0), 1.0 / np.maximum(f.std(0), 1e-3))
    S.set_learned_proposal(net, mix=0.1)
    _, _, hemi = S.cell_proposal()
    assert np.std(hemi.astype(np.float64) / 2**23) > 1e-3  # hemisphere split varies
    rays = 20000
    ql, sl = S.solve(rays=rays, seed=11, precision=mcrt.MCRT_FP32, proposal=mcrt.MCRT_PROPOSAL_CELL)
    qp, sp = S.solve(rays=rays, seed=12, precision=mcrt.MCRT_FP32)
    z = ((ql - qp) / np.sqrt(sl**2 + sp**2)).reshape(-1)
    assert abs(z.mean()) < 4.0 / np.sqrt(z.size)
    assert np.mean(np.abs(z) > 3.0) < 0.01
    assert 0.8 < np.mean(z**2) < 1.25
    net.close()
    S.close()


def test_training_lowers_the_work_to_reach_a_given_error():
    """Train on multigrid tallies of small seeded fields; on a held-out field,
    with the multigrid march in both arms, the learned proposal needs less GPU
    time than the plain one for the same p95 error."""
    torch = _torch()
    ds = learn.build_dataset(grid_shape=(64, 64, 64), seeds=range(24), rays=512,
                             cells_per_field=8192, mg=1)
    K = ds.K
    net = mcrt.Mlp(K)
    mean, inv = learn.feature_norm(ds)
    theta = learn.init_theta(K, ds.p0.mean(0).cpu().numpy(), seed=0)
    net.set_params(theta, mean, inv)
    l0 = learn.mean_loss(net, ds, c0=12.0)
    learn.train(net, ds, steps=1500, lr=2e-3, c0=12.0)
    l1 = learn.mean_loss(net, ds, c0=12.0)
    assert l1 < 0.8 * l0, (l0, l1)
    grid, kd, T, x = inputs.nongrey_channel(64, 64, 64, seed=1000, x_mode="field")
    S = _solver(grid, kd, T, x)
    res = learn.compare_on_field(S, net, rays=512, seed=3, reps=3, mg_levels=5, mg_steps=5)
    assert res["speedup_to_1pct"] > 1.1, res
    net.close()
    S.close()
