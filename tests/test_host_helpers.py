"""Host-side helpers of the learned-proposal driver, on the CPU (no library call).

- rel_sigma_p95: the per-cell 1% criterion of the benchmark, the 95th percentile
  over cells of sigma_i / max(|Q_i|, 0.05 mean |Q|).  Checked on a hand-worked
  case, against its floor for cells with Q near 0, and for scale invariance.
- dense_cost: the dataset-wide mean steps per ray of each spectral point, the
  ratio sum_c sum_h p_k p_h c[c,k,h] / sum_c p_k (with p_h = 1/2), and the
  largest mean for a point no ray drew.  Checked against a hand-worked dataset.
"""
import numpy as np
import pytest

from paper_1810_00188_gb300 import learn


def test_rel_sigma_p95_hand_worked():
    # |Q| = 1, 2, 4, 1 -> mean 2, floor 0.1; every |Q| is above the floor
    q = np.array([1.0, -2.0, 4.0, 1.0])
    s = np.array([0.01, 0.04, 0.04, 0.03])
    # s / |Q| = 0.01, 0.02, 0.01, 0.03; the 95th percentile of 4 values, linear between
    # order statistics:
    # position 0.95 * 3 = 2.85 between the sorted values 0.02 and 0.03
    expect = 0.02 + 0.85 * (0.03 - 0.02)
    assert learn.rel_sigma_p95(q, s) == pytest.approx(expect, rel=1e-12)


def test_rel_sigma_p95_floor_for_vanishing_q():
    # Q = 0 in most cells: the floor 0.05 mean |Q| sets their scale
    q = np.zeros(100)
    q[0] = 100.0                      # mean |Q| = 1, floor 0.05
    s = np.full(100, 0.005)
    assert learn.rel_sigma_p95(q, s) == pytest.approx(0.1, rel=1e-12)


def test_rel_sigma_p95_is_scale_free():
    rng = np.random.default_rng(1)
    q = rng.normal(size=(4, 5, 6))
    s = rng.random((4, 5, 6)) * 0.1
    base = learn.rel_sigma_p95(q, s)
    for f in (1e-6, 3.0, 1e9):
        assert learn.rel_sigma_p95(f * q, f * s) == pytest.approx(base, rel=1e-12)
    assert learn.rel_sigma_p95(q, 2 * s) == pytest.approx(2 * base, rel=1e-12)


def test_dense_cost_is_the_dataset_mean_steps_per_point():
    torch = pytest.importorskip("torch")
    # 2 cells, 3 spectral points; point 2 is never drawn (zero tallies)
    p0 = torch.tensor([[0.5, 0.5, 0.0], [0.25, 0.75, 0.0]])
    # tallies c[c,k,h] = mean over rays of steps / (p_k p_h): a cell whose rays
    # at point k take s steps on average has c = s / (p_k / 2) summed over the
    # two hemispheres with equal shares
    steps = torch.tensor([[4.0, 2.0, 0.0], [8.0, 6.0, 0.0]])
    cost = torch.zeros(2, 3, 2)
    for c in range(2):
        for k in range(2):
            # half of the point's rays in each hemisphere: sum_h p_h c = s / p_k
            cost[c, k, :] = steps[c, k] / p0[c, k]
    ds = learn.Dataset(feat=torch.zeros(2, 12), mom=torch.zeros(2, 3, 2), cost=cost, p0=p0,
                       wgt=torch.ones(2), K=3, fields=1)
    sbar = learn.dense_cost(ds).double()
    # sum_c p_k (steps / p_k) / sum_c p_k = sum_c steps_c / sum_c p_k
    expect0 = (4.0 + 8.0) / (0.5 + 0.25)
    expect1 = (2.0 + 6.0) / (0.5 + 0.75)
    assert sbar[0].item() == pytest.approx(expect0, rel=1e-12)
    assert sbar[1].item() == pytest.approx(expect1, rel=1e-12)
    # the undrawn point gets the largest mean seen
    assert sbar[2].item() == pytest.approx(max(expect0, expect1), rel=1e-12)
    # every cell and hemisphere now carries the same dense cost
    assert tuple(ds.cost.shape) == (2, 3, 2)
    assert torch.allclose(ds.cost[0], ds.cost[1]) and torch.allclose(ds.cost[..., 0], ds.cost[..., 1])
