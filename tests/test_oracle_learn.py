"""Pins of the oracle's learned-proposal parts (features, second-moment tallies,
network forward/backward, Adam, integer counts) to closed forms, special cases
and brute force -- nothing here compares the oracle with itself."""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
from paper_1810_00188_gb300 import inputs

K_SMALL = 6


def _grid(nx=6, ny=8, nz=5, eps=(1.0, 1.0), Tw=(500.0, 1000.0)):
    return inputs.Grid(nx, ny, nz, 3.0, 2.0, 2.5, eps_wall=eps, T_wall=Tw)


# ---- features ----------------------------------------------------------------

def test_features_linear_in_y():
    """T = a + b y: centred and one-sided differences are exact, the x-z
    gradient is zero, the 3^3 mean is T_j inside and shifted by b dy / 2 at the
    walls (the neighbourhood is cut there)."""
    g = _grid(eps=(0.7, 0.9))
    kd = inputs.make_grey_kdist(0.8)
    a, b = 600.0, 150.0
    dy = g.ly / g.ny
    yc = (np.arange(g.ny) + 0.5) * dy
    T = np.broadcast_to((a + b * yc)[None, :, None], (g.nz, g.ny, g.nx)).copy()
    x = np.full(T.shape, 0.1)
    f = oracle.features(g, kd, T, x, T_max=1234.0)
    f = f.reshape(g.nz, g.ny, g.nx, 12)
    h = g.ly / 2
    for j in range(g.ny):
        Tj = a + b * yc[j]
        row = f[2, j, 3]
        assert row[0] == pytest.approx(Tj / 1000)
        assert row[1] == pytest.approx(0.1)
        assert row[2] == pytest.approx(yc[j] / h - 1)
        assert row[3] == pytest.approx(0.5) and row[4] == pytest.approx(1.0)
        assert row[5] == (0.7 if yc[j] < h else 0.9)
        assert row[6] == pytest.approx(h * b / 1000, rel=1e-12)
        assert abs(row[7]) < 1e-12
        mean = Tj + (b * dy / 2 if j == 0 else (-b * dy / 2 if j == g.ny - 1 else 0.0))
        assert row[8] == pytest.approx(mean / Tj, rel=1e-12)
        # std of 3 rows (or 2 at a wall) of a linear profile, 9 cells each
        vals = [a + b * yc[jj] for jj in (j - 1, j, j + 1) if 0 <= jj < g.ny]
        assert row[9] == pytest.approx(np.std(vals) / Tj, rel=1e-10)
        assert row[11] == pytest.approx(1234.0 / Tj)


def test_features_periodic_gradient_and_grey_planck_mean():
    """T = a + c cos(2 pi x / lx): the centred difference is
    -c sin(2 pi x_i / lx) sin(2 pi dx / lx) / dx; with a grey table the Planck
    mean absorption coefficient is kappa x / x_ref."""
    g = _grid(nx=8)
    kap = 1.7
    kd = inputs.make_grey_kdist(kap)
    a, c = 900.0, 40.0
    dx = g.lx / g.nx
    xc = (np.arange(g.nx) + 0.5) * dx
    T = np.broadcast_to((a + c * np.cos(2 * np.pi * xc / g.lx))[None, None, :], (g.nz, g.ny, g.nx)).copy()
    xh = np.full(T.shape, 0.05)
    f = oracle.features(g, kd, T, xh).reshape(g.nz, g.ny, g.nx, 12)
    h = g.ly / 2
    d = -c * np.sin(2 * np.pi * xc / g.lx) * np.sin(2 * np.pi * dx / g.lx) / dx
    np.testing.assert_allclose(f[1, 3, :, 7], h * np.abs(d) / 1000, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(f[..., 10], kap * 0.05 / kd.x_ref * h, rtol=1e-12)
    assert np.all(np.abs(f[..., 6]) < 1e-12)


def test_features_uniform_field():
    g = _grid()
    kd = inputs.make_kdist(0)
    T = np.full((g.nz, g.ny, g.nx), 1000.0)
    f = oracle.features(g, kd, T, None)
    np.testing.assert_allclose(f[:, 8], 1.0, rtol=1e-14)
    np.testing.assert_allclose(f[:, 9], 0.0, atol=1e-14)
    np.testing.assert_allclose(f[:, 1], kd.x_ref)
    np.testing.assert_allclose(f[:, 11], 1000.0 / 1000.0)  # T_max is the medium maximum (1000)
    with pytest.raises(ValueError):
        oracle.features(g, kd, T, None, cells=[g.ncells])


# ---- second-moment tallies -----------------------------------------------------

def _probs(cn, cg, nb, ng):
    pn = np.diff(np.concatenate([[0], cn.astype(np.float64)])) / 2.0**32
    pg = np.diff(np.concatenate([np.zeros((nb, 1)), cg.astype(np.float64)], axis=1), axis=1) / 2.0**32
    return (pn[:, None] * pg).reshape(-1)


def test_tally_reweights_to_plain_second_moment():
    """Dividing the tallies by the probabilities they were drawn with gives back
    the plain per-cell mean of Y^2 exactly (up to rounding)."""
    grid, kd, T, x = inputs.nongrey_channel(6, 8, 5, seed=3, x_mode="field")
    r = oracle.solve(grid, kd, T, x, rays=200, seed=5, tally=True)
    cn, cg, _ = oracle.plain_proposal(grid, kd, T, x)
    p0 = _probs(cn, cg, kd.n_bands, kd.n_g)
    tl = r["tally"]
    back = (tl / (p0[:, None] * 0.5)).sum(axis=(-1, -2))
    np.testing.assert_allclose(back, r["sum_y2"] / 200, rtol=1e-12)
    # the cost tallies weighted by the drawing probabilities give the mean steps
    steps = (r["tally_cost"] * (p0[:, None] * 0.5)).sum(axis=(-1, -2))
    np.testing.assert_allclose(steps, r["steps"].astype(np.float64) / 200, rtol=1e-12)
    # only spectral points / hemispheres that were drawn are non-zero
    assert np.count_nonzero(tl) <= tl.shape[0] * tl.shape[1] * tl.shape[2] * 200


def test_tally_predicts_second_moment_under_another_proposal():
    """sum m / (q_k q_h) from plain tallies is an unbiased estimate of E[Y^2]
    under proposal q: compare with a direct solve under q (many rays)."""
    grid, kd, T, x = inputs.nongrey_channel(4, 6, 4, seed=1, x_mode="field")
    nb, ng = kd.n_bands, kd.n_g
    cn, cg, _ = oracle.plain_proposal(grid, kd, T, x)
    p0 = _probs(cn, cg, nb, ng)
    # an alternative proposal within a bounded ratio of the plain one (so that
    # the reweighted estimates stay light-tailed), biased upward
    qk = p0 * (1.0 + 0.6 * np.cos(np.arange(nb * ng)))
    qk /= qk.sum()
    q_up = 0.7
    pc = oracle.learned_counts(qk, nb, ng, q_up)
    qk_exact = _probs(pc[0], pc[1], nb, ng)
    qh = np.array([pc[2], 2**23 - pc[2]]) / 2.0**23
    # Y^2 is heavy-tailed: many rays on a few cells, compared in total
    rays, box, nbx = 100000, (0, 2, 2, 4, 0, 1), 4
    plain = oracle.solve(grid, kd, T, x, rays=rays, seed=1, tally=True, box=box)
    pred = (plain["tally"] / (qk_exact[:, None] * qh[None, :])).sum()
    prop = (np.tile(pc[0], (nbx, 1)), np.tile(pc[1].reshape(-1), (nbx, 1)), np.full(nbx, pc[2]))
    direct = oracle.solve(grid, kd, T, x, rays=rays, seed=2, proposal=prop, box=box)
    ratio = pred / (direct["sum_y2"].sum() / rays)
    assert 0.93 < ratio < 1.07, ratio
    # the mean steps per ray under q, predicted from the plain cost tallies
    cpred = (plain["tally_cost"] * (qk_exact[:, None] * qh[None, :])).sum()
    cdir = direct["steps"].astype(np.float64).sum() / rays
    assert abs(cpred / cdir - 1) < 0.02, (cpred, cdir)


# ---- network -------------------------------------------------------------------

def _theta_zero(K):
    return np.zeros(oracle.mlp_nparams(K))


def _split(theta, K):
    H, F = 64, 12
    o = 0
    parts = {}
    for name, size in (("W1", H * F), ("b1", H), ("W2", H * H), ("b2", H), ("W3", (K + 2) * H),
                       ("b3", K + 2)):
        parts[name] = theta[o:o + size]
        o += size
    assert o == theta.size
    return parts


def test_mlp_param_count():
    assert oracle.mlp_nparams(320) == 64 * 12 + 64 + 64 * 64 + 64 + 322 * 64 + 322 == 25922


def test_mlp_forward_constant_network_is_uniform_mix():
    K = K_SMALL
    th = _theta_zero(K)
    p0 = np.array([0.5, 0.2, 0.1, 0.1, 0.05, 0.05])
    feat = np.random.default_rng(0).normal(size=(3, 12))
    q = oracle.mlp_forward(th, K, np.zeros(12), np.ones(12), feat, p0, mix=0.1)
    np.testing.assert_allclose(q[:, :K], np.broadcast_to(0.9 / K + 0.1 * p0, (3, K)), rtol=1e-15)
    np.testing.assert_allclose(q[:, K:], 0.5, rtol=1e-15)


def test_mlp_forward_chain_through_gelu():
    """One active path: x -> a1 = (x0 - mu) s -> gelu -> gelu -> z_k = c_k v."""
    K = K_SMALL
    th = _theta_zero(K)
    P = _split(th, K)
    P["W1"][0 * 12 + 0] = 1.0
    P["W2"][0 * 64 + 0] = 1.0
    c = np.array([0.3, -1.0, 2.0, 0.0, 0.5, -0.2, 1.5, -0.5])
    P["W3"][np.arange(K + 2) * 64] = c
    fmean = np.full(12, 0.25)
    finv = np.full(12, 2.0)
    feat = np.zeros((1, 12))
    feat[0, 0] = 1.1
    gelu = lambda v: 0.5 * v * (1 + erf(v / math.sqrt(2)))
    v = gelu(gelu((1.1 - 0.25) * 2.0))
    z = c * v
    s = np.exp(z[:K] - z[:K].max())
    s /= s.sum()
    up = 1 / (1 + np.exp(z[K + 1] - z[K]))
    q = oracle.mlp_forward(th, K, fmean, finv, feat, np.full(K, 1.0 / K), mix=0.0)
    np.testing.assert_allclose(q[0, :K], s, rtol=1e-13)
    assert q[0, K] == pytest.approx(up, rel=1e-13)
    assert q[0, K + 1] == pytest.approx(1 - up, rel=1e-13)


def _rand_problem(K, n, seed):
    rng = np.random.default_rng(seed)
    th = rng.normal(scale=0.3, size=oracle.mlp_nparams(K))
    feat = rng.normal(size=(n, 12))
    m = rng.exponential(size=(n, K, 2)) * (rng.random((n, K, 2)) < 0.6)
    p0 = rng.dirichlet(np.ones(K), size=n)
    return th, feat, m, p0


def _rand_cost(K, n, seed):
    rng = np.random.default_rng(seed)
    return rng.exponential(scale=20.0, size=(n, K, 2)) * (rng.random((n, K, 2)) < 0.7)


@pytest.mark.parametrize("with_cost", [False, True])
def test_mlp_gradient_matches_finite_differences(with_cost):
    K, n = K_SMALL, 5
    th, feat, m, p0 = _rand_problem(K, n, 1)
    fmean, finv = np.zeros(12), np.ones(12)
    kw = dict(mix=0.1, cost=_rand_cost(K, n, 3) if with_cost else None, c0=6.0)
    L, gr = oracle.mlp_loss_grad(th, K, fmean, finv, feat, m, p0, **kw)
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(64 * 12, 6, replace=False),              # W1
                          64 * 12 + rng.choice(64, 3, replace=False),           # b1
                          64 * 13 + rng.choice(64 * 64, 6, replace=False),      # W2
                          oracle.mlp_nparams(K) - (K + 2) - (K + 2) * 64 + rng.choice((K + 2) * 64, 6, replace=False),
                          oracle.mlp_nparams(K) - (K + 2) + np.arange(K + 2)])  # b3
    for i in idx:
        e = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[i] += e
        tm[i] -= e
        Lp, _ = oracle.mlp_loss_grad(tp, K, fmean, finv, feat, m, p0, **kw)
        Lm, _ = oracle.mlp_loss_grad(tm, K, fmean, finv, feat, m, p0, **kw)
        fd = (Lp - Lm) / (2 * e)
        assert gr[i] == pytest.approx(fd, rel=2e-5, abs=1e-9), i


def test_mlp_loss_optimum_is_sqrt_of_separable_moments():
    """For m[k][h] = a_k b_h the second moment sum m / (q_k q_h) is smallest at
    q_k ~ sqrt(a_k), q_h ~ sqrt(b_h) (Cauchy-Schwarz), where it equals
    (sum sqrt a)^2 (sum sqrt b)^2 and the gradient vanishes (no mixture)."""
    K = K_SMALL
    a = np.array([4.0, 1.0, 0.25, 9.0, 0.01, 1.0])
    bh = np.array([1.0, 4.0])
    m = (a[:, None] * bh[None, :])[None]
    p0 = np.full((1, K), 1.0 / K)
    th = _theta_zero(K)
    P = _split(th, K)
    P["b3"][:K] = 0.5 * np.log(a)
    P["b3"][K:] = 0.5 * np.log(bh)
    L, gr = oracle.mlp_loss_grad(th, K, np.zeros(12), np.ones(12), np.zeros((1, 12)), m, p0, mix=0.0)
    M2 = (m[0] / (p0[0][:, None] * 0.5)).sum()
    assert L == pytest.approx(np.sqrt(a).sum() ** 2 * np.sqrt(bh).sum() ** 2 / M2, rel=1e-12)
    assert np.abs(gr).max() < 1e-12
    # any other logits give a larger loss
    P["b3"][0] += 0.3
    L2, _ = oracle.mlp_loss_grad(th, K, np.zeros(12), np.ones(12), np.zeros((1, 12)), m, p0, mix=0.0)
    assert L2 > L


def test_mlp_cost_optimum():
    """With cost c[k][h] = g_k and c0 = 0 the spectral part of
    A(q) C(q) = (sum a_k / q_k)(sum g_k q_k)(sum b_h / q_h) is smallest at
    q_k ~ sqrt(a_k / g_k) (Cauchy-Schwarz) with value (sum sqrt(a_k g_k))^2:
    the loss there is the closed form and the gradient vanishes."""
    K = K_SMALL
    a = np.array([4.0, 1.0, 0.25, 9.0, 0.01, 1.0])
    gk = np.array([1.0, 30.0, 2.0, 5.0, 1.0, 0.5])
    bh = np.array([1.0, 4.0])
    m = (a[:, None] * bh[None, :])[None]
    cost = np.broadcast_to(gk[:, None], (K, 2))[None].copy()
    p0 = np.full((1, K), 1.0 / K)
    th = _theta_zero(K)
    P = _split(th, K)
    P["b3"][:K] = 0.5 * np.log(a / gk)
    P["b3"][K:] = 0.5 * np.log(bh)
    kw = dict(mix=0.0, cost=cost, c0=0.0)
    L, gr = oracle.mlp_loss_grad(th, K, np.zeros(12), np.ones(12), np.zeros((1, 12)), m, p0, **kw)
    A0 = (m[0] / (p0[0][:, None] * 0.5)).sum()
    C0 = (cost[0] * (p0[0][:, None] * 0.5)).sum()
    best = np.sqrt(a * gk).sum() ** 2 * np.sqrt(bh).sum() ** 2
    assert L == pytest.approx(best / (A0 * C0), rel=1e-12)
    assert np.abs(gr).max() < 1e-12


def test_mlp_softmax_gradients_sum_to_zero():
    """Shifting all spectral logits (or both hemisphere logits) by a constant
    changes nothing: the b3 gradient sums to zero over each group."""
    K = K_SMALL
    th, feat, m, p0 = _rand_problem(K, 4, 7)
    _, gr = oracle.mlp_loss_grad(th, K, np.zeros(12), np.ones(12), feat, m, p0, mix=0.1)
    gb3 = gr[-(K + 2):]
    scale = np.abs(gb3).max()
    assert abs(gb3[:K].sum()) < 1e-12 * max(scale, 1)
    assert abs(gb3[K:].sum()) < 1e-12 * max(scale, 1)


# ---- Adam ------------------------------------------------------------------------

def test_adam_first_steps_closed_form():
    """With a constant gradient the bias-corrected moments are g and g^2, so
    every step moves theta by lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th, m1, m2 = np.ones(4), np.zeros(4), np.zeros(4)
    for t in (1, 2, 3):
        th_prev = th.copy()
        th, m1, m2 = oracle.adam(th, g, m1, m2, t, lr=0.01, eps=1e-8)
        np.testing.assert_allclose(th, th_prev - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


# ---- integer counts ----------------------------------------------------------------

def test_learned_counts_are_exact_and_close():
    rng = np.random.default_rng(4)
    nb, ng = 40, 8
    q = rng.dirichlet(np.ones(nb * ng) * 0.3)
    q[5] = 0.0
    cn, cg, hemi = oracle.learned_counts(q, nb, ng, 0.3)
    assert cn[-1] == 2**32 and np.all(cg[:, -1] == 2**32)
    pn = np.diff(np.concatenate([[0], cn.astype(np.int64)]))
    wn = q.reshape(nb, ng).sum(1)
    assert np.all(pn >= 1)
    # binary32 decisions: the probabilities, sums and quotient carry relative
    # errors of a few 2^-24 (at most (nb + ng + 3) 2^-24); plus the floors
    p = wn / wn.sum()
    assert np.all(np.abs(pn - p * 2**32) <= (nb + 8 + 3) * 2.0**-24 * p * 2**32 + nb + 1)
    pg = np.diff(np.concatenate([np.zeros((nb, 1), np.int64), cg.astype(np.int64)], axis=1), axis=1)
    assert pg[0, 5] == 0 and np.all(pg.reshape(-1)[q > 0] >= 1)
    assert hemi == int(math.floor(0.3 * 2**23 + 0.5))
    assert oracle.learned_counts(q, nb, ng, 0.0)[2] == 1
    assert oracle.learned_counts(q, nb, ng, 1.0)[2] == 2**23 - 1


def _gamma(n):
    """Higham's gamma_n = n u / (1 - n u), u = 2^-24 (binary32 unit roundoff): the
    relative error bound of a recursive sum of n + 1 nonnegative terms."""
    from fractions import Fraction
    u = Fraction(1, 2**24)
    return n * u / (1 - n * u)


def test_learned_counts_against_exact_rationals():
    """The binary32 count rule against exact rational arithmetic on the same
    binary32-rounded inputs x_k = RN32(q_k).  For K nonnegative weights summed in
    order, |fl(sum) - sum| <= gamma_(K-1) sum; the quotient adds one rounding
    (1 + delta, |delta| <= u) and the floor at most one count.  So a count m_k of
    a weight with exact share r_k = x_k / sum x obeys

        |m_k - 2^32 r_k| <= 2^32 r_k e + 1,  e = (1 + u) / (1 - gamma) - 1

    (e bounds the larger side: (1 - u) / (1 + gamma) >= 1 - e), except the
    remainder bin (the first largest weight), whose error is at most the sum of
    the others'.  The band level compounds the in-band sums (gamma_(ng - 1)) and
    the sum over bands (gamma_(nb - 1)).  A wrong order of rounding, a dropped
    floor or a misplaced remainder breaks these bounds by whole counts."""
    from fractions import Fraction
    rng = np.random.default_rng(41)
    u = Fraction(1, 2**24)
    for nb, ng, alpha in ((40, 8, 0.3), (7, 5, 2.0), (3, 2, 0.05)):
        q = rng.dirichlet(np.ones(nb * ng) * alpha)
        q[rng.integers(0, nb * ng, 3)] = 0.0
        cn, cg, _ = oracle.learned_counts(q, nb, ng, 0.5)
        x = [Fraction(float(np.float32(v))) for v in q]
        pg = np.diff(np.concatenate([np.zeros((nb, 1), np.int64), cg.astype(np.int64)], axis=1), axis=1)
        ga = _gamma(ng - 1)
        e_g = (1 + u) / (1 - ga) - 1
        band = []
        for n in range(nb):
            xs = x[n * ng:(n + 1) * ng]
            s = sum(xs)
            band.append(s)
            if s == 0:  # never drawn: uniform counts
                assert np.all(np.abs(pg[n] - 2**32 / ng) <= ng)
                continue
            kmax = int(np.argmax(np.array([float(v) for v in xs])))
            for k in range(ng):
                target = Fraction(2**32) * xs[k] / s
                if xs[k] == 0:
                    assert pg[n, k] == 0
                elif k != kmax:
                    assert abs(pg[n, k] - target) <= target * e_g + 1, (n, k)
            others = sum(Fraction(2**32) * xs[k] / s * e_g + 1 for k in range(ng) if k != kmax)
            assert abs(pg[n, kmax] - Fraction(2**32) * xs[kmax] / s) <= others
        # bands: in-band binary32 sums, then their binary32 sum, then the quotient
        gb = _gamma(nb - 1)
        e_n = (1 + ga) * (1 + u) / ((1 - ga) * (1 - gb)) - 1
        W = sum(band)
        pn = np.diff(np.concatenate([[0], cn.astype(np.int64)]))
        kmax = int(np.argmax(np.array([float(np.float32(sum(np.float32(v) for v in
                                                              q[n * ng:(n + 1) * ng])))
                                       for n in range(nb)])))
        others = 0
        for n in range(nb):
            target = Fraction(2**32) * band[n] / W
            if n == kmax:
                continue
            assert abs(pn[n] - target) <= target * e_n + 1, n
            others += target * e_n + 1
        assert abs(pn[kmax] - Fraction(2**32) * band[kmax] / W) <= others
        # the counts are exact partitions of 2^32
        assert int(cn[-1]) == 2**32 and np.all(cg[:, -1] == 2**32)


def test_learned_counts_reproduce_dyadic_probabilities():
    """Probabilities that are multiples of 2^-24 (one band: exact in binary32, and
    so are all their partial sums below 1) come back as the same counts."""
    rng = np.random.default_rng(5)
    c = rng.integers(1, 2**18, size=8).astype(np.int64) * 2**8
    c[-1] += 2**32 - c.sum()
    q = c.astype(np.float64) / 2.0**32
    cn, cg, _ = oracle.learned_counts(q, 1, 8, 0.5)
    np.testing.assert_array_equal(cg[0], np.cumsum(c).astype(np.uint64))
    assert cn[0] == 2**32


def test_skewed_cell_proposal_is_unbiased_against_quadrature():
    """Per-cell proposals far from the plain one (spectral points re-weighted,
    70/30 hemisphere split) leave the estimate unbiased: the MC mean matches the
    deterministic angular quadrature of the same estimand (centre origin)."""
    grid = inputs.Grid(4, 8, 4, 2.0, 2.0, 2.0, T_wall=(500.0, 1000.0))
    kd = inputs.make_kdist(3, n_bands=3, n_g=2)
    T, x = inputs.channel_fields(grid, 16, fluct=0.15, x_mode="field")
    nc, nb, ng = grid.ncells, kd.n_bands, kd.n_g
    rng = np.random.default_rng(23)
    cn = np.zeros((nc, nb), np.uint64)
    cg = np.zeros((nc, nb * ng), np.uint64)
    hemi = np.zeros(nc, np.uint32)
    for c in range(nc):
        q = rng.dirichlet(np.ones(nb * ng))
        a, b, h = oracle.learned_counts(0.8 * q + 0.2 / (nb * ng), nb, ng, 0.7 if c % 2 else 0.3)
        cn[c], cg[c], hemi[c] = a, b.reshape(-1), h
    q_quad = oracle.quadrature(grid, kd, T, x, nmu_panels=48, nmu_per_panel=4, nphi=192,
                               origin=1, tol=1e-12)
    res = oracle.solve(grid, kd, T, x, rays=4096, seed=29, tol=1e-12, origin=1,
                       proposal=(cn, cg, hemi))
    z = (res["q"].reshape(-1) - q_quad) / res["sigma"].reshape(-1)
    assert np.max(np.abs(z)) < 4.5, np.round(z, 2)
    assert np.sqrt(np.mean(z**2)) < 1.4


def test_batch_time_ratio_mode():
    """Mode 1: one sample gives the per-cell ratio (mode 0); the loss and its
    gradient do not depend on the scale of the weights; and the gradient
    matches central finite differences."""
    K, n = K_SMALL, 6
    th, feat, m, p0 = _rand_problem(K, n, 9)
    cost = _rand_cost(K, n, 10)
    w = np.random.default_rng(11).uniform(0.1, 3.0, n)
    z12, o12 = np.zeros(12), np.ones(12)
    L0, g0 = oracle.mlp_loss_grad(th, K, z12, o12, feat[:1], m[:1], p0[:1], cost=cost[:1], c0=2.0)
    L1, g1 = oracle.mlp_loss_grad(th, K, z12, o12, feat[:1], m[:1], p0[:1], cost=cost[:1], c0=2.0,
                                  wgt=w[:1], mode=1)
    assert L1 == pytest.approx(L0, rel=1e-12)
    np.testing.assert_allclose(g1, g0, rtol=1e-10, atol=1e-14)
    kw = dict(cost=cost, c0=2.0, mode=1)
    La, ga = oracle.mlp_loss_grad(th, K, z12, o12, feat, m, p0, wgt=w, **kw)
    Lb, gb = oracle.mlp_loss_grad(th, K, z12, o12, feat, m, p0, wgt=7.5 * w, **kw)
    assert Lb == pytest.approx(La, rel=1e-12)
    np.testing.assert_allclose(gb, ga, rtol=1e-10, atol=1e-14)
    rng = np.random.default_rng(12)
    for i in np.concatenate([rng.choice(64 * 12, 4, replace=False),
                             oracle.mlp_nparams(K) - (K + 2) + np.arange(K + 2)]):
        e = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[i] += e
        tm[i] -= e
        Lp, _ = oracle.mlp_loss_grad(tp, K, z12, o12, feat, m, p0, wgt=w, **kw)
        Lm, _ = oracle.mlp_loss_grad(tm, K, z12, o12, feat, m, p0, wgt=w, **kw)
        assert ga[i] == pytest.approx((Lp - Lm) / (2 * e), rel=2e-5, abs=1e-9), i
