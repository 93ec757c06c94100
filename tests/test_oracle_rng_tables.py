"""Oracle pins: the counter-based generator, the table lookup and the quantised pdfs.

The paper draws R_theta, R_phi, R_n, R_g uniformly on (0, 1) (Eq. 9, Eq. 17,
Algorithm 1 "Initialize") and interpolates its property tables linearly in T
(Section 2.2).  These tests hold the oracle to properties that independent
routines (numpy, scipy) or the mathematics fix.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1810_00188_gb300 import inputs


def _draws(n, block=0, snap=0, key=(0, 0)):
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n) % 4096
    ctr[:, 1] = np.arange(n) // 4096
    ctr[:, 2] = block
    ctr[:, 3] = snap
    return oracle.philox(ctr, key)


@pytest.mark.parametrize("ctr,key,expect", [
    # Known-answer vectors published with the reference implementation of the
    # generator (Random123, Salmon et al., SC'11): Philox4x32 with 10 rounds on an
    # all-zero input, an all-ones input, and the hexadecimal digits of pi
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
])
def test_philox4x32_10_known_answers(ctr, key, expect):
    """The generator's identity: the multipliers, the Weyl key increments, the
    word permutation and the round count are fixed by these outputs (a single
    wrong constant or round changes every word)."""
    out = oracle.philox(np.array(ctr, dtype=np.uint32), np.array(key, dtype=np.uint32))
    assert tuple(int(v) for v in out[0]) == expect


def test_philox_words_uniform_chi2():
    w = _draws(1 << 18)
    for lane in range(4):
        h = np.bincount((w[:, lane] >> 24).astype(np.int64), minlength=256)
        chi2 = ((h - h.mean()) ** 2 / h.mean()).sum()
        # 255 dof: mean 255, sd ~22.6; 5 sd band
        assert 140 < chi2 < 370, (lane, chi2)


def test_philox_bits_balanced_and_lanes_independent():
    w = _draws(1 << 16).astype(np.uint64)
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint64)) & 1).astype(np.float64)
    p = bits.mean(axis=0)
    assert np.all(np.abs(p - 0.5) < 5 * 0.5 / np.sqrt(w.shape[0]))
    u = oracle.uniform(w.astype(np.uint32))
    c = np.corrcoef(u.T)
    off = c[~np.eye(4, dtype=bool)]
    assert np.all(np.abs(off) < 5 / np.sqrt(w.shape[0]))


def test_philox_counter_and_key_sensitivity():
    base = _draws(4096)
    other_block = _draws(4096, block=1)
    other_snap = _draws(4096, snap=1)
    other_key = _draws(4096, key=(1, 0))
    for alt in (other_block, other_snap, other_key):
        # distinct streams: no word agrees beyond chance, and values uncorrelated
        assert np.mean(alt == base) < 1e-3
        r = np.corrcoef(oracle.uniform(base[:, 0]), oracle.uniform(alt[:, 0]))[0, 1]
        assert abs(r) < 5 / np.sqrt(4096)


def test_philox_uniformity_ks_and_serial_pairs():
    u = oracle.uniform(_draws(1 << 15)[:, 2])
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    # successive counters: 2D pairs uniform on a 16x16 grid
    h, _, _ = np.histogram2d(u[:-1], u[1:], bins=16, range=[[0, 1], [0, 1]])
    chi2 = ((h - h.mean()) ** 2 / h.mean()).sum()
    assert stats.chi2.sf(chi2, 255) > 1e-4


def test_uniform_mapping_open_interval_exact():
    w = np.array([0, 511, 512, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    u = oracle.uniform(w)
    assert u[0] == 0.5 * 2.0**-23 and u[1] == u[0]
    assert u[2] == 1.5 * 2.0**-23
    assert u[3] == 1.0 - 0.5 * 2.0**-23
    assert u[4] == 0.5 + 0.5 * 2.0**-23
    assert np.all((u > 0) & (u < 1))
    # every value of the 23-bit grid (plus 1/2) is exact in binary32 and binary64
    allw = (np.arange(0, 1 << 23, 977, dtype=np.uint64) << np.uint64(9)).astype(np.uint32)
    ua = oracle.uniform(allw)
    assert np.all(ua.astype(np.float32).astype(np.float64) == ua)
    assert np.all(np.array([oracle.lib().orc_uniform(int(v)) for v in allw[:64]]) == ua[:64])


def test_interp_matches_numpy_inside_and_clamps_outside():
    rng = np.random.default_rng(3)
    v = rng.uniform(0.1, 10.0, 17)
    T0, dT = 300.0, 20.0
    nodes = T0 + dT * np.arange(v.size)
    for T in list(rng.uniform(300.0, 620.0, 50)) + list(nodes):
        assert oracle.interp(v, T0, dT, T) == pytest.approx(np.interp(T, nodes, v), rel=1e-13, abs=1e-13)
    assert oracle.interp(v, T0, dT, 100.0) == v[0]
    assert oracle.interp(v, T0, dT, 5000.0) == pytest.approx(v[-1], rel=1e-15)


def test_quantize_counts_properties():
    rng = np.random.default_rng(5)
    for K in (1, 2, 8, 40, 320):
        w = rng.uniform(0, 1, K) ** 8
        w[rng.integers(0, K, max(1, K // 10))] = 0.0
        if not np.any(w > 0):
            w[0] = 1.0
        cum = oracle.quantize(w)
        m = np.diff(np.concatenate([[0], cum.astype(np.int64)]))
        assert cum[-1] == 2**32
        assert np.all(m >= 0)
        assert np.all((m >= 1) == (w > 0))  # positive weight <=> drawable
        target = w / w.sum() * 2.0**32
        # every count within one count of its target except the remainder bin
        big = np.argmax(w)
        others = np.delete(np.abs(m - target), big)
        assert np.all(others <= 1.0 + 1e-6)
        assert abs(m[big] - target[big]) <= K + 1
    with pytest.raises(ValueError):
        oracle.quantize(np.zeros(4))


def test_plain_proposal_follows_planck_tmax_pdf():
    """f_n ~ B_n(T_max) sum_g w_g k_{n,g}(T_max), f_g(n) ~ w_g k_{n,g} (Eqs. 13, 16)."""
    grid, kd, T, x = inputs.nongrey_channel(8, 8, 8, seed=1)
    cn, cg, tmax = oracle.plain_proposal(grid, kd, T, x)
    assert tmax == pytest.approx(max(T.max(), 1000.0))
    nodes = kd.T_nodes()
    k_m = np.array([[np.interp(tmax, nodes, kd.kappa[n, g]) for g in range(kd.n_g)]
                    for n in range(kd.n_bands)])
    B_m = np.array([np.interp(tmax, nodes, kd.B[n]) for n in range(kd.n_bands)])
    fn = B_m * (kd.w_g[None, :] * k_m).sum(1)
    fn /= fn.sum()
    pn = np.diff(np.concatenate([[0], cn.astype(np.int64)])) / 2.0**32
    assert np.allclose(pn, fn, atol=2 * kd.n_bands / 2.0**32, rtol=1e-9)
    for n in range(kd.n_bands):
        fg = kd.w_g * k_m[n] / (kd.w_g * k_m[n]).sum()
        pg = np.diff(np.concatenate([[0], cg[n].astype(np.int64)])) / 2.0**32
        assert np.allclose(pg, fg, atol=2 * kd.n_g / 2.0**32, rtol=1e-9)


def test_sampled_band_frequencies_match_quantised_pdf():
    """Drawing n from R_n and g from R_g (Eq. 17) reproduces p(n, g)."""
    grid, kd, T, x = inputs.nongrey_channel(8, 8, 8, seed=2)
    cn, cg, _ = oracle.plain_proposal(grid, kd, T, x)
    w = _draws(1 << 17)
    n = np.searchsorted(cn, w[:, 2].astype(np.uint64), side="right")
    g = np.array([np.searchsorted(cg[a], b, side="right") for a, b in zip(n, w[:, 3].astype(np.uint64))])
    pn = np.diff(np.concatenate([[0], cn.astype(np.int64)])) / 2.0**32
    hn = np.bincount(n, minlength=kd.n_bands)
    keep = pn * w.shape[0] > 20
    chi2 = ((hn[keep] - pn[keep] * w.shape[0]) ** 2 / (pn[keep] * w.shape[0])).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4
    assert np.all(g < kd.n_g)
