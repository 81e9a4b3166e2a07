"""Pins of the oracle's discrete step-frequency set (Sec. V: the frequency takes
one of a few values, drawn uniformly; the Naive optimiser keeps one force
Gaussian per frequency): the draw against exact rational arithmetic and
uniformity, the one-value set against the fixed-frequency path it must reduce
to, and the per-frequency Naive update against a brute-force sort."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2403_11383_b300 import workloads as W


def _cfg(**kw):
    c = W.config("naive_freqset_k10000_h12")
    c.update(K=64, H=6)
    c.update(kw)
    return c


def test_bin_is_the_interval_holding_the_uniform(orc):
    # sample k's entry b satisfies b / n <= u < (b + 1) / n for the 24-bit uniform
    # u of the frequency draw's first Philox word (exact rationals)
    seed, ctrl, it = 9, 4, (3 << 32) + 11
    for n in (1, 2, 3, 5, 8):
        for k in range(0, 4000, 7):
            w = orc.philox4x32_10([k, 0, it & 0xffffffff, it >> 32], [seed, ctrl])
            u = Fraction(int(w[0]) >> 8, 1 << 24)
            b = orc.freq_bin(seed, ctrl, k, it, n)
            assert 0 <= b < n
            assert Fraction(b, n) <= u < Fraction(b + 1, n), (n, k, b, u)


def test_bins_are_uniform(orc):
    N, n = 90_000, 3
    b = np.array([orc.freq_bin(1, 2, k, 5, n) for k in range(N)])
    counts = np.bincount(b, minlength=n)
    sd = np.sqrt(N * (1 / n) * (1 - 1 / n))
    assert np.all(np.abs(counts - N / n) < 5 * sd), counts
    # consecutive samples are not correlated in their entries
    same = np.mean(b[1:] == b[:-1])
    assert abs(same - 1 / n) < 5 * np.sqrt((1 / n) * (1 - 1 / n) / (N - 1))


def test_one_value_set_reduces_to_the_fixed_frequency(orc):
    # a set of one frequency f is the fixed-frequency controller at q_init = f,
    # plus the regulariser rho (f - f_n)^2 on every cost (Sec. V)
    for P_knots in (0, 3):
        cs = _cfg(P=P_knots, freq_set_mhz=(2000,), q_init=1300)
        cf = _cfg(P=P_knots, q_init=2000)
        cf.pop("freq_set_mhz")
        ps, pf = orc.make_params(cs), orc.make_params(cf)
        pr = W.problem(cs)
        g = orc.make_gait(pr["gait"])
        ms, vs = orc.init_dist(ps, g)
        mf, vf = orc.init_dist(pf, g)
        np.testing.assert_array_equal(ms, mf)
        np.testing.assert_array_equal(vs, vf)
        ms2, vs2 = orc.warm_shift(ps, g, 2, ms, vs)
        mf2, vf2 = orc.warm_shift(pf, g, 2, mf, vf)
        np.testing.assert_array_equal(ms2, mf2)
        np.testing.assert_array_equal(vs2, vf2)
        Js, qs, ths, _ = orc.rollout(ps, g, pr["x0"], pr["xref"], pr["f_ext"], ms, vs, 3, want_theta=True)
        Jf, qf, thf, _ = orc.rollout(pf, g, pr["x0"], pr["xref"], pr["f_ext"], mf, vf, 3, want_theta=True)
        np.testing.assert_array_equal(ths, thf)
        assert np.all(qs == 2000) and np.all(qf == 2000)
        reg = cs["cost"]["rho"] * (2.0 - cs["cost"]["f_nominal"]) ** 2
        fin = np.isfinite(Jf)
        np.testing.assert_array_equal(Js[fin], Jf[fin] + reg)
        assert np.array_equal(np.isfinite(Js), fin)


def test_each_block_is_the_single_frequency_distribution(orc):
    # block b of a multi-value set starts, and warm-shifts, like a fixed-frequency
    # controller at that frequency
    cs = _cfg(H=20, freq_set_mhz=(1300, 2000, 2400))
    ps = orc.make_params(cs)
    pr = W.problem(cs)
    g = orc.make_gait(pr["gait"])
    assert orc.dim(ps) == 3 * 12 * 20 and orc.sample_dim(ps) == 12 * 20
    m, v = orc.init_dist(ps, g)
    rng = np.random.default_rng(0)
    m = m + rng.normal(size=m.size)  # a non-trivial distribution to shift
    m2, v2 = orc.warm_shift(ps, g, 3, m, v)
    nf = 12 * 20
    for b, f in enumerate(cs["freq_set_mhz"]):
        cf = _cfg(H=20, q_init=f)
        cf.pop("freq_set_mhz")
        pf = orc.make_params(cf)
        mf, vf = orc.init_dist(pf, g)
        np.testing.assert_array_equal(orc.init_dist(ps, g)[0][b * nf:(b + 1) * nf], mf)
        mf2, vf2 = orc.warm_shift(pf, g, 3, m[b * nf:(b + 1) * nf], v[b * nf:(b + 1) * nf])
        np.testing.assert_array_equal(m2[b * nf:(b + 1) * nf], mf2)
        np.testing.assert_array_equal(v2[b * nf:(b + 1) * nf], vf2)
    # the frequencies change the nominal contact schedule, hence the tails differ
    assert not np.array_equal(orc.init_dist(ps, g)[0][:nf], orc.init_dist(ps, g)[0][2 * nf:])


def test_samples_draw_from_their_frequency_gaussian(orc):
    cs = _cfg(K=300, freq_set_mhz=(1300, 2000, 2400))
    ps = orc.make_params(cs)
    pr = W.problem(cs)
    g = orc.make_gait(pr["gait"])
    nf = 12 * cs["H"]
    m = np.concatenate([np.full(nf, 10.0 * (b + 1)) for b in range(3)])
    v = np.concatenate([np.full(nf, 0.25 * (b + 1)) for b in range(3)])
    J, q, th, _ = orc.rollout(ps, g, pr["x0"], pr["xref"], pr["f_ext"], m, v, 2, want_theta=True)
    for k in range(cs["K"]):
        b = orc.freq_bin(cs["seed"], cs["ctrl"], k, 2, 3)
        assert q[k] == cs["freq_set_mhz"][b]
        eps = np.array([orc.normal(cs["seed"], cs["ctrl"], k, n, 2) for n in range(nf)])
        np.testing.assert_allclose(th[k], 10.0 * (b + 1) + np.sqrt(0.25 * (b + 1)) * eps, rtol=1e-15, atol=1e-13)


def _brute_naive(J, q, th, fs, mean, nf):
    mean = mean.copy()
    winners = []
    for b, f in enumerate(fs):
        idx = np.nonzero((q == f) & np.isfinite(J))[0]
        if idx.size == 0:
            winners.append(-1)
            continue
        order = np.lexsort((idx, J[idx]))  # by cost, then index
        w = int(idx[order[0]])
        winners.append(w)
        mean[b * nf:(b + 1) * nf] = th[w, :nf]
    cand = [(J[w], w, b) for b, w in enumerate(winners) if w >= 0]
    bs = min(cand)[2] if cand else -1
    return bs, np.array(winners, dtype=np.int32), mean


def test_naive_sets_against_brute_force(orc):
    fs = (1300, 2000, 2400)
    cs = _cfg(K=200, H=2, freq_set_mhz=fs)
    ps = orc.make_params(cs)
    nf = 24
    rng = np.random.default_rng(3)
    for trial in range(20):
        J = rng.integers(0, 15, size=200).astype(float)  # many ties
        J[rng.random(200) < 0.2] = np.inf
        q = rng.choice(fs, size=200).astype(np.uint32)
        if trial == 1:
            q[q == 2000] = 1300  # one frequency drawn by nobody
        if trial == 2:
            J[q == 2400] = np.inf  # one frequency with only non-finite costs
        th = rng.normal(size=(200, nf))
        mean = rng.normal(size=3 * nf)
        bs, best, m = orc.naive_sets(ps, J, q, th, mean)
        bs0, best0, m0 = _brute_naive(J, q, th, fs, mean, nf)
        assert bs == bs0
        np.testing.assert_array_equal(best, best0)
        np.testing.assert_array_equal(m, m0)
    bs, best, m = orc.naive_sets(ps, np.full(200, np.inf), q, th, mean)
    assert bs == -1 and np.all(best == -1)
    np.testing.assert_array_equal(m, mean)  # nothing finite: every mean kept


def test_solve_reports_the_best_frequency(orc):
    fs = (1300, 2000, 2400)
    cs = _cfg(K=96, H=8, iterations=2, freq_set_mhz=fs)
    ps = orc.make_params(cs)
    pr = W.problem(cs)
    g = orc.make_gait(pr["gait"])
    m0, v0 = orc.init_dist(ps, g)
    r = orc.solve(ps, g, pr["x0"], pr["xref"], pr["f_ext"], 0, 7, m0, v0)
    assert r["status"] == orc.OK
    # re-run the last iteration by hand from the first iteration's update
    J0, q0, th0, _ = orc.rollout(ps, g, pr["x0"], pr["xref"], pr["f_ext"], m0, v0, 7, want_theta=True)
    _, _, m1 = orc.naive_sets(ps, J0, q0, th0, m0)
    J1, q1, th1, _ = orc.rollout(ps, g, pr["x0"], pr["xref"], pr["f_ext"], m1, v0, 8, want_theta=True)
    bs, best, m2 = orc.naive_sets(ps, J1, q1, th1, m1)
    np.testing.assert_array_equal(r["J"], J1)
    np.testing.assert_array_equal(r["mean"], m2)
    np.testing.assert_array_equal(r["var"], v0)  # Naive keeps the covariance
    np.testing.assert_array_equal(r["elite"][:3], best)
    kbest = int(np.lexsort((np.arange(96), J1))[0])
    assert fs[bs] == q1[kbest] and r["f_mean"] == pytest.approx(fs[bs] / 1000.0)
    assert r["beta"] == J1[kbest]
    nf = 12 * 8
    np.testing.assert_array_equal(r["u0"], orc.first_control(ps, g, m2[bs * nf:(bs + 1) * nf]))
    np.testing.assert_array_equal(m2[bs * nf:(bs + 1) * nf], th1[kbest])
