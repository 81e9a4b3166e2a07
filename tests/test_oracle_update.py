"""Pins of the oracle's distribution updates (MPPI, elite, Naive), initial
distribution, warm start and whole rollouts against invariants, special cases,
library routines and closed forms."""
import copy

import numpy as np
import pytest
from scipy.special import softmax

from paper_2403_11383_b300 import workloads as W


# ------------------------------------------------------------------ MPPI (Alg. 5)

def test_mppi_matches_softmax_weights(orc):
    rng = np.random.default_rng(0)
    J = rng.uniform(0, 5, size=300)
    th = rng.normal(size=(300, 7))
    for lam in (0.1, 1.0, 3.0):
        st, mean, ess, beta = orc.mppi(J, th, lam)
        w = softmax(-J / lam)
        assert st == orc.OK and beta == J.min()
        assert abs(w.sum() - 1.0) < 1e-12
        np.testing.assert_allclose(mean, w @ th, rtol=1e-12, atol=1e-13)
        assert ess == pytest.approx(1.0 / np.sum(w * w), rel=1e-12)


def test_mppi_limits_and_invariance(orc):
    rng = np.random.default_rng(1)
    J = rng.uniform(0, 5, size=100)
    J[40] = J[17] = J.min() - 1.0  # two tied best samples
    th = rng.normal(size=(100, 5))
    # lambda -> 0: the argmin, and on ties the equal-weight mean of the tied samples
    _, m0, ess0, _ = orc.mppi(J, th, 1e-8)
    np.testing.assert_allclose(m0, 0.5 * (th[17] + th[40]), atol=1e-12)
    assert ess0 == pytest.approx(2.0)
    J2 = J.copy()
    J2[40] += 1e-3
    _, m1, _, _ = orc.mppi(J2, th, 1e-8)
    np.testing.assert_allclose(m1, th[17], atol=1e-12)
    # lambda -> infinity: the plain sample mean
    _, minf, essinf, _ = orc.mppi(J, th, 1e9)
    np.testing.assert_allclose(minf, th.mean(axis=0), atol=1e-8)
    assert essinf == pytest.approx(100, rel=1e-6)
    # invariant to a constant added to every cost
    _, ma, _, _ = orc.mppi(J, th, 0.7)
    _, mb, _, _ = orc.mppi(J + 123.0, th, 0.7)
    np.testing.assert_allclose(ma, mb, atol=1e-12)
    # K = 1 returns its own sample
    _, m, ess, _ = orc.mppi(J[:1], th[:1], 0.1)
    np.testing.assert_allclose(m, th[0], atol=0)
    assert ess == 1.0


def test_mppi_ignores_infinite_costs_and_reports_divergence(orc):
    th = np.arange(12.0).reshape(4, 3)
    J = np.array([np.inf, 2.0, np.inf, 2.0])
    st, m, _, _ = orc.mppi(J, th, 0.1)
    np.testing.assert_allclose(m, 0.5 * (th[1] + th[3]))
    st, _, _, _ = orc.mppi(np.full(4, np.inf), th, 0.1)
    assert st == orc.DIVERGED


# ------------------------------------------------------------------ elite (Alg. 1)

def test_elite_select_matches_lexsort(orc):
    rng = np.random.default_rng(2)
    for K, Ke in ((1000, 50), (333, 333), (64, 1), (5000, 410)):
        J = np.round(rng.uniform(0, 3, size=K), 2)  # many exact ties
        J[rng.integers(0, K, size=5)] = np.nan
        J[rng.integers(0, K, size=5)] = np.inf
        idx = orc.elite_select(J, Ke)
        key = np.where(np.isnan(J), np.inf, J)
        order = np.lexsort((np.arange(K), key))
        np.testing.assert_array_equal(idx, order[:Ke])


def test_elite_refit_special_cases(orc):
    rng = np.random.default_rng(3)
    th = rng.normal(size=(200, 6)) * 3 + 1
    floor = np.full(6, 0.01)
    mean, var = orc.elite_refit(th, np.arange(200), floor)
    np.testing.assert_allclose(mean, th.mean(axis=0), atol=1e-13)
    np.testing.assert_allclose(var, th.var(axis=0, ddof=0), rtol=1e-12)
    # one elite: its own sample, variance at the floor
    mean, var = orc.elite_refit(th, np.array([42]), floor)
    np.testing.assert_array_equal(mean, th[42])
    np.testing.assert_array_equal(var, floor)
    # subset: mean/variance of exactly those rows
    sub = np.array([3, 9, 150, 77])
    mean, var = orc.elite_refit(th, sub, floor)
    np.testing.assert_allclose(mean, th[sub].mean(axis=0), atol=1e-13)
    np.testing.assert_allclose(var, np.maximum(th[sub].var(axis=0), floor), rtol=1e-12)


# ------------------------------------------------------------------ initial distribution / warm start

def test_init_distribution_hover(orc):
    c = W.config("plain_mppi_k512_h12")
    P = orc.make_params(c)
    g = orc.make_gait(W.gait("trot", 123_456_789))
    mean, var = orc.init_dist(P, g)
    assert mean.size == 12 * 12
    mg = 21.0 * 9.81
    for j in range(12):
        n = sum(orc.stance(g, i, 2000, 20000, j) for i in range(4))
        mz = mean.reshape(12, 4, 3)[j, :, 2]
        np.testing.assert_allclose(mz, mg / n)
        np.testing.assert_array_equal(mean.reshape(12, 4, 3)[j, :, :2], 0)
    np.testing.assert_array_equal(var, 400.0)


def test_warm_shift_per_step(orc):
    c = W.config("adaptive_elite_k8192_h25")
    P = orc.make_params(c)
    g = orc.make_gait(W.gait("trot", 0))
    rng = np.random.default_rng(4)
    D = orc.dim(P)
    mean, var = rng.normal(size=D), rng.uniform(1, 2, size=D)
    m2, v2 = orc.warm_shift(P, g, 2, mean, var)
    np.testing.assert_array_equal(m2[: 12 * 23], mean[24: 12 * 25])
    np.testing.assert_array_equal(v2[: 12 * 23], var[24: 12 * 25])
    # frequency entry untouched; tail takes the initial rule under the new phase
    assert m2[-1] == mean[-1] and v2[-1] == var[-1]
    mi, vi = orc.init_dist(P, g)
    np.testing.assert_array_equal(m2[12 * 23: 12 * 25], mi[12 * 23: 12 * 25])
    np.testing.assert_array_equal(v2[12 * 23: 12 * 25], vi[12 * 23: 12 * 25])
    m0, v0 = orc.warm_shift(P, g, 0, mean, var)
    np.testing.assert_array_equal(m0, mean)


def test_warm_shift_spline_is_time_shift(orc):
    c = W.config("spline_k262144_h100")
    P = orc.make_params(c)
    g = orc.make_gait(W.gait("trot", 0))
    rng = np.random.default_rng(5)
    D = orc.dim(P)
    mean, var = rng.normal(size=D), rng.uniform(1, 2, size=D)
    m1, v1 = orc.warm_shift(P, g, 1, mean, var)
    np.testing.assert_array_equal(v1, var)
    # a linear-in-time knot sequence stays linear: shifted by one step, and the
    # last knot holds the end value
    dt, H = 0.01, 100
    tk = np.linspace(0, (H - 1) * dt, 4)
    lin = np.zeros(D)
    for p in range(4):
        lin[12 * p: 12 * p + 12] = 5.0 + 2.0 * tk[p]
    l1, _ = orc.warm_shift(P, g, 1, lin, var)
    for p in range(4):
        t = min(tk[p] + dt, tk[-1])
        np.testing.assert_allclose(l1[12 * p: 12 * p + 12], 5.0 + 2.0 * t, atol=1e-12)


# ------------------------------------------------------------------ whole rollouts

def _zero_noise(c):
    c = copy.deepcopy(c)
    c["sigma_init"] = 0.0
    return c


def test_rollout_zero_noise_all_samples_equal(orc):
    c = _zero_noise(W.config("plain_mppi_k512_h12"))
    c["K"] = 64
    P = orc.make_params(c)
    pr = W.problem(c)
    g = orc.make_gait(pr["gait"])
    mean, var = orc.init_dist(P, g)
    J, q, th, _ = orc.rollout(P, g, pr["x0"], pr["xref"], None, mean, var, 0, want_theta=True)
    assert np.all(J == J[0]) and np.all(th == mean)
    st, m, ess, _ = orc.mppi(J, th, 0.1)
    np.testing.assert_allclose(m, mean, atol=1e-12)
    assert ess == pytest.approx(64)


def test_rollout_ballistic_cost_closed_form(orc):
    # duty 0: every leg always in swing, so forces are zeroed and the body flies.
    # The cost is charged on x_0 .. x_{H-1} of the closed-form flight (Alg. 2).
    c = W.config("plain_mppi_k512_h12")
    c["K"] = 8
    P = orc.make_params(c)
    g = orc.make_gait({"offset": (0, 0, 0, 0), "duty": 0, "phase0": 0})
    pr = W.problem(c)
    x0, xref = pr["x0"].copy(), pr["xref"]
    x0[3:6] = 0
    x0[9:12] = 0
    mean, var = orc.init_dist(P, g)
    J, _, _, _ = orc.rollout(P, g, x0, xref, None, np.full_like(mean, 50.0), var, 0)
    Q = np.array(W.COST["Q"])
    dt, gz = 0.02, -9.81
    want = 0.0
    for j in range(12):
        x = x0.copy()
        x[0:3] = x0[0:3] + x0[6:9] * j * dt + np.array([0, 0, gz]) * dt * dt * j * (j - 1) / 2
        x[6:9] = x0[6:9] + np.array([0, 0, gz]) * j * dt
        want += np.sum(Q * (x - xref[j]) ** 2)
    np.testing.assert_allclose(J, want, rtol=1e-12)


@pytest.mark.parametrize("w_t", [0.0, 2.5])
def test_terminal_cost_on_the_flight_closed_form(orc, w_t):
    # the optional terminal cost charges x_H (the state after the last step)
    # against the last reference, weighted by w_t, on top of Alg. 2's stage costs
    c = copy.deepcopy(W.config("plain_mppi_k512_h12"))
    c["K"] = 4
    c["cost"] = dict(c["cost"], w_terminal=w_t)
    P = orc.make_params(c)
    g = orc.make_gait({"offset": (0, 0, 0, 0), "duty": 0, "phase0": 0})
    pr = W.problem(c)
    x0, xref = pr["x0"].copy(), pr["xref"]
    x0[3:6] = 0
    x0[9:12] = 0
    mean, var = orc.init_dist(P, g)
    J, _, _, _ = orc.rollout(P, g, x0, xref, None, mean, var, 0)
    Q = np.array(W.COST["Q"])
    dt, gz = 0.02, -9.81

    def flight(j):
        x = x0.copy()
        x[0:3] = x0[0:3] + x0[6:9] * j * dt + np.array([0, 0, gz]) * dt * dt * j * (j - 1) / 2
        x[6:9] = x0[6:9] + np.array([0, 0, gz]) * j * dt
        return x

    want = sum(np.sum(Q * (flight(j) - xref[j]) ** 2) for j in range(12))
    want += w_t * np.sum(Q * (flight(12) - xref[11]) ** 2)
    np.testing.assert_allclose(J, want, rtol=1e-12)


def test_rollout_hover_cost_closed_form(orc):
    # duty 1: all legs in stance; zero noise, vertical m|g|/4 per leg, level body
    # at rest: the state never moves, J = H (state error + force cost)
    c = _zero_noise(W.config("plain_mppi_k512_h12"))
    c["K"] = 4
    P = orc.make_params(c)
    g = orc.make_gait({"offset": (0, 0, 0, 0), "duty": W.PHASE_ONE, "phase0": 0})
    x0 = np.zeros(12)
    x0[2] = 0.31
    xref = np.zeros((12, 12))
    xref[:, 2] = 0.30
    xref[:, 6] = 0.3
    mean, var = orc.init_dist(P, g)
    fz = 21.0 * 9.81 / 4
    np.testing.assert_allclose(mean.reshape(12, 4, 3)[:, :, 2], fz)
    J, _, _, _ = orc.rollout(P, g, x0, xref, None, mean, var, 0)
    per_step = 50 * 0.01 ** 2 + 5 * 0.3 ** 2 + 4 * 1e-5 * fz ** 2
    np.testing.assert_allclose(J, 12 * per_step, rtol=1e-12)


def test_adaptive_regulariser_and_frequency(orc):
    c = W.config("adaptive_elite_k8192_h25")
    c["K"] = 256
    c["sigma_init"] = 0.0
    P = orc.make_params(c)
    pr = W.problem(c)
    g = orc.make_gait(pr["gait"])
    mean, var = orc.init_dist(P, g)
    J, q, th, margin = orc.rollout(P, g, pr["x0"], pr["xref"], pr["f_ext"], mean, var, 0,
                                   want_theta=True)
    assert np.all((q >= 1000) & (q <= 4000))
    np.testing.assert_array_equal(th[:, -1], q / 1000.0)
    # two samples with the same frequency have the same cost (forces are noise-free)
    for qq in np.unique(q)[:5]:
        sel = J[q == qq]
        assert np.all(sel == sel[0])
    # the regulariser: forcing a frequency changes J by rho (f - f_n)^2 plus the schedule effect;
    # with all legs always in stance the schedule is irrelevant and only the regulariser moves J
    g4 = orc.make_gait({"offset": (0, 0, 0, 0), "duty": W.PHASE_ONE, "phase0": 0})
    x0 = np.zeros(12)
    x0[2] = 0.3
    m4 = mean.copy()
    m4[:-1].reshape(25, 4, 3)[:, :, 2] = 21.0 * 9.81 / 4
    ja, _ = orc.rollout_sample(P, g4, x0, pr["xref"], None, m4, var, 0, 0, 1300)
    jb, _ = orc.rollout_sample(P, g4, x0, pr["xref"], None, m4, var, 0, 0, 2300)
    assert np.isfinite(ja)
    assert jb - ja == pytest.approx(1.0 * (2.3 - 1.3) ** 2, rel=1e-9)


def test_solve_naive_is_best_sample(orc):
    c = W.config("plain_mppi_k512_h12")
    c["method"] = "naive"
    c["K"] = 200
    P = orc.make_params(c)
    pr = W.problem(c)
    g = orc.make_gait(pr["gait"])
    mean, var = orc.init_dist(P, g)
    J, _, th, _ = orc.rollout(P, g, pr["x0"], pr["xref"], None, mean, var, 0, want_theta=True)
    r = orc.solve(P, g, pr["x0"], pr["xref"], None, 0, 0, mean, var)
    np.testing.assert_array_equal(r["mean"], th[np.argmin(J)])
    np.testing.assert_array_equal(r["var"], var)
    np.testing.assert_array_equal(r["J"], J)


def test_solve_iterations_compose(orc):
    # one solve with I iterations equals I single-iteration solves without shift
    c = W.config("adaptive_elite_k8192_h25")
    c["K"] = 300
    c["elite_count"] = 15
    c["iterations"] = 3
    P3 = orc.make_params(c)
    c1 = dict(c, iterations=1)
    P1 = orc.make_params(c1)
    pr = W.problem(c)
    g = orc.make_gait(pr["gait"])
    mean, var = orc.init_dist(P3, g)
    r3 = orc.solve(P3, g, pr["x0"], pr["xref"], pr["f_ext"], 0, 10, mean, var)
    m, v = mean, var
    for i in range(3):
        r = orc.solve(P1, g, pr["x0"], pr["xref"], pr["f_ext"], 0, 10 + i, m, v)
        m, v = r["mean"], r["var"]
    np.testing.assert_array_equal(r3["mean"], m)
    np.testing.assert_array_equal(r3["var"], v)


def test_rollout_threads_identical(orc):
    c = W.config("adaptive_elite_k8192_h25")
    c["K"] = 512
    P = orc.make_params(c)
    pr = W.problem(c)
    g = orc.make_gait(pr["gait"])
    mean, var = orc.init_dist(P, g)
    J1, q1, _, _ = orc.rollout(P, g, pr["x0"], pr["xref"], pr["f_ext"], mean, var, 3, nthreads=1)
    J4, q4, _, _ = orc.rollout(P, g, pr["x0"], pr["xref"], pr["f_ext"], mean, var, 3, nthreads=4)
    np.testing.assert_array_equal(J1, J4)
    np.testing.assert_array_equal(q1, q4)
