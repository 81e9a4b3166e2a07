"""Pins of the oracle's spline policy inside the rollout (Sec. IV-B, Alg. 4 pi):
the force of axis n at step j is sum_p B[j][p] theta_2[12 p + n], zeroed on
swing legs.  The basis itself is pinned against scipy elsewhere; these tests
pin its use in the rollout (basis row and column, knot and axis strides, the
stance mask) through closed forms and through the per-step policy, which the
ballistic, hover and worked-cost pins already fix.

All rollouts here draw with zero variance, so every sample is the mean."""
import copy

import numpy as np
import pytest
from scipy.interpolate import CubicSpline

from paper_2403_11383_b300 import workloads as W

ALWAYS = {"offset": (0, 0, 0, 0), "duty": W.PHASE_ONE, "phase0": 0}  # every leg in stance at every step


def _cfg(H, P, dt_us, Q=None, R=None, w_fc=None):
    c = W.config("plain_mppi_k512_h12")
    c = copy.deepcopy(c)
    c.update(K=1, H=H, P=P, dt_us=dt_us)
    if Q is not None:
        c["cost"]["Q"] = tuple(Q)
    if R is not None:
        c["cost"]["R"] = tuple(R)
    if w_fc is not None:
        c["cost"]["w_fc"] = w_fc
    return c


def _cost(orc, cfg, gait, mean, x0, xref):
    P = orc.make_params(cfg)
    g = orc.make_gait(gait)
    mean = np.asarray(mean, dtype=np.float64)
    J, _, _, _ = orc.rollout(P, g, x0, xref, np.zeros(3), mean, np.zeros(mean.size), 0)
    return float(J[0])


def _problem(H, dt_us, seed=0):
    rng = np.random.default_rng(seed)
    x0 = W.initial_state(rng)
    xref = W.reference(H, dt_us, x0, (0.3, 0.1))
    return x0, xref


@pytest.mark.parametrize("P", [2, 3, 4, 6, 8])
@pytest.mark.parametrize("gname", ["trot", "crawl"])
def test_constant_knots_equal_constant_per_step_forces(orc, P, gname):
    # the basis rows sum to 1, so knots all equal to c give the force c at every
    # step: the same rollout as the per-step policy with c at every step
    H, dt_us = 16, 20000
    x0, xref = _problem(H, dt_us, P)
    gait = W.gait(gname, 123456789)
    rng = np.random.default_rng(10 + P)
    c = np.tile([0.0, 0.0, 21.0 * 9.81 / 2.4], 4) + rng.normal(0.0, 2.0, 12)
    Js = _cost(orc, _cfg(H, P, dt_us), gait, np.tile(c, P), x0, xref)
    Jp = _cost(orc, _cfg(H, 0, dt_us), gait, np.tile(c, H), x0, xref)
    assert np.isfinite(Js)
    assert Js == pytest.approx(Jp, rel=1e-11)


@pytest.mark.parametrize("P", [2, 3, 4, 6, 8])
def test_linear_knots_equal_linear_per_step_forces(orc, P):
    # a natural cubic spline through knots linear in t_p is that line, so the
    # force at step j is a + b t_j
    H, dt_us = 20, 10000
    dt = dt_us * 1e-6
    x0, xref = _problem(H, dt_us, 20 + P)
    gait = W.gait("pace", 987654321)
    rng = np.random.default_rng(30 + P)
    a = np.tile([0.0, 0.0, 21.0 * 9.81 / 2.4], 4) + rng.normal(0.0, 2.0, 12)
    b = rng.normal(0.0, 20.0, 12)
    tk = np.arange(P) * (H - 1) * dt / (P - 1)
    tj = np.arange(H) * dt
    knots = (a[None, :] + tk[:, None] * b[None, :]).ravel()
    steps = (a[None, :] + tj[:, None] * b[None, :]).ravel()
    Js = _cost(orc, _cfg(H, P, dt_us), gait, knots, x0, xref)
    Jp = _cost(orc, _cfg(H, 0, dt_us), gait, steps, x0, xref)
    assert np.isfinite(Js)
    assert Js == pytest.approx(Jp, rel=1e-10)


@pytest.mark.parametrize("P", [2, 3, 4, 6, 8])
@pytest.mark.parametrize("gname", ["always", "trot"])
def test_unit_knot_reads_out_one_basis_column(orc, P, gname):
    # Knot p of axis n (leg i = n // 3, component a = n % 3) set to A, all other
    # entries 0.  Forces are world-frame, so the linear velocity obeys
    #   v_a(j+1) = v_a(j) + dt (st_i(j) A s_p(t_j) / m + g_a)
    # whatever the attitude does, with s_p the natural cubic spline through the
    # unit vector e_p at the knots (scipy's, independent of the oracle's basis).
    # With Q weighting only v_a, no force weight and no friction penalty, the
    # cost is sum_j v_a(j)^2 over the pre-step states (Alg. 2).
    H, dt_us = 20, 10000
    dt = dt_us * 1e-6
    m, gvec = 21.0, np.array([0.0, 0.0, -9.81])
    tk = np.arange(P) * (H - 1) * dt / (P - 1)
    tj = np.arange(H) * dt
    gait = ALWAYS if gname == "always" else W.gait("trot", 250000000)
    x0 = np.zeros(12)
    x0[2] = 0.30
    xref = np.zeros((H, 12))
    A = 7.0
    for p in range(P):
        e = np.zeros(P)
        e[p] = 1.0
        col = np.interp(tj, tk, e) if P == 2 else CubicSpline(tk, e, bc_type="natural")(tj)
        for n in (0, 4, 8, 11, 2 + 3 * (p % 4)):
            leg, ax = n // 3, n % 3
            Q = np.zeros(12)
            Q[6 + ax] = 1.0
            cfg = _cfg(H, P, dt_us, Q=Q, R=(0.0, 0.0, 0.0), w_fc=0.0)
            mean = np.zeros(12 * P)
            mean[12 * p + n] = A
            st = [orc.stance(gait, leg, cfg["q_init"], dt_us, j) for j in range(H)]
            v, want = 0.0, 0.0
            for j in range(H):
                want += v * v
                v += dt * (st[j] * A * col[j] / m + gvec[ax])
            got = _cost(orc, cfg, gait, mean, x0, xref.ravel())
            assert got == pytest.approx(want, rel=1e-12, abs=1e-15), (p, n)


def test_spline_sampled_forces_are_mean_plus_deviation(orc):
    # with variance, the knots of sample k are mean + sigma eps (eps the oracle's
    # normals, counter draw 1 + n / 6); the rollout must use exactly these knots:
    # the same cost as a zero-variance rollout about those knots
    H, P, dt_us = 12, 4, 20000
    cfg = _cfg(H, P, dt_us)
    cfg["K"] = 3
    Pp = orc.make_params(cfg)
    gait = W.gait("trot", 42)
    g = orc.make_gait(gait)
    x0, xref = _problem(H, dt_us, 5)
    mean = np.tile([0.0, 0.0, 60.0], 4 * P)
    var = np.full(12 * P, 9.0)
    J, _, th, _ = orc.rollout(Pp, g, x0, xref, np.zeros(3), mean, var, 7, want_theta=True)
    for k in range(3):
        eps = np.array([orc.normal(cfg["seed"], 0, k, n, 7) for n in range(12 * P)])
        np.testing.assert_allclose(th[k], mean + 3.0 * eps, rtol=0, atol=1e-12)
        c1 = copy.deepcopy(cfg)
        c1["K"] = 1
        assert _cost(orc, c1, gait, th[k], x0, xref) == pytest.approx(J[k], rel=1e-13)
