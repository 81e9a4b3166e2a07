"""Pins of the oracle's model (Eq. (1)), integrator, gait schedule, stage cost
and spline basis against closed forms, library routines, brute force and
hand-worked values."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.interpolate import CubicSpline
from scipy.spatial.transform import Rotation

from conftest import golden
from paper_2403_11383_b300 import workloads as W


@pytest.fixture(scope="module")
def params(orc):
    return orc.make_params(W.config("plain_mppi_k512_h12"))


# ------------------------------------------------------------------ rotations

def test_rotation_matches_scipy(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        rpy = rng.uniform(-1.2, 1.2, size=3)
        R = orc.rotation(rpy)
        ref = Rotation.from_euler("ZYX", [rpy[2], rpy[1], rpy[0]]).as_matrix()
        np.testing.assert_allclose(R, ref, atol=1e-14)


def test_euler_rates_by_differentiation(orc):
    # R^T dR/dt must equal skew(omega) when the angles move at E'^{-1}(Phi) omega
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(30):
        rpy = rng.uniform(-1.0, 1.0, size=3)
        w = rng.normal(size=3)
        rates = orc.euler_rates(rpy, w)
        Rp, Rm = orc.rotation(rpy + h * rates), orc.rotation(rpy - h * rates)
        Rdot = (Rp - Rm) / (2 * h)
        S = orc.rotation(rpy).T @ Rdot
        np.testing.assert_allclose(S, -S.T, atol=1e-8)
        np.testing.assert_allclose([S[2, 1], S[0, 2], S[1, 0]], w, atol=1e-8)


# ------------------------------------------------------------------ dynamics

def test_ballistic_flight_closed_form(orc, params):
    # all contacts open: v_j = v_0 + g j dt, p_j = p_0 + v_0 j dt + g dt^2 j (j - 1) / 2
    dt = 0.02
    x = np.array([0.1, -0.2, 0.5, 0, 0, 0, 0.3, -0.1, 1.2, 0, 0, 0], dtype=float)
    x0 = x.copy()
    g = np.array([0, 0, -9.81])
    for j in range(1, 41):
        x = orc.srbd_step(params, x, np.zeros(12), dt)
        v = x0[6:9] + g * j * dt
        p = x0[0:3] + x0[6:9] * j * dt + g * dt * dt * j * (j - 1) / 2
        np.testing.assert_allclose(x[6:9], v, atol=1e-12)
        np.testing.assert_allclose(x[0:3], p, atol=1e-12)
        np.testing.assert_array_equal(x[3:6], 0)
        np.testing.assert_array_equal(x[9:12], 0)


def test_external_force_adds_acceleration(orc, params):
    fe = np.array([0.0, 60.0, 0.0])
    d0 = orc.srbd_deriv(params, np.zeros(12), np.zeros(12))
    d1 = orc.srbd_deriv(params, np.zeros(12), np.zeros(12), fe)
    np.testing.assert_allclose(d1[6:9] - d0[6:9], fe / 21.0, atol=1e-15)
    np.testing.assert_array_equal(d1[9:12], d0[9:12])


def test_constant_force_and_hover(orc, params):
    # four stance legs with equal vertical forces F/4 and level attitude: no torque,
    # v_j = v_0 + (F/m + g) j dt exactly; F = m|g| hovers.
    dt = 0.02
    m = 21.0
    for F in (m * 9.81, 300.0):
        gam = np.tile([0.0, 0.0, F / 4], 4)
        x = np.array([0, 0, 0.3, 0, 0, 0, 0.2, 0, 0, 0, 0, 0], dtype=float)
        x0 = x.copy()
        d = orc.srbd_deriv(params, x, gam)
        np.testing.assert_allclose(d[9:12], 0, atol=1e-13)
        for j in range(1, 26):
            x = orc.srbd_step(params, x, gam, dt)
        az = F / m - 9.81
        assert x[8] == pytest.approx(az * 25 * dt, abs=1e-11)
        assert x[6] == pytest.approx(0.2, abs=1e-15)
        np.testing.assert_allclose(x[3:6], 0, atol=1e-13)
        if F == m * 9.81:
            np.testing.assert_allclose(x[2], x0[2], atol=1e-12)


def test_single_leg_torque_direction(orc, params):
    # a vertical push under the front-left foot (+x, +y offset, below the CoM) at level
    # attitude gives tau = r x F = (0.13 F, -0.24 F, 0): positive roll accel, negative pitch accel
    F = 10.0
    gam = np.zeros(12)
    gam[2] = F
    d = orc.srbd_deriv(params, np.zeros(12), gam)
    np.testing.assert_allclose(d[9:12], [0.13 * F / 0.07, -0.24 * F / 0.26, 0.0], atol=1e-13)
    # a lateral (+y world) push under the same foot: tau = r x (0,F,0) = (0.30 F, 0, 0.24 F)
    gam = np.zeros(12)
    gam[1] = F
    d = orc.srbd_deriv(params, np.zeros(12), gam)
    np.testing.assert_allclose(d[9:12], [0.30 * F / 0.07, 0.0, 0.24 * F / 0.24], atol=1e-13)


def test_principal_axis_spin_exact(orc, params):
    # torque-free spin about body z with roll = pitch = 0: omega constant, yaw_j = yaw_0 + w j dt
    dt = 0.01
    x = np.zeros(12)
    x[2] = 0.5
    x[5] = 0.3
    x[11] = 2.0
    for j in range(1, 101):
        x = orc.srbd_step(params, x, np.zeros(12), dt)
    assert x[11] == 2.0 and x[9] == 0.0 and x[10] == 0.0
    assert x[5] == pytest.approx(0.3 + 2.0 * 100 * dt, abs=1e-12)


def _spin_drift(orc, params, dt, T=0.5):
    x = np.zeros(12)
    x[9:12] = [0.5, 0.4, 0.3]
    I = np.array([0.07, 0.26, 0.24])
    w0 = x[9:12].copy()
    E0, L0 = 0.5 * np.sum(I * w0 * w0), np.linalg.norm(I * w0)
    for _ in range(int(round(T / dt))):
        x = orc.srbd_step(params, x, np.zeros(12), dt)
    w = x[9:12]
    return 0.5 * np.sum(I * w * w) - E0, np.linalg.norm(I * w) - L0


def test_torque_free_drift_is_first_order(orc, params):
    # explicit Euler: energy and |L| drift are O(dt); halving dt halves them
    e1, l1 = _spin_drift(orc, params, 0.002)
    e2, l2 = _spin_drift(orc, params, 0.001)
    assert 0.45 <= e2 / e1 <= 0.55
    assert 0.45 <= l2 / l1 <= 0.55


def test_mirror_symmetry(orc, params):
    # reflecting y (and roll, yaw, the y velocity, roll/yaw rates) and swapping
    # left/right legs (y force flipped) maps the derivative onto its mirror image
    rng = np.random.default_rng(3)
    flip = np.array([1, -1, 1, -1, 1, -1, 1, -1, 1, -1, 1, -1], dtype=float)
    for _ in range(20):
        x = rng.normal(scale=0.3, size=12)
        gam = rng.normal(scale=30, size=12)
        xm = x * flip
        gm = gam.reshape(4, 3)[[1, 0, 3, 2]] * np.array([1, -1, 1])
        d = orc.srbd_deriv(params, x, gam)
        dm = orc.srbd_deriv(params, xm, gm.ravel())
        np.testing.assert_allclose(dm, d * flip, atol=1e-10)


# ------------------------------------------------------------------ gait schedule

@pytest.mark.parametrize("gname", ["trot", "pace", "crawl"])
def test_schedule_against_rational_arithmetic(orc, gname):
    rng = np.random.default_rng(4)
    for _ in range(20):
        phase0 = int(rng.integers(0, W.PHASE_ONE))
        q = int(rng.integers(1000, 4001))
        dt_us = int(rng.choice([10000, 20000]))
        g = W.gait(gname, phase0)
        for leg in range(4):
            for j in range(0, 60):
                ph = (Fraction(phase0 + g["offset"][leg], W.PHASE_ONE)
                      + Fraction(q, 1000) * Fraction(dt_us, 10 ** 6) * j)
                ph -= math.floor(ph)
                want = 1 if ph < Fraction(g["duty"], W.PHASE_ONE) else 0
                assert orc.stance(g, leg, q, dt_us, j) == want


def test_schedule_trot_two_hertz_pattern(orc):
    # f = 2 Hz, dt = 0.02 s, D = 0.6: 15 stance steps then 10 swing steps, repeating
    g = W.gait("trot", 0)
    pattern = [orc.stance(g, 0, 2000, 20000, j) for j in range(50)]
    assert pattern == ([1] * 15 + [0] * 10) * 2
    # diagonal pairs move together; FR is half a cycle away from FL
    for j in range(50):
        assert orc.stance(g, 0, 2000, 20000, j) == orc.stance(g, 3, 2000, 20000, j)
        assert orc.stance(g, 1, 2000, 20000, j) == orc.stance(g, 2, 2000, 20000, j)
    assert [orc.stance(g, 1, 2000, 20000, j) for j in range(25)] == [1] * 3 + [0] * 10 + [1] * 12


# ------------------------------------------------------------------ stage cost

def _cost_cases():
    out = []
    with open(golden("stage_cost_cases.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, x, gam, st, want = [t.strip() for t in line.split("|")]
            out.append((name, [float(v) for v in x.split()], [float(v) for v in gam.split()],
                        [int(v) for v in st.split()], float(want)))
    return out


@pytest.mark.parametrize("case", _cost_cases(), ids=lambda c: c[0])
def test_stage_cost_worked_values(orc, params, case):
    name, x, gam, st, want = case
    xr = np.zeros(12)
    xr[2] = 0.30
    assert orc.stage_cost(params, x, xr, gam, st) == pytest.approx(want, rel=1e-12, abs=1e-15)


# ------------------------------------------------------------------ spline basis

@pytest.mark.parametrize("H,P,dt", [(100, 4, 0.01), (25, 5, 0.02), (12, 2, 0.02), (50, 8, 0.02)])
def test_spline_basis_identities(orc, H, P, dt):
    B = orc.spline_basis(H, P, dt)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-13)
    tk = np.linspace(0, (H - 1) * dt, P)
    t = np.arange(H) * dt
    # linear knot values are reproduced exactly
    np.testing.assert_allclose(B @ (3.0 - 2.0 * tk), 3.0 - 2.0 * t, atol=1e-12)
    # against the library natural cubic spline
    rng = np.random.default_rng(P)
    for _ in range(5):
        y = rng.normal(size=P)
        if P == 2:
            ref = np.interp(t, tk, y)
        else:
            ref = CubicSpline(tk, y, bc_type="natural")(t)
        np.testing.assert_allclose(B @ y, ref, atol=1e-12)
        for j in (0, H // 3, H - 1):
            assert orc.spline_at(H, P, dt, y, t[j]) == pytest.approx(ref[j], abs=1e-12)
