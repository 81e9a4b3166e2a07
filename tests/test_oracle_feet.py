"""Pins of the oracle's world-fixed stance feet (Eq. (1) with p_cf,i = p_f,i - p_c,
feet on the ground z = 0) and the touchdown foothold rule (Sec. IV-D): agreement
with the body-fixed lever arms where the two coincide, static moment balance,
the closed-form pitch acceleration of an offset centre of pressure, and the
foothold's dependence on position, velocity, desired velocity, attitude and
stance time; whole rollouts that hover with footholds placed at touchdown."""
import copy

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2403_11383_b300 import workloads as W

MASS, G = 21.0, 9.81
INERTIA = np.array([0.07, 0.26, 0.24])
OFF = np.asarray(W.MODEL["foot"], dtype=float)


@pytest.fixture(scope="module")
def params(orc):
    return orc.make_params(W.config("worldfeet_mppi_k4096_h25"))


def _rz(yaw):
    return Rotation.from_euler("z", yaw).as_matrix()


def test_level_body_matches_body_fixed_lever_arms(orc, params):
    # level attitude, CoM 0.30 m above the ground: feet under the body-frame foot
    # offsets are exactly the body-fixed model's contact points
    rng = np.random.default_rng(0)
    for _ in range(50):
        x = np.zeros(12)
        x[:2] = rng.uniform(-1, 1, 2)
        x[2] = 0.30
        x[5] = rng.uniform(-np.pi, np.pi)
        x[6:] = rng.normal(size=6)
        gam = rng.normal(scale=60.0, size=12)
        feet = np.array([x[:2] + (_rz(x[5]) @ OFF[i])[:2] for i in range(4)]).ravel()
        np.testing.assert_allclose(orc.srbd_deriv_feet(params, x, gam, feet), orc.srbd_deriv(params, x, gam),
                                   rtol=1e-11, atol=1e-11)


def test_centre_of_pressure_under_the_com_gives_no_torque(orc, params):
    # vertical forces whose centre of pressure lies under the CoM: zero moment at any attitude
    rng = np.random.default_rng(1)
    for _ in range(50):
        x = np.zeros(12)
        x[:3] = [rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.2, 0.4)]
        x[3:6] = rng.uniform(-0.4, 0.4, 3)
        feet = rng.uniform(-0.5, 0.5, size=(4, 2))
        f = rng.uniform(10, 80, size=4)
        cop = (f[:, None] * feet).sum(0) / f.sum()
        feet = feet - cop + x[:2]  # shift the feet so that the centre of pressure is under the CoM
        gam = np.zeros((4, 3))
        gam[:, 2] = f
        d = orc.srbd_deriv_feet(params, x, gam.ravel(), feet.ravel())
        np.testing.assert_allclose(d[9:12], 0, atol=1e-12)


def test_offset_centre_of_pressure_pitches_the_body(orc, params):
    # level body at rest, total vertical force F with the centre of pressure delta
    # ahead of the CoM: omega_dot_y = -delta F / I_yy exactly, no roll or yaw
    x = np.zeros(12)
    x[2] = 0.3
    for delta in (-0.05, 0.02, 0.1):
        f = np.array([40.0, 60.0, 50.0, 55.0])
        feet = OFF[:, :2] + [delta, 0.0]
        cop = (f[:, None] * feet).sum(0) / f.sum()
        feet = feet - [0.0, cop[1]]  # keep the lateral centre of pressure under the CoM
        gam = np.zeros((4, 3))
        gam[:, 2] = f
        d = orc.srbd_deriv_feet(params, x, gam.ravel(), feet.ravel())
        assert d[10] == pytest.approx(-cop[0] * f.sum() / INERTIA[1], rel=1e-12)
        assert abs(d[9]) < 1e-12 and abs(d[11]) < 1e-12


def test_foothold_properties(orc, params):
    duty, q = 600_000_000, 2000
    tst = 0.6 / 2.0
    rng = np.random.default_rng(2)
    x = np.zeros(12)
    x[:3] = [0.4, -0.3, 0.3]
    x[5] = 0.7
    vd = np.array([0.5, -0.2])
    for leg in range(4):
        # at rest with no desired velocity: under the hip
        f0 = orc.foothold(params, x, [0, 0], q, duty, leg)
        np.testing.assert_allclose(f0, x[:2] + (_rz(0.7) @ OFF[leg])[:2], atol=1e-15)
        # linear in the CoM velocity with slope sqrt(z / g), in the desired velocity
        # with slope T_st / 2 - sqrt(z / g); translation equivariant
        s = np.sqrt(0.3 / G)
        for a in range(2):
            xv = x.copy()
            xv[6 + a] += 0.37
            dv = orc.foothold(params, xv, vd, q, duty, leg) - orc.foothold(params, x, vd, q, duty, leg)
            np.testing.assert_allclose(dv, np.eye(2)[a] * 0.37 * s, atol=1e-14)
        dd = orc.foothold(params, x, vd, q, duty, leg) - f0
        np.testing.assert_allclose(dd, vd * (tst / 2 - s), atol=1e-14)
        sh = rng.normal(size=2)
        xs = x.copy()
        xs[:2] += sh
        np.testing.assert_allclose(orc.foothold(params, xs, vd, q, duty, leg),
                                   orc.foothold(params, x, vd, q, duty, leg) + sh, atol=1e-14)
        # stance time T_st = D_f / f_s: doubling the frequency halves the feed-forward term
        d2 = orc.foothold(params, x, vd, 2 * q, duty, leg) - f0
        np.testing.assert_allclose(dd - d2, vd * tst / 4, atol=1e-14)
    # roll and pitch move the hip: the hip is R (offset x, offset y, 0) from the CoM
    xr = x.copy()
    xr[3:6] = [0.3, -0.2, 0.7]
    R = Rotation.from_euler("ZYX", [0.7, -0.2, 0.3]).as_matrix()
    for leg in range(4):
        h = np.array([OFF[leg, 0], OFF[leg, 1], 0.0])
        np.testing.assert_allclose(orc.foothold(params, xr, [0, 0], q, duty, leg), xr[:2] + (R @ h)[:2], atol=1e-14)
    # a CoM below the ground counts as height 0
    xb = x.copy()
    xb[2] = -0.1
    xb[6] = 1.0
    np.testing.assert_allclose(orc.foothold(params, xb, [0, 0], q, duty, 0), x[:2] + (_rz(0.7) @ OFF[0])[:2],
                               atol=1e-15)


def _hover_case(orc, world, vd=0.0):
    c = copy.deepcopy(W.config("worldfeet_mppi_k4096_h25"))
    c.update(K=4, sigma_init=0.0, world_feet=world)
    P = orc.make_params(c)
    g = orc.make_gait(W.gait("trot", 123_456_789))
    x0 = np.zeros(12)
    x0[2] = 0.30
    xref = np.zeros((c["H"], 12))
    xref[:, 2] = 0.30
    xref[:, 6] = vd
    feet = OFF[:, :2].ravel()
    mean, var = orc.init_dist(P, g)
    J, _, _, _ = orc.rollout(P, g, x0, xref, None, mean, var, 0, feet=feet if world else None)
    return J


def test_trot_hover_with_footholds_at_touchdown(orc):
    # a level body at rest on a trot: each stance pair (or all four legs) carries
    # m|g| vertically with zero moment, the body never moves, every touchdown
    # lands under its hip, and the rollout matches the body-fixed lever arms
    Jw = _hover_case(orc, True)
    Jb = _hover_case(orc, False)
    np.testing.assert_allclose(Jw, Jb, rtol=1e-12)
    # with a desired velocity the touchdown footholds move ahead of the hips and
    # the moments (hence the costs) differ from the body-fixed model
    assert not np.allclose(_hover_case(orc, True, vd=0.5), _hover_case(orc, False, vd=0.5), rtol=1e-6)
