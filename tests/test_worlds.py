"""Pins of the simulated worlds against the FP64 oracle's model.

The serving workload advances its robots with `serving.Plant` and the
closed-loop episodes with `episodes.Body`; both restate Eq. (1) (body-fixed
lever arms, and stance feet fixed on the ground with footholds at touchdown,
Sec. IV-D) in vectorised numpy.  The product may not call the oracle, so each
restatement is checked here against the oracle's `srbd_deriv`,
`srbd_deriv_feet`, `srbd_step`, `foothold` and `cone_project` on random states.
"""
import numpy as np
import pytest

from paper_2403_11383_b300 import episodes as E
from paper_2403_11383_b300 import serving as SV
from paper_2403_11383_b300 import workloads as W


@pytest.fixture(scope="module")
def params(orc):
    return orc.make_params(W.config("plain_mppi_k512_h12"))


def _states(rng, n):
    x = np.zeros((n, 12))
    x[:, 0:3] = rng.uniform(-1.0, 1.0, size=(n, 3))
    x[:, 2] = rng.uniform(0.15, 0.5, size=n)
    x[:, 3:6] = rng.uniform(-0.8, 0.8, size=(n, 3))
    x[:, 6:9] = rng.normal(0.0, 0.5, size=(n, 3))
    x[:, 9:12] = rng.normal(0.0, 2.0, size=(n, 3))
    return x


def test_serving_plant_derivative_is_eq1(orc, params):
    rng = np.random.default_rng(0)
    n = 64
    plant = SV.Plant(n, W.MODEL, rng)
    x = _states(rng, n)
    u = rng.normal(0.0, 40.0, size=(n, 12)) + np.tile([0.0, 0.0, 60.0], 4)
    st = rng.random((n, 4)) < 0.6
    plant.push_sel = np.stack([rng.uniform(-80, 80, n), rng.uniform(-80, 80, n), np.zeros(n)], -1)
    got = plant._deriv_raw(x, u, st)
    for r in range(n):
        gam = (u[r].reshape(4, 3) * st[r][:, None]).ravel()
        want = orc.srbd_deriv(params, x[r], gam, f_ext=plant.push_sel[r])
        np.testing.assert_allclose(got[r], want, rtol=1e-12, atol=1e-10)


def test_serving_plant_step_is_explicit_euler(orc, params):
    # one control interval of 5 ms is one substep: x + h f(x, u) under the stance
    # flags of the current phase, with the current push as the external force
    rng = np.random.default_rng(1)
    n = 32
    plant = SV.Plant(n, W.MODEL, rng)
    plant.push_change[:] = np.inf
    plant.push = np.stack([rng.uniform(-80, 80, n), rng.uniform(-80, 80, n), np.zeros(n)], -1)
    x = _states(rng, n)
    x[:, 3:5] = rng.uniform(-0.3, 0.3, size=(n, 2))
    x[:, 2] = rng.uniform(0.25, 0.35, size=n)
    plant.x[:] = x
    u = rng.normal(0.0, 30.0, size=(n, 12)) + np.tile([0.0, 0.0, 50.0], 4)
    g = W.gait("trot", 0)
    offset = np.asarray(g["offset"], dtype=np.int64)
    duty = np.full(n, g["duty"], dtype=np.int64)
    phase = rng.integers(0, W.PHASE_ONE, size=n).astype(np.uint32)
    q = rng.integers(1000, 4001, size=n).astype(np.float64)
    h = 0.005
    idx = np.arange(n)
    plant.advance(idx, h, u, phase, q, offset, duty, now=0.0)
    for r in range(n):
        st = ((int(phase[r]) + offset) % W.PHASE_ONE) < duty[r]
        gam = (u[r].reshape(4, 3) * st[:, None]).ravel()
        want = orc.srbd_step(params, x[r], gam, h, f_ext=plant.push[r])
        np.testing.assert_allclose(plant.x[r], want, rtol=1e-12, atol=1e-12)


def _body(rng, n, q_mhz=2000):
    return E.Body(n, W.MODEL, W.gait("trot", 0), rng, q_mhz)


def test_episode_world_friction_is_the_cone_projection(orc):
    rng = np.random.default_rng(2)
    G = rng.normal(0.0, 50.0, size=(200, 3))
    got = E.Body.friction(G, 0.5)
    for r in range(200):
        np.testing.assert_allclose(got[r], orc.cone_project(0.5, G[r]), rtol=1e-12, atol=1e-12)


def test_episode_world_footholds(orc, params):
    rng = np.random.default_rng(3)
    n = 16
    body = _body(rng, n)
    body.x = _states(rng, n)
    body.q = rng.integers(1000, 4001, size=n).astype(np.float64)
    vd = rng.uniform(-0.5, 0.5, size=(n, 2))
    legs = np.ones((n, 4), dtype=bool)
    body.land(legs, vd)
    for r in range(n):
        for leg in range(4):
            want = orc.foothold(params, body.x[r], vd[r], int(body.q[r]), body.duty, leg)
            np.testing.assert_allclose(body.feet[r, leg], want, rtol=1e-12, atol=1e-12)


def test_episode_world_step_is_eq1_with_ground_feet(orc):
    # one step: legs that touch down land at the foothold, stance forces are
    # projected onto the cone, and the state moves by h f(x, Gamma) with the lever
    # arms p_f,i - p_c (the world wrench's force acts as the external force)
    cfg = W.config("plain_mppi_k512_h12")
    cfg["world_feet"] = True
    P = orc.make_params(cfg)
    rng = np.random.default_rng(4)
    n = 24
    body = _body(rng, n)
    x = _states(rng, n)
    x[:, 3:5] = rng.uniform(-0.4, 0.4, size=(n, 2))
    body.x = x.copy()
    body.q = rng.integers(1000, 4001, size=n).astype(np.float64)
    body.prev = rng.random((n, 4)) < 0.5
    prev, feet0 = body.prev.copy(), body.feet.copy()
    u = rng.normal(0.0, 30.0, size=(n, 12)) + np.tile([0.0, 0.0, 60.0], 4)
    wrench = np.zeros((n, 6))
    wrench[:, :3] = rng.uniform(-20, 20, size=(n, 3))
    vd = rng.uniform(-0.5, 0.5, size=(n, 2))
    h = 0.005
    st = body.stance()
    body.step(u, wrench, h, vd, 0.5)
    for r in range(n):
        feet = feet0[r].copy()
        for leg in range(4):
            if st[r, leg] and not prev[r, leg]:
                feet[leg] = orc.foothold(P, x[r], vd[r], int(body.q[r]), body.duty, leg)
        np.testing.assert_allclose(body.feet[r], feet, rtol=1e-12, atol=1e-12)
        gam = np.concatenate([orc.cone_project(0.5, u[r, 3 * i:3 * i + 3]) * st[r, i] for i in range(4)])
        xd = orc.srbd_deriv_feet(P, x[r], gam, feet.ravel(), f_ext=wrench[r, :3])
        np.testing.assert_allclose(body.x[r], x[r] + h * xd, rtol=1e-12, atol=1e-12)
