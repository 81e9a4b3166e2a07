"""Pins of the oracle's friction-cone constraint on the policy output (Sec. IV-B):
the projection is characterised by Moreau's decomposition (the projected force
lies in the cone, the remainder in the polar cone, the two orthogonal), is
idempotent and leaves forces inside the cone untouched; rollouts whose forces
stay inside the cone are unchanged by it."""
import copy

import numpy as np
import pytest

from paper_2403_11383_b300 import workloads as W


@pytest.mark.parametrize("mu", [0.3, 0.5, 1.2])
def test_moreau_decomposition(orc, mu):
    rng = np.random.default_rng(int(mu * 10))
    for _ in range(2000):
        f = rng.normal(scale=50.0, size=3)
        p = orc.cone_project(mu, f)
        r = f - p
        scale = max(1.0, np.linalg.norm(f))
        assert np.hypot(p[0], p[1]) <= mu * p[2] + 1e-12 * scale  # p in the cone
        assert mu * np.hypot(r[0], r[1]) <= -r[2] + 1e-12 * scale  # remainder in the polar cone
        assert abs(p @ r) <= 1e-10 * scale ** 2  # orthogonal
        np.testing.assert_allclose(orc.cone_project(mu, p), p, atol=1e-12 * scale)  # idempotent


def test_inside_and_polar_cases(orc):
    for f in ([0.0, 0.0, 10.0], [3.0, -4.0, 10.0], [0.0, 0.0, 0.0], [5.0, 0.0, 10.0]):
        np.testing.assert_array_equal(orc.cone_project(0.5, f), f)
    np.testing.assert_array_equal(orc.cone_project(0.5, [1.0, 0.0, -10.0]), 0.0)  # pulling on the ground
    # a purely tangential force lands on the cone boundary at 45 degrees in (|s|, t) scaled by mu
    p = orc.cone_project(1.0, [2.0, 0.0, 0.0])
    np.testing.assert_allclose(p, [1.0, 0.0, 1.0], atol=1e-15)


def test_forces_inside_the_cone_leave_rollouts_unchanged(orc):
    c = copy.deepcopy(W.config("plain_mppi_k512_h12"))
    c.update(K=8, sigma_init=0.0)
    pr = W.problem(c)
    g = orc.make_gait(pr["gait"])
    Js = []
    for proj in (False, True):
        c["friction_project"] = proj
        P = orc.make_params(c)
        m, v = orc.init_dist(P, g)  # vertical mean forces: inside the cone
        Js.append(orc.rollout(P, g, pr["x0"], pr["xref"], pr["f_ext"], m, v, 0)[0])
    np.testing.assert_array_equal(Js[0], Js[1])


def test_projection_removes_the_penalty_and_changes_the_forces(orc):
    c = copy.deepcopy(W.config("plain_mppi_k512_h12"))
    c.update(K=64)
    pr = W.problem(c)
    g = orc.make_gait(pr["gait"])
    out = {}
    for proj in (False, True):
        c["friction_project"] = proj
        P = orc.make_params(c)
        m, v = orc.init_dist(P, g)
        out[proj] = orc.rollout(P, g, pr["x0"], pr["xref"], pr["f_ext"], m, v, 0, want_theta=True)
    # the same samples (theta is the decision variable, not the applied force) ...
    np.testing.assert_array_equal(out[False][2], out[True][2])
    # ... but different applied forces and no friction penalty: the costs differ
    assert not np.allclose(out[False][0], out[True][0])
