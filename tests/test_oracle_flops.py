"""The FLOP model of the roofline (profiles/oracle_flop_model.json) against the
oracle's counting build: the stored coefficients are what oracle/count_flops.py
derives now, the counting build computes the same costs as the oracle, its
counts follow hand-read operation counts of small functions, and the model
bounds the count of randomly sampled rollouts."""
import json
import os

import numpy as np
import pytest

from paper_2403_11383_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cf(orc):
    import importlib.util
    spec = importlib.util.spec_from_file_location("count_flops", os.path.join(ROOT, "oracle", "count_flops.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


@pytest.fixture(scope="module")
def stored():
    with open(os.path.join(ROOT, "profiles", "oracle_flop_model.json")) as f:
        return json.load(f)


def test_stored_model_is_recomputed(cf, stored):
    per_step, _ = cf.fit_rollout((0,))
    spline, _ = cf.fit_rollout((2, 4, 8))
    mppi, _ = cf.fit_mppi()
    assert stored["per_step"]["coef"] == per_step
    assert stored["spline"]["coef"] == spline
    assert stored["mppi_flop"]["coef"] == mppi


def test_counting_build_computes_the_oracle_costs(orc):
    cfg = W.config("adaptive_elite_k8192_h25")
    cfg["K"] = 16
    prob = W.problem(cfg)
    P, g = orc.make_params(cfg), orc.make_gait(prob["gait"])
    m, v = orc.init_dist(P, g)
    for k in range(16):
        _, Jc = orc.count_rollout(P, g, prob["x0"], prob["xref"], prob["f_ext"], m, v, 3, k)
        J, _ = orc.rollout_sample(P, g, prob["x0"], prob["xref"], prob["f_ext"], m, v, 3, k)
        assert Jc == J or (np.isinf(Jc) and np.isinf(J))


def test_counts_of_small_functions_by_hand(orc):
    # stage cost, no leg in stance: per state e = x - xr, J += Q e e (4 FLOP), per
    # force J += R g g (3 FLOP): 12 * 4 + 12 * 3 = 84; each stance leg inside the
    # cone adds |G_xy| (2 mul, 1 add, 1 sqrt), mu G_z and the difference (2), and
    # J += w_fc pen (2): 8
    L = orc.lib_flops()
    P = orc.make_params(W.config("plain_mppi_k512_h12"))
    x, xr = np.linspace(0.1, 1.2, 12), np.zeros(12)
    gam = np.tile([1.0, 2.0, 50.0], 4)
    for n_stance in range(5):
        st = np.array([1] * n_stance + [0] * (4 - n_stance), dtype=np.int32)
        L.orc_flops_reset()
        L.orc_stage_cost(orc.C.byref(P), orc._p(x), orc._p(xr), orc._p(gam), orc._p(st))
        c = orc._flops_read()
        assert c["flop"] == 84 + 8 * n_stance
        assert c["sqrt"] == n_stance
    # MPPI over K samples of dimension D: beta, then per sample w = exp(-(J - b) / l)
    # (2 + exp), Omega += w (1), w /= Omega (1), s2 += w w (2), per entry s += w theta
    # (2), and 1 / s2 (1)
    K, D = 7, 5
    c = orc.count_mppi(np.arange(K, dtype=float), np.ones((K, D)), 1.0)
    assert c["flop"] == K * 2 + K * 4 + K * D * 2 + 1
    assert c["fn"] == K


def test_model_bounds_sampled_rollouts(orc, stored):
    # with sampled forces some friction-penalty terms are active: each adds 2 FLOP
    coef = stored["per_step"]["coef"]["flop"]
    for name, gname in (("plain_mppi_k512_h12", "trot"), ("adaptive_elite_k8192_h25", "crawl")):
        cfg = W.config(name)
        cfg.update(K=8, gait=gname)
        prob = W.problem(cfg)
        P, g = orc.make_params(cfg), orc.make_gait(prob["gait"])
        m, v = orc.init_dist(P, g)
        J, q, _, _ = orc.rollout(P, g, prob["x0"], prob["xref"], prob["f_ext"], m, v, 0)
        for k in range(8):
            c, _ = orc.count_rollout(P, g, prob["x0"], prob["xref"], prob["f_ext"], m, v, 0, k)
            S = sum(orc.stance(prob["gait"], i, int(q[k]), cfg["dt_us"], j) for i in range(4)
                    for j in range(cfg["H"]))
            F = coef[0] + coef[1] * cfg["H"] + coef[2] * S + coef[3] * int(cfg["adaptive"])
            assert F <= c["flop"] <= F + 4 * S
            assert (c["flop"] - F) % 2 == 0
