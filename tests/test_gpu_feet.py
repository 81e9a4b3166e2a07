"""GPU parity of stance feet fixed on the ground with footholds placed at
touchdown (Eq. (1) with p_cf,i = p_f,i - p_c; Sec. IV-D), through the C ABI:
MPPI at full size, ragged sizes and the spline policy, the elite update with
sampled step frequencies, the discrete frequency set, warm-started ticks with
new feet, host inputs, and the argument checks."""
import numpy as np
import pytest

import oracle as orc
from gpu_helpers import (MEAN_ATOL, CudaRun, OracleRun, alt_frequency, check_costs, check_frequencies, dev,
                         elite_band_ok, f32, mppi_parity)
from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    S.lib()
    return torch


def test_mppi_full_size(cuda):
    cfg = W.config("worldfeet_mppi_k4096_h25")
    rep = mppi_parity(cfg, W.problem(cfg), "worldfeet")
    assert rep["gated"] > 0.1 * cfg["K"]


@pytest.mark.parametrize("K,H,P,tile", [(777, 12, 0, 64), (130, 7, 0, 256), (3000, 25, 4, 128)])
def test_ragged_sizes_and_spline(cuda, K, H, P, tile):
    cfg = W.config("worldfeet_mppi_k4096_h25")
    cfg.update(K=K, H=H, P=P, seed=K + H, sigma_init=5.0 if P else 20.0)
    mppi_parity(cfg, W.problem(cfg), f"worldfeet K{K} P{P}", tile=tile)


def test_elite_with_sampled_frequencies(cuda):
    # per-sample stance times change both the contact schedule and the footholds
    cfg = W.config("adaptive_elite_k8192_h25")
    cfg.update(K=2048, H=25, iterations=1, world_feet=True, seed=17, compare_mppi=False)
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob), OracleRun(cfg, prob)
    J, q, th, margin, kap = o.rollout()
    r = g.solve()
    Jg, qg, eg = g.read(S.BUF_COST), g.read(S.BUF_FREQ), g.read(S.BUF_ELITE)
    amb = check_frequencies(qg, q, margin)
    check_costs(Jg, J, kap, skip=amb)
    Ke = cfg["elite_count"]
    assert np.all(np.diff(eg) > 0) and eg.size == Ke
    alt = {int(i): o.sample(int(i), alt_frequency(o, int(i)))[0] for i in np.nonzero(amb)[0]}
    elite_band_ok(eg, J, Ke, kap, alt)
    # the refit is the elite mean / biased variance of the selected samples
    mg, vg = g.state()
    thg = th.copy()
    thg[:, -1] = qg / 1000.0
    sel = thg[eg]
    np.testing.assert_allclose(mg, sel.mean(axis=0), atol=MEAN_ATOL, rtol=1e-5)
    assert r["status"] == S.OK
    g.close()


def test_frequency_set_with_world_feet(cuda):
    from test_gpu_freqset import _check_iteration
    cfg = W.config("naive_freqset_k10000_h12")
    cfg.update(K=3000, H=25, world_feet=True, seed=23)
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob), OracleRun(cfg, prob)
    _check_iteration(cfg, g, o, g.solve())
    g.close()


def test_warm_tick_with_new_feet(cuda):
    cfg = W.config("worldfeet_mppi_k4096_h25")
    cfg.update(K=2048, seed=29)
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob), OracleRun(cfg, prob)
    g.solve()
    mg, vg = g.state()
    gait = dict(prob["gait"])
    gait["phase0"] = (gait["phase0"] + 2000 * cfg["dt_us"]) % W.PHASE_ONE
    feet2 = prob["feet"] + 0.01  # the robot has moved its feet
    o.g = orc.make_gait(gait)
    o.feet = np.float64(f32(feet2))
    o.mean, o.var = orc.warm_shift(o.P, o.g, 1, mg.astype(np.float64), vg.astype(np.float64))
    o.iter = 1
    J, q, th, margin, kap = o.rollout()
    g.solve(shift=1, gait=gait, feet=dev(feet2))
    check_costs(g.read(S.BUF_COST), J, kap)
    g.close()


def test_host_inputs_equal_device_inputs(cuda):
    import torch
    cfg = W.config("worldfeet_mppi_k4096_h25")
    cfg.update(K=1024, seed=31)
    prob = W.problem(cfg)
    a, b = CudaRun(cfg, prob), CudaRun(cfg, prob)
    ra = a.solve()
    hb = b.ctl.solve_host(f32(prob["x0"]), f32(prob["xref"]), prob["gait"], f32(prob["f_ext"]), 0,
                          feet=f32(prob["feet"]))
    torch.cuda.synchronize()
    rb = S.parse_result(bytes(hb))
    assert ra["u0"].tolist() == rb["u0"].tolist() and ra["cost_min"] == rb["cost_min"]
    np.testing.assert_array_equal(a.read(S.BUF_COST), b.read(S.BUF_COST))
    np.testing.assert_array_equal(a.state()[0], b.state()[0])
    a.close()
    b.close()


def test_missing_feet_is_rejected(cuda):
    cfg = W.config("worldfeet_mppi_k4096_h25")
    cfg.update(K=256)
    prob = W.problem(cfg)
    g = CudaRun(cfg, prob)
    with pytest.raises(S.SBSError) as e:
        g.ctl.solve(g.x0, g.xref, prob["gait"], g.fext, 0)
    assert e.value.status == S.ERR_INVALID_ARG
    g.close()
