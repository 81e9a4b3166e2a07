"""Stored and regenerated sampled deviations (Alg. 1 Sampling): a solve whose
rollout stores no deviations, and whose MPPI sums and elite / Naive refits
regenerate them from their Philox counters, gives the bits of a solve that
stores them, in plain solves over warm-started ticks (every policy and update,
the extended model features, two samples per thread) and in batched ticks."""
import numpy as np
import pytest

from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    S.lib()
    return torch


def _dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


CASES = {
    # MPPI at an intermediate temperature: many samples per tile carry weight
    "mppi_k3001_lam30": dict(K=3001, H=12, tile=128, lam=30.0),
    "mppi_pair_k4096_lam30": dict(K=4096, H=20, tile=256, lam=30.0, spt=2),
    "mppi_adaptive_k2000": dict(K=2000, H=25, tile=64, adaptive=True, lam=50.0),
    "elite_k8192_adaptive_cmp": dict(K=8192, H=25, method="elite", elite_count=410, adaptive=True,
                                     compare_mppi=True),
    "elite_k40000_lanes1024": dict(K=40000, H=6, method="elite", elite_count=2500),
    "elite_spline_p4": dict(K=5000, H=30, P=4, dt_us=10000, method="elite", elite_count=50, adaptive=True),
    "elite_spline_p4_pair": dict(K=5000, H=30, P=4, dt_us=10000, tile=256, method="elite", elite_count=50,
                                 adaptive=True, spt=2),
    "mppi_spline_p3_pair": dict(K=3000, H=25, P=3, dt_us=10000, tile=128, lam=30.0, spt=2),
    "naive_freqset": dict(K=3000, H=12, method="naive", q_init=1300, freq_set_mhz=(1300, 2000, 2400)),
    "mppi_worldfeet_friction": dict(K=2048, H=25, world_feet=True, friction_project=True, lam=30.0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_plain_regenerate_equals_store(name):
    import torch
    cfg = W.config("plain_mppi_k512_h12")
    upd = dict(CASES[name])
    spt = upd.pop("spt", 1)
    cfg.update(upd, seed=654)
    prob = W.problem(cfg)
    x0, xr, fe = _dev(prob["x0"]), _dev(prob["xref"]), _dev(prob["f_ext"])
    feet = _dev(prob["feet"]) if "feet" in prob else None
    ctl = {}
    for mode in (S.THETA_STORE, S.THETA_REGENERATE):
        ctl[mode] = S.Controller(cfg)
        ctl[mode].set_theta_mode(mode)
        ctl[mode].set_samples_per_thread(spt)
    for tick in range(3):
        g = dict(prob["gait"])
        g["phase0"] = (g["phase0"] + tick * cfg["q_init"] * cfg["dt_us"]) % W.PHASE_ONE
        res = {m: c.solve(x0, xr, g, fe, 0 if tick == 0 else 1, feet=feet).clone() for m, c in ctl.items()}
        torch.cuda.synchronize()
        np.testing.assert_array_equal(res[S.THETA_STORE].cpu().numpy(), res[S.THETA_REGENERATE].cpu().numpy())
        bufs = [S.BUF_MEAN, S.BUF_VAR, S.BUF_COST, S.BUF_FREQ]
        if cfg["method"] != "mppi":
            bufs.append(S.BUF_ELITE)
        if cfg.get("compare_mppi"):
            bufs.append(S.BUF_MPPI_MEAN)
        for b in bufs:
            np.testing.assert_array_equal(ctl[S.THETA_STORE].read(b).cpu().numpy(),
                                          ctl[S.THETA_REGENERATE].read(b).cpu().numpy(), err_msg=f"{name} {b}")
    for c in ctl.values():
        c.close()


@pytest.mark.parametrize("mode", [S.BATCH_GRID, S.BATCH_PERSISTENT])
def test_batched_regenerate_equals_store(mode):
    import torch
    mix = W.batch_mix(12, seed=91)
    for c, _ in mix:
        c.update(tile=128, lam=20.0)
    sets = {m: [S.Controller(c) for c, _ in mix] for m in (S.THETA_STORE, S.THETA_REGENERATE)}
    tens = [(_dev(p["x0"]), _dev(p["xref"]), _dev(p["f_ext"])) for _, p in mix]
    n = len(mix)
    batches, res = {}, {}
    for m in sets:
        b = S.Batch(n, sum(c.workspace_bytes() + 256 for c in sets[m]))
        b.set_mode(mode)
        b.set_theta_mode(m)
        assert b.theta_mode() == m
        batches[m] = b
        res[m] = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for tick in range(3):
        for m in sets:
            probs = [sets[m][i].problem(tens[i][0], tens[i][1], mix[i][1]["gait"], tens[i][2],
                                        0 if tick == 0 else 1) for i in range(n)]
            batches[m].solve(sets[m], probs, res[m])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(res[S.THETA_STORE].cpu().numpy(), res[S.THETA_REGENERATE].cpu().numpy())
        for i in range(n):
            for which in (S.BUF_MEAN, S.BUF_VAR):
                np.testing.assert_array_equal(sets[S.THETA_STORE][i].read(which).cpu().numpy(),
                                              sets[S.THETA_REGENERATE][i].read(which).cpu().numpy())
    for b in batches.values():
        b.close()


def test_autotune_in_an_arena_for_regenerated_deviations():
    # an arena sized for regenerated deviations: the autotuner skips the stored
    # settings (refused before any launch) and keeps one that fits; the next tick
    # equals a batch's that ran the same ticks with the kept setting; an arena that
    # fits nothing is refused
    import torch
    mix = W.batch_mix(6, seed=93)
    for c, _ in mix:
        c.update(tile=128, lam=20.0)
    ta = [S.Controller(c) for c, _ in mix]
    tb = [S.Controller(c) for c, _ in mix]
    tens = [(_dev(p["x0"]), _dev(p["xref"]), _dev(p["f_ext"])) for _, p in mix]
    n = len(mix)
    small = sum(c.workspace_bytes_mode(S.THETA_REGENERATE) + 256 for c in ta)
    assert small < sum(c.workspace_bytes_mode(S.THETA_STORE) + 256 for c in ta)
    ba = S.Batch(n, small)
    ra = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    rb = torch.empty_like(ra)
    pa = [ta[i].problem(*tens[i][:2], mix[i][1]["gait"], tens[i][2], 1) for i in range(n)]
    pb = [tb[i].problem(*tens[i][:2], mix[i][1]["gait"], tens[i][2], 1) for i in range(n)]
    grid_ms, pers_ms = ba.autotune(ta, pa, ra, ticks=1)
    assert 0 < grid_ms < 1e29 and 0 < pers_ms < 1e29
    assert ba.theta_mode() == S.THETA_REGENERATE
    bb = S.Batch(n, small)
    bb.set_theta_mode(S.THETA_REGENERATE)
    bb.set_mode(ba.mode())
    bb.set_samples_per_thread(ba.samples_per_thread())
    for _ in range(2 * 2 * 2):  # 2 launch modes x 2 sample counts x (1 + 1) ticks, regenerated only
        bb.solve(tb, pb, rb)
    ba.solve(ta, pa, ra)
    bb.solve(tb, pb, rb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ra.cpu().numpy(), rb.cpu().numpy())
    for i in range(n):
        np.testing.assert_array_equal(ta[i].read(S.BUF_MEAN).cpu().numpy(), tb[i].read(S.BUF_MEAN).cpu().numpy())
    tiny = S.Batch(n, 4096)
    with pytest.raises(S.SBSError) as e:
        tiny.autotune(ta, pa, ra, ticks=1)
    assert e.value.status == S.ERR_BUDGET
    for b in (ba, bb, tiny):
        b.close()
