"""Two samples per thread (packed FP32x2 arithmetic) against one: every result,
cost, frequency, elite list and distribution is bit-identical, in plain solves
over warm-started ticks and in batched ticks of both launch modes, for the
per-step and the spline policy."""
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


def _outputs(ctl, cfg):
    out = {"mean": ctl.read(S.BUF_MEAN).cpu().numpy(), "var": ctl.read(S.BUF_VAR).cpu().numpy(),
           "J": ctl.read(S.BUF_COST).cpu().numpy(), "q": ctl.read(S.BUF_FREQ).cpu().numpy()}
    if cfg["method"] != "mppi":
        out["elite"] = ctl.read(S.BUF_ELITE).cpu().numpy()
    if cfg.get("compare_mppi"):
        out["mppi"] = ctl.read(S.BUF_MPPI_MEAN).cpu().numpy()
    return out


CASES = {
    "mppi_k3001_t64": dict(K=3001, H=12, tile=64),
    "mppi_k40000_t128_groups": dict(K=40000, H=10, tile=128),
    "mppi_adaptive_k5000_t256": dict(K=5000, H=25, tile=256, adaptive=True, gait="crawl"),
    "elite_k4096_t128_adaptive_cmp": dict(K=4096, H=25, tile=128, method="elite", elite_count=205, adaptive=True,
                                          compare_mppi=True),
    "elite_k70000_hist_t256": dict(K=70000, H=8, tile=256, method="elite", elite_count=700),
    "naive_k777_t64": dict(K=777, H=12, tile=64, method="naive"),
    "mppi_terminal_fext_t128": dict(K=2000, H=20, tile=128, gait="pace", f_ext=(5.0, -8.0, 0.0)),
    "mppi_h128_t256": dict(K=1500, H=128, dt_us=1000, tile=256),
    # the shortest horizons and a single sample
    "mppi_h1_k200_t64": dict(K=200, H=1, tile=64),
    "elite_h1_adaptive_k1000": dict(K=1000, H=1, method="elite", elite_count=50, adaptive=True),
    "naive_k1_h2": dict(K=1, H=2, method="naive"),
    "spline_mppi_p4_h2_t64": dict(K=500, H=2, P=4, dt_us=10000, tile=64),
    # spline policy (every compiled knot count)
    "spline_mppi_p4_adaptive_t256": dict(K=3000, H=30, P=4, dt_us=10000, tile=256, lam=30.0, adaptive=True),
    "spline_elite_p3_t128": dict(K=4096, H=25, P=3, dt_us=10000, tile=128, method="elite", elite_count=100),
    "spline_naive_p8_t64": dict(K=1000, H=20, P=8, dt_us=10000, tile=64, method="naive"),
    "spline_mppi_p2_terminal_t128": dict(K=2000, H=40, P=2, dt_us=10000, tile=128, lam=20.0),
    "spline_elite_p6_cmp_t256": dict(K=5000, H=50, P=6, dt_us=10000, tile=256, method="elite", elite_count=50,
                                      adaptive=True, compare_mppi=True),
    "spline_mppi_p4_h128_t128": dict(K=700, H=128, P=4, dt_us=5000, tile=128),
}


@pytest.mark.parametrize("name", list(CASES))
def test_plain_solves_pair_equals_single(name):
    import torch
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(CASES[name], seed=321)
    if name in ("mppi_terminal_fext_t128", "spline_mppi_p2_terminal_t128"):
        cfg["cost"] = dict(cfg["cost"], w_terminal=2.0)
    prob = W.problem(cfg)
    x0, xr, fe = _dev(prob["x0"]), _dev(prob["xref"]), _dev(prob["f_ext"])
    a, b = S.Controller(cfg), S.Controller(cfg)
    a.set_samples_per_thread(1)
    b.set_samples_per_thread(2)
    assert a.samples_per_thread() == 1 and b.samples_per_thread() == 2
    for tick in range(3):
        g = dict(prob["gait"])
        g["phase0"] = (g["phase0"] + tick * cfg["q_init"] * cfg["dt_us"]) % W.PHASE_ONE
        ra = a.solve(x0, xr, g, fe, 0 if tick == 0 else 1).clone()
        rb = b.solve(x0, xr, g, fe, 0 if tick == 0 else 1).clone()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ra.cpu().numpy(), rb.cpu().numpy())
        oa, ob = _outputs(a, cfg), _outputs(b, cfg)
        for key in oa:
            np.testing.assert_array_equal(oa[key], ob[key], err_msg=f"{name} tick {tick} {key}")
    a.close()
    b.close()


@pytest.mark.parametrize("mode", [S.BATCH_GRID, S.BATCH_PERSISTENT])
def test_batched_pair_equals_single(mode):
    import torch
    mix = W.batch_mix(12, seed=77)
    for c, _ in mix:
        c["tile"] = 128
    sets = {1: [S.Controller(c) for c, _ in mix], 2: [S.Controller(c) for c, _ in mix]}
    tens = [(_dev(p["x0"]), _dev(p["xref"]), _dev(p["f_ext"])) for _, p in mix]
    n = len(mix)
    res = {}
    batches = {}
    for spt in (1, 2):
        b = S.Batch(n, sum(c.workspace_bytes() + 256 for c in sets[spt]))
        b.set_mode(mode)
        b.set_samples_per_thread(spt)
        assert b.samples_per_thread() == spt
        batches[spt] = b
        res[spt] = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for tick in range(3):
        for spt in (1, 2):
            probs = [sets[spt][i].problem(tens[i][0], tens[i][1], mix[i][1]["gait"], tens[i][2],
                                          0 if tick == 0 else 1) for i in range(n)]
            batches[spt].solve(sets[spt], probs, res[spt])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(res[1].cpu().numpy(), res[2].cpu().numpy())
        for i in range(n):  # a batched controller's costs stay in the batch's arena: compare its distribution
            for which in (S.BUF_MEAN, S.BUF_VAR):
                np.testing.assert_array_equal(sets[1][i].read(which).cpu().numpy(),
                                              sets[2][i].read(which).cpu().numpy())
    for b in batches.values():
        b.close()


@pytest.mark.parametrize("mode", [S.BATCH_GRID, S.BATCH_PERSISTENT])
def test_batched_spline_pair_equals_single(mode):
    # spline controllers of uneven K, H and method in one batch (4 knots, 128-sample
    # tiles): the elite / Naive controllers' launch and the MPPI controllers'
    import torch
    rng = np.random.default_rng(11)
    mix = []
    for i in range(10):
        cfg = W.config("plain_mppi_k512_h12")
        cfg.update(K=int(rng.choice([256, 1000, 3000])), H=int(rng.choice([10, 25, 50])), P=4, dt_us=10000,
                   tile=128, method=["mppi", "elite", "naive"][i % 3], adaptive=bool(i % 2), seed=100 + i,
                   ctrl=i, lam=25.0)
        if cfg["method"] == "elite":
            cfg["elite_count"] = max(1, cfg["K"] // 20)
        mix.append((cfg, W.problem(cfg)))
    sets = {1: [S.Controller(c) for c, _ in mix], 2: [S.Controller(c) for c, _ in mix]}
    tens = [(_dev(p["x0"]), _dev(p["xref"]), _dev(p["f_ext"])) for _, p in mix]
    n = len(mix)
    res, batches = {}, {}
    for spt in (1, 2):
        b = S.Batch(n, sum(c.workspace_bytes() + 256 for c in sets[spt]))
        b.set_mode(mode)
        b.set_samples_per_thread(spt)
        batches[spt] = b
        res[spt] = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for tick in range(3):
        for spt in (1, 2):
            probs = [sets[spt][i].problem(tens[i][0], tens[i][1], mix[i][1]["gait"], tens[i][2],
                                          0 if tick == 0 else 1) for i in range(n)]
            batches[spt].solve(sets[spt], probs, res[spt])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(res[1].cpu().numpy(), res[2].cpu().numpy())
        for i in range(n):
            for which in (S.BUF_MEAN, S.BUF_VAR):
                np.testing.assert_array_equal(sets[1][i].read(which).cpu().numpy(),
                                              sets[2][i].read(which).cpu().numpy())
    for b in batches.values():
        b.close()


NOISE_WARP_CASES = [n for n in CASES if "spline" not in n]
# the extended model features (the frequency set, ground-fixed feet, friction projection)
EXT_CASES = {
    "naive_freqset_k10000": dict(K=10000, H=12, method="naive", q_init=1300, freq_set_mhz=(1300, 2000, 2400)),
    "mppi_worldfeet_k2048": dict(K=2048, H=25, world_feet=True, lam=30.0),
    "mppi_friction_adaptive_k3001": dict(K=3001, H=20, friction_project=True, adaptive=True, lam=30.0, tile=64),
    "naive_freqset_k5000_t256": dict(K=5000, H=25, method="naive", q_init=2000, freq_set_mhz=(1500, 2000, 2500),
                                     tile=256),
}
CASES.update({f"ext_{k}": v for k, v in EXT_CASES.items()})
NOISE_WARP_CASES += [f"ext_{k}" for k in EXT_CASES]


@pytest.mark.parametrize("theta", [S.THETA_STORE, S.THETA_REGENERATE])
@pytest.mark.parametrize("name", NOISE_WARP_CASES)
def test_plain_solves_noise_warps_equal_single(name, theta):
    # one sample per thread with a producer thread drawing its normals one step
    # ahead (2T threads per tile) against the one-sample launch
    import torch
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(CASES[name], seed=322)
    if name == "mppi_terminal_fext_t128":
        cfg["cost"] = dict(cfg["cost"], w_terminal=2.0)
    prob = W.problem(cfg)
    x0, xr, fe = _dev(prob["x0"]), _dev(prob["xref"]), _dev(prob["f_ext"])
    feet = _dev(prob["feet"]) if "feet" in prob else None
    a, b = S.Controller(cfg), S.Controller(cfg)
    for c in (a, b):
        c.set_theta_mode(theta)
    a.set_samples_per_thread(1)
    b.set_samples_per_thread(S.SPT_NOISE_WARPS)
    assert b.samples_per_thread() == S.SPT_NOISE_WARPS
    for tick in range(3):
        g = dict(prob["gait"])
        g["phase0"] = (g["phase0"] + tick * cfg["q_init"] * cfg["dt_us"]) % W.PHASE_ONE
        ra = a.solve(x0, xr, g, fe, 0 if tick == 0 else 1, feet=feet).clone()
        rb = b.solve(x0, xr, g, fe, 0 if tick == 0 else 1, feet=feet).clone()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ra.cpu().numpy(), rb.cpu().numpy())
        oa, ob = _outputs(a, cfg), _outputs(b, cfg)
        for key in oa:
            np.testing.assert_array_equal(oa[key], ob[key], err_msg=f"{name} tick {tick} {key}")
    a.close()
    b.close()


def test_autotune_keeps_results():
    # the autotuner may pick either sample count: the next tick equals a
    # one-sample-per-thread batch's
    import torch
    mix = W.batch_mix(6, seed=78)
    for c, _ in mix:
        c["tile"] = 256
    ta = [S.Controller(c) for c, _ in mix]
    tb = [S.Controller(c) for c, _ in mix]
    tens = [(_dev(p["x0"]), _dev(p["xref"]), _dev(p["f_ext"])) for _, p in mix]
    n = len(mix)
    ba = S.Batch(n, sum(c.workspace_bytes() + 256 for c in ta))
    bb = S.Batch(n, sum(c.workspace_bytes() + 256 for c in tb))
    bb.set_samples_per_thread(1)
    ra = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    rb = torch.empty_like(ra)
    pa = [ta[i].problem(*tens[i][:2], mix[i][1]["gait"], tens[i][2], 1) for i in range(n)]
    pb = [tb[i].problem(*tens[i][:2], mix[i][1]["gait"], tens[i][2], 1) for i in range(n)]
    # 2 launch modes x 2 sample counts x 2 deviation modes x (1 + 2) ticks, real solves
    ba.autotune(ta, pa, ra, ticks=2)
    assert ba.samples_per_thread() in (1, 2) and ba.theta_mode() in (S.THETA_STORE, S.THETA_REGENERATE)
    for _ in range(2 * 2 * 2 * 3):
        bb.solve(tb, pb, rb)
    ba.solve(ta, pa, ra)
    bb.solve(tb, pb, rb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ra.cpu().numpy(), rb.cpu().numpy())
    ba.close()
    bb.close()


def test_plain_autotune_keeps_results():
    # sbs_autotune times 2 sample counts x 2 deviation modes (1 + 3 solves each)
    # and keeps the fastest; the controller then continues with the same bits as
    # one solved the same number of times with the defaults
    import torch
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(K=20000, H=20, tile=256, seed=5)
    prob = W.problem(cfg)
    x0, xr, fe = _dev(prob["x0"]), _dev(prob["xref"]), _dev(prob["f_ext"])
    a, b = S.Controller(cfg), S.Controller(cfg)
    ra = torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    rb = torch.empty_like(ra)
    pa = a.problem(x0, xr, prob["gait"], fe, 1)
    ms = a.autotune(pa, ra, ticks=3)
    assert set(ms) == {(sp, rg) for sp in (1, 2, S.SPT_NOISE_WARPS) for rg in (0, 1)}
    assert all(v > 0 for v in ms.values())
    best = min(ms, key=ms.get)
    assert (a.samples_per_thread(), a.theta_mode()) == best
    for _ in range(len(ms) * 4):
        b.solve(x0, xr, prob["gait"], fe, 1, rb)
    a.solve(x0, xr, prob["gait"], fe, 1, ra)
    b.solve(x0, xr, prob["gait"], fe, 1, rb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ra.cpu().numpy(), rb.cpu().numpy())
    np.testing.assert_array_equal(a.read(S.BUF_MEAN).cpu().numpy(), b.read(S.BUF_MEAN).cpu().numpy())
    a.close()
    b.close()
