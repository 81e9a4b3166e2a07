"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  Tolerances are documented in gpu_helpers."""
import copy
import math

import numpy as np
import pytest

import oracle as orc
from gpu_helpers import (MEAN_ATOL, CudaRun, OracleRun, alt_frequency, check_costs, check_frequencies, dev,
                         elite_band_ok, elite_parity, f32, mppi_parity, mppi_tolerance)
from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    S.lib()
    return torch


def golden_kat():
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append(v)
    return rows


# ------------------------------------------------------------------ random numbers

def test_philox_gpu_known_answers_and_oracle(cuda):
    torch = cuda
    rows = golden_kat()
    rng = np.random.default_rng(0)
    extra = rng.integers(0, 2 ** 32, size=(4093, 6), dtype=np.uint64)
    allv = np.array([r[:6] for r in rows] + extra.tolist(), dtype=np.uint64)
    ctr = torch.tensor(allv[:, :4].astype(np.uint32).view(np.int32), device="cuda")
    key = torch.tensor(allv[:, 4:6].astype(np.uint32).view(np.int32), device="cuda")
    out = S.philox(ctr, key).cpu().numpy().view(np.uint32)
    for i, r in enumerate(rows):
        assert out[i].tolist() == r[6:10]
    for i in range(len(rows), allv.shape[0], 7):
        want = orc.philox4x32_10(allv[i, :4].astype(np.uint32), allv[i, 4:6].astype(np.uint32))
        assert out[i].tolist() == want.tolist()


def _radius_bound(seed, ctrl, k, n, it):
    """Bound on the force normal's radius error from the hardware base-2
    logarithm: log2 of u1 = (a + 1) 2^-21 is off by at most 2^-22 on [0.5, 1] and
    2 ulp below (3 with the scaling), so ln u1 is off by e = 2^-22 ln 2 there and
    r = sqrt(-2 ln u1) moves by at most min(2 e / r, sqrt(2 e))."""
    w = orc.philox4x32_10(np.array([k, 1 + n // 6, it & 0xFFFFFFFF, it >> 32], dtype=np.uint32),
                          np.array([seed, ctrl], dtype=np.uint32))
    a = int(orc.uniforms21(w)[2 * ((n % 6) // 2)])
    u1 = (a + 1) / 2.0 ** 21
    ln = math.log(u1)
    e = 2.0 ** -22 * math.log(2.0) if u1 >= 0.5 else 3.0 * 2.0 ** -23 * abs(ln)
    r = math.sqrt(-2.0 * ln)
    return math.sqrt(2.0 * e) if r == 0.0 else min(2.0 * e / r, math.sqrt(2.0 * e))


def test_hardware_square_root_bound(cuda):
    # every single-precision mantissa of both exponent parities ([1, 4)), then
    # scaled arguments: relative error below 1.1e-7 (under one ulp) against double
    # precision, and an exact zero (the bound the normals' radius and the cone
    # norm rely on)
    torch = cuda
    bits = np.arange(0x3F800000, 0x3F800000 + (1 << 24), dtype=np.uint32)
    x = bits.view(np.float32)
    y = S.sqrt_hw(torch.from_numpy(x).cuda()).cpu().numpy()
    rel = np.abs(y.astype(np.float64) - np.sqrt(x.astype(np.float64))) / np.sqrt(x.astype(np.float64))
    assert rel.max() <= 1.1e-7, rel.max()
    ulp = np.abs(y.astype(np.float64) - np.sqrt(x.astype(np.float64))) / np.spacing(y)
    assert ulp.max() < 1.0, ulp.max()
    xs = np.float32([0.0, 1e-30, 3.7e-9, 4.2, 1.5e12, 3e38])
    ys = S.sqrt_hw(torch.from_numpy(xs).cuda()).cpu().numpy()
    assert ys[0] == 0.0
    np.testing.assert_allclose(ys, np.sqrt(xs.astype(np.float64)), rtol=1.1e-7)


def test_normals_gpu_vs_oracle(cuda):
    seed, ctrl, it = 11, 3, (1 << 32) + 7
    nk, nn = 1024, 50
    z = S.normals(seed, ctrl, it, 5, nk, nn).cpu().numpy()
    ref = np.array([[orc.freq_normal(seed, ctrl, 5 + i, it)] +
                    [orc.normal(seed, ctrl, 5 + i, n, it) for n in range(nn)] for i in range(nk)])
    # the frequency normal: accurate logarithm, hardware angle
    np.testing.assert_allclose(z[:, 0], ref[:, 0], rtol=2e-6, atol=3e-6)
    # force normals: plus the radius bound of the hardware logarithm, per normal
    bound = np.array([[_radius_bound(seed, ctrl, 5 + i, n, it) for n in range(nn)] for i in range(nk)])
    err = np.abs(z[:, 1:] - ref[:, 1:])
    assert np.all(err <= 3e-6 + 2e-6 * np.abs(ref[:, 1:]) + 1.05 * bound), np.max(err - bound)
    # the bound is large only at the smallest radii: almost every normal is as close as before
    assert np.mean(err <= 3e-6 + 2e-6 * np.abs(ref[:, 1:])) >= 0.99


# ------------------------------------------------------------------ single solves

def test_plain_mppi_single_solve(cuda):
    cfg = W.config("plain_mppi_k512_h12")
    rep = mppi_parity(cfg, W.problem(cfg), "c1")
    assert rep["gated"] >= 0.99 * cfg["K"]  # all but a few chaotic samples are gated


@pytest.mark.parametrize("K,H,gait,tile", [(1000, 7, "trot", 128), (77, 3, "pace", 64), (1, 5, "crawl", 128),
                                           (3001, 20, "crawl", 256), (150, 1, "trot", 64), (33, 2, "pace", 64)])
def test_mppi_ragged_and_small(cuda, K, H, gait, tile):
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(K=K, H=H, gait=gait, tile=tile, seed=K)
    mppi_parity(cfg, W.problem(cfg), f"K{K}")


@pytest.mark.parametrize("name,upd", [
    ("elite_h1_adaptive", dict(K=1000, H=1, method="elite", elite_count=50, adaptive=True)),
    ("elite_spline_p3_h2", dict(K=700, H=2, P=3, dt_us=10000, tile=64, method="elite", elite_count=35)),
    ("spline_p4_h2", dict(K=500, H=2, P=4, dt_us=10000, tile=64)),
])
def test_shortest_horizons(cuda, name, upd):
    # one step (the warm shift then re-initialises the whole mean) and the shortest
    # spline horizon (four knots on two steps)
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(upd, seed=11)
    prob = W.problem(cfg)
    rep = (mppi_parity if cfg["method"] == "mppi" else elite_parity)(cfg, prob, name)
    assert rep["gated"] >= 0.95 * cfg["K"], rep  # 98.6 % for the one-step adaptive elite solve


@pytest.mark.parametrize("method", ["mppi", "elite"])
def test_longest_horizon(cuda, method):
    # H at its maximum (128 steps) with 256-sample tiles; dt = 1 ms keeps the
    # 0.128 s open-loop horizon well conditioned
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(K=777, H=128, dt_us=1000, tile=256, seed=128, method=method,
               elite_count=W.elite_count(0.05, 777) if method == "elite" else 1)
    prob = W.problem(cfg)
    rep = (mppi_parity if method == "mppi" else elite_parity)(cfg, prob, f"H128 {method}", tile=256)
    assert rep["gated"] >= 0.9 * cfg["K"], rep


def test_mppi_k1_returns_its_sample(cuda):
    cfg = W.config("plain_mppi_k512_h12")
    cfg["K"] = 1
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob), OracleRun(cfg, prob)
    J, q, th, margin, kap = o.rollout()
    g.solve()
    mg, _ = g.state()
    np.testing.assert_allclose(mg, th[0], atol=1e-4, rtol=1e-6)
    g.close()


@pytest.mark.parametrize("lam,tile", [(1e-7, 128), (1e6, 256), (1e6, 64)])
def test_mppi_weight_extremes(cuda, lam, tile):
    # lambda -> 0: a tile keeps nonzero weights only within a few ulps of its best
    # cost, and the update is the best sample (Alg. 5 with beta = min J); lambda
    # -> inf: every finite sample has weight ~1 and the update is the plain
    # sample mean.  The FP64 update is taken from the GPU's own costs (the staged
    # parity of the update), on the oracle's samples.
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(K=3001, lam=lam, seed=97, tile=tile)
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob, tile=tile), OracleRun(cfg, prob)
    J, q, th, margin, kap = o.rollout()
    g.solve()
    Jg = g.read(S.BUF_COST).astype(np.float64)
    mg, _ = g.state()
    _, mo, _, _ = orc.mppi(Jg, th, lam)
    assert np.all(np.abs(mg - mo) <= MEAN_ATOL), np.max(np.abs(mg - mo))
    fin = np.isfinite(Jg)
    if lam < 1.0:
        gap = np.sort(Jg[fin])[1] - Jg[fin].min()
        if gap * 1.0 / lam > 120.0:  # the second-best weight underflows: the best sample alone
            np.testing.assert_allclose(mg, th[int(np.argmin(Jg))], atol=MEAN_ATOL, rtol=0)
    else:
        np.testing.assert_allclose(mg, th[fin].mean(axis=0), atol=MEAN_ATOL, rtol=0)
    g.close()


def test_mppi_many_tiles_hierarchical_combine(cuda):
    # 40 000 samples = 313 tiles = 20 groups of 16: exercises the two-level combine
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(K=40000, seed=9)
    mppi_parity(cfg, W.problem(cfg), "K40000")


def test_adaptive_elite_iteration0_full_size(cuda):
    # the adaptive elite workload (K=8192, H=25, 60 N push): iteration 0
    cfg = W.config("adaptive_elite_k8192_h25")
    cfg["iterations"] = 1
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob), OracleRun(cfg, prob)
    J, q, th, margin, kap = o.rollout()
    r = g.solve()
    Jg, qg = g.read(S.BUF_COST), g.read(S.BUF_FREQ)
    amb = check_frequencies(qg, q, margin)
    check_costs(Jg, J, kap, skip=amb)
    Ke = cfg["elite_count"]
    eg = g.read(S.BUF_ELITE)
    assert np.all(np.diff(eg) > 0) and eg.size == Ke
    alt = {}
    for i in np.nonzero(amb)[0]:
        alt[int(i)] = o.sample(int(i), alt_frequency(o, int(i)))[0]
    elite_band_ok(eg, J, Ke, kap, alt)
    # the refit is the elite mean / biased variance of the selected samples
    mg, vg = g.state()
    thg = th.copy()
    thg[:, -1] = qg / 1000.0
    sel = thg[eg]
    np.testing.assert_allclose(mg, sel.mean(axis=0), atol=MEAN_ATOL, rtol=1e-5)
    vref = np.maximum(sel.var(axis=0), np.r_[np.full(thg.shape[1] - 1, cfg["sigma_min"] ** 2),
                                             cfg["sigma_f_min"] ** 2])
    np.testing.assert_allclose(vg, vref, rtol=2e-4, atol=1e-6)
    assert r["cost_min"] == pytest.approx(float(np.min(Jg)), rel=0)
    # MPPI on the same noise
    mm = g.read(S.BUF_MPPI_MEAN)
    st, mo, _, _ = orc.mppi(J, th, cfg["lam"])
    tol = mppi_tolerance(J, th, kap, cfg["lam"], mo)
    assert np.all(np.abs(mm[:-1] - mo[:-1]) <= tol[:-1])
    g.close()


def _well_conditioned_elite():
    cfg = W.config("adaptive_elite_k8192_h25")
    cfg.update(H=12, K=4096, elite_count=W.elite_count(0.05, 4096), seed=21, iterations=1)
    return cfg


def test_elite_iterations_track_oracle(cuda):
    # five warm-started elite iterations compared iteration by iteration while the
    # elite sets agree (a swap at a near tie ends the comparison)
    cfg = _well_conditioned_elite()
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob), OracleRun(cfg, prob)
    compared = 0
    for it in range(5):
        J, q, th, margin, kap = o.rollout()
        r = g.solve()
        Jg, qg, eg = g.read(S.BUF_COST), g.read(S.BUF_FREQ), g.read(S.BUF_ELITE)
        amb = check_frequencies(qg, q, margin)
        check_costs(Jg, J, kap, skip=amb)
        ro = o.solve()
        mg, vg = g.state()
        if not np.array_equal(np.sort(ro["elite"]), eg):
            elite_band_ok(eg, J, cfg["elite_count"], kap)
            break
        np.testing.assert_allclose(mg, ro["mean"], atol=MEAN_ATOL, rtol=1e-5)
        np.testing.assert_allclose(vg, ro["var"], rtol=2e-4, atol=1e-6)
        np.testing.assert_allclose(r["u0"], ro["u0"], atol=MEAN_ATOL)
        assert r["q_freq"] == pytest.approx(round(1000 * min(4.0, max(1.0, ro["f_mean"]))), abs=1)
        compared += 1
    assert compared >= 1
    g.close()


def test_naive_is_best_sample(cuda):
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(method="naive", K=1500, seed=5)
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob), OracleRun(cfg, prob)
    J, q, th, margin, kap = o.rollout()
    r = g.solve()
    Jg = g.read(S.BUF_COST)
    check_costs(Jg, J, kap)
    best = int(np.lexsort((np.arange(J.size), J))[0])
    kb = int(np.lexsort((np.arange(Jg.size), Jg))[0])
    assert kb == best or abs(J[kb] - J[best]) <= 2e-4 * abs(J[best])
    mg, vg = g.state()
    np.testing.assert_allclose(mg, th[kb], atol=MEAN_ATOL)
    np.testing.assert_array_equal(vg, f32(o.var))
    g.close()


def test_naive_with_sampled_frequency(cuda):
    # Naive with the Gaussian step frequency: the best sample's forces and its
    # quantised frequency become the mean, variances kept (Alg. 3)
    cfg = W.config("adaptive_elite_k8192_h25")
    cfg.update(method="naive", K=3000, H=12, iterations=1, compare_mppi=False, seed=83)
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob), OracleRun(cfg, prob)
    J, q, th, margin, kap = o.rollout()
    r = g.solve()
    Jg, qg, eg = g.read(S.BUF_COST), g.read(S.BUF_FREQ), g.read(S.BUF_ELITE)
    amb = check_frequencies(qg, q, margin)
    check_costs(Jg, J, kap, skip=amb)
    kb = int(np.lexsort((np.arange(Jg.size), Jg))[0])
    assert eg.tolist() == [kb, 0]  # the winner of the single force block, then that block
    mg, vg = g.state()
    np.testing.assert_allclose(mg[:-1], th[kb, :-1], atol=MEAN_ATOL)
    assert mg[-1] == np.float32(qg[kb] / 1000.0)
    np.testing.assert_array_equal(vg, f32(o.var))
    assert r["q_freq"] == qg[kb] and r["cost_min"] == float(Jg[kb]) and r["ess"] == 1.0
    g.close()


def test_iterations_compose_on_gpu(cuda):
    # one solve with I iterations equals I single-iteration solves, bit for bit
    cfg = W.config("adaptive_elite_k8192_h25")
    cfg.update(K=2048, seed=7)
    prob = W.problem(cfg)
    g5 = CudaRun(cfg, prob)
    r5 = g5.solve()
    m5, v5 = g5.state()
    c1 = dict(cfg, iterations=1)
    g1 = CudaRun(c1, prob)
    for _ in range(5):
        r1 = g1.solve()
    m1, v1 = g1.state()
    np.testing.assert_array_equal(m5, m1)
    np.testing.assert_array_equal(v5, v1)
    np.testing.assert_array_equal(r5["u0"], r1["u0"])
    assert r5["iter"] == r1["iter"] == 4
    g5.close()
    g1.close()


def test_warm_start_two_ticks(cuda):
    # second tick shifted by one step from the first tick's solution
    cfg = W.config("plain_mppi_k512_h12")
    cfg["seed"] = 3
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob), OracleRun(cfg, prob)
    g.solve()
    o.solve()
    gait2 = dict(prob["gait"])
    gait2["phase0"] = (gait2["phase0"] + 2000 * 20000) % W.PHASE_ONE
    o.g = orc.make_gait(gait2)
    J, q, th, margin, kap = None, None, None, None, None
    m_shift, v_shift = orc.warm_shift(o.P, o.g, 1, o.mean, o.var)
    o.mean, o.var = m_shift, v_shift
    J, q, th, margin, kap = o.rollout()
    g.solve(shift=1, gait=gait2)
    Jg = g.read(S.BUF_COST)
    check_costs(Jg, J, kap)
    st, mo, _, _ = orc.mppi(J, th, cfg["lam"])
    mg, vg = g.state()
    tol = mppi_tolerance(J, th, kap, cfg["lam"], mo)
    # the first tick's GPU/oracle means differ within their tolerance; that difference
    # enters the second tick's sampling mean linearly
    assert np.all(np.abs(mg - mo) <= tol + 2 * MEAN_ATOL)
    np.testing.assert_allclose(vg, v_shift, rtol=1e-6)
    g.close()


def test_spline_full_size_update(cuda):
    # the spline workload at full size (K = 262 144, H = 100, 4 knots, adaptive
    # frequency): the staged update against FP64 on the oracle's samples of all
    # K draws, from the GPU's own costs and frequencies.  Elite (Alg. 1 Update):
    # the 2 622 elites are the first K_e of the GPU's (cost, index) order, and the
    # refit is their FP64 mean and floored biased variance.  MPPI on the same
    # samples (Alg. 5): the FP64 weighted mean of the GPU's costs, and twice at a
    # temperature where the effective sample size is intermediate.
    cfg = W.config("spline_k262144_h100")
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob), OracleRun(cfg, prob)
    g.solve()
    Jg = g.read(S.BUF_COST).astype(np.float64)
    qg, eg = g.read(S.BUF_FREQ), g.read(S.BUF_ELITE)
    _, _, th, _, _ = o.rollout(kappa=False, nthreads=orc.max_threads())
    th[:, -1] = qg / 1000.0
    Ke = cfg["elite_count"]
    np.testing.assert_array_equal(eg, np.sort(np.lexsort((np.arange(cfg["K"]), Jg))[:Ke]))
    sel = th[eg]
    mg, vg = g.state()
    np.testing.assert_allclose(mg, sel.mean(axis=0), atol=MEAN_ATOL, rtol=1e-5)
    floor = np.r_[np.full(th.shape[1] - 1, cfg["sigma_min"] ** 2), cfg["sigma_f_min"] ** 2]
    np.testing.assert_allclose(vg, np.maximum(sel.var(axis=0), floor), rtol=2e-4, atol=1e-6)
    mm = g.read(S.BUF_MPPI_MEAN)
    _, mo, _, _ = orc.mppi(Jg, th, cfg["lam"])
    assert np.all(np.abs(mm - mo) <= MEAN_ATOL), float(np.max(np.abs(mm - mo)))
    g.close()
    # intermediate weights at full size: lambda from the GPU's costs of this solve
    # (the rollout does not depend on lambda, so the costs repeat bit for bit)
    fin = np.isfinite(Jg)
    spread = np.sort(Jg[fin])
    for lam in (spread[100] - spread[0], spread[3000] - spread[0]):
        c2 = dict(cfg, lam=float(lam), method="mppi", compare_mppi=False)
        g2 = CudaRun(c2, prob)
        r2 = g2.solve()
        J2 = g2.read(S.BUF_COST).astype(np.float64)
        np.testing.assert_array_equal(J2, Jg)
        m2, _ = g2.state()
        _, mo2, ess2, _ = orc.mppi(J2, th, float(lam))
        print(f"lambda {lam:.4g}: ESS oracle {ess2:.1f} gpu {r2['ess']:.1f}")
        assert 10.0 <= ess2 <= cfg["K"] / 10.0
        assert np.all(np.abs(m2 - mo2) <= MEAN_ATOL), float(np.max(np.abs(m2 - mo2)))
        assert r2["ess"] == pytest.approx(ess2, rel=1e-4)
        assert r2["n_finite"] == int(fin.sum())
        g2.close()


def test_spline_full_size_sampled(cuda):
    # the spline workload at full size (K=262144, H=100, 4 knots): sampled costs
    cfg = W.config("spline_k262144_h100")
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob), OracleRun(cfg, prob)
    r = g.solve()
    Jg, qg, eg = g.read(S.BUF_COST), g.read(S.BUF_FREQ), g.read(S.BUF_ELITE)
    rng = np.random.default_rng(1)
    ks = np.r_[rng.choice(cfg["K"], 150, replace=False), eg[:50]]
    J = np.array([o.sample(int(k))[0] for k in ks])
    kap = np.array([o.kappa(int(k)) for k in ks])
    qo = np.array([orc.quantise_freq(o.mean[-1], np.sqrt(o.var[-1]), orc.freq_normal(cfg["seed"], 0, int(k), 0),
                                     cfg["f_min"], cfg["f_max"]) for k in ks])
    amb = check_frequencies(qg[ks], qo[:, 0].astype(np.uint32), qo[:, 1])
    check_costs(Jg[ks], J, kap, skip=amb)
    assert eg.size == cfg["elite_count"] and np.all(np.diff(eg) > 0)
    # every elite's cost is at most every non-elite's (on the GPU's own costs), and
    # the list is exactly the first K_e of the (cost, index) order
    mask = np.zeros(cfg["K"], bool)
    mask[eg] = True
    assert Jg[mask].max() <= Jg[~mask].min()
    np.testing.assert_array_equal(eg, np.sort(np.lexsort((np.arange(cfg["K"]), Jg))[:cfg["elite_count"]]))
    g.close()


@pytest.mark.parametrize("name,extra", [
    ("plain_mppi_k512_h12", dict(K=2048, seed=71)),
    ("spline_k262144_h100", dict(K=3000, H=25, dt_us=20000, method="mppi", compare_mppi=False, sigma_init=5.0,
                                 seed=73)),
])
def test_terminal_cost_parity(cuda, name, extra):
    cfg = W.config(name)
    cfg.update(extra)
    cfg["cost"] = dict(cfg["cost"], w_terminal=4.0)
    mppi_parity(cfg, W.problem(cfg), f"terminal {name}")


@pytest.mark.parametrize("K,frac", [(32769, 0.05), (40000, 0.3), (70001, 0.01)])
def test_large_k_selection_is_the_cost_index_order(cuda, K, frac):
    # elite selections above the shared-memory size run as five multi-block passes
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(K=K, method="elite", elite_count=W.elite_count(frac, K), seed=K % 97)
    prob = W.problem(cfg)
    g = CudaRun(cfg, prob)
    for shift in (0, 1):
        r = g.solve(shift=shift)
        Jg, eg = g.read(S.BUF_COST), g.read(S.BUF_ELITE)
        want = np.sort(np.lexsort((np.arange(K), Jg))[:cfg["elite_count"]])
        np.testing.assert_array_equal(eg, want)
        assert r["cost_min"] == float(Jg.min()) and r["n_finite"] == int(np.isfinite(Jg).sum())
    g.close()


def test_spline_small_mppi_parity(cuda):
    cfg = W.config("spline_k262144_h100")
    cfg.update(K=3000, H=25, dt_us=20000, method="mppi", compare_mppi=False, sigma_init=5.0, seed=8)
    mppi_parity(cfg, W.problem(cfg), "spline-small")


@pytest.mark.parametrize("P,tile", [(2, 128), (3, 64), (6, 128), (8, 128), (8, 256)])
def test_spline_knot_counts_mppi(cuda, P, tile):
    # every compiled knot count: 2-4 knots keep one float4 of deviations per
    # force axis and thread, 6 and 8 two
    cfg = W.config("spline_k262144_h100")
    cfg.update(K=3001, H=25, P=P, dt_us=20000, method="mppi", compare_mppi=False, sigma_init=5.0, seed=40 + P,
               tile=tile)
    mppi_parity(cfg, W.problem(cfg), f"spline-P{P}-T{tile}", tile=tile)


@pytest.mark.parametrize("P", [3, 8])
def test_spline_knot_counts_elite(cuda, P):
    # the elite refit of every knot and the frequency (one refit block per knot)
    cfg = W.config("spline_k262144_h100")
    cfg.update(K=3001, H=25, P=P, dt_us=20000, compare_mppi=False, sigma_init=5.0, seed=50 + P, tile=128,
               elite_count=W.elite_count(0.02, 3001))
    elite_parity(cfg, W.problem(cfg), f"spline-elite-P{P}", tile=128)


@pytest.mark.parametrize("P", [4, 6, 8])
def test_spline_warm_start_two_ticks(cuda, P):
    # the second tick samples about the first tick's knots moved one step along the
    # spline (the knot shift map), on both sides
    cfg = W.config("spline_k262144_h100")
    cfg.update(K=2001, H=25, P=P, dt_us=20000, method="mppi", compare_mppi=False, sigma_init=5.0, seed=60 + P,
               tile=128)
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob, tile=128), OracleRun(cfg, prob)
    g.solve()
    o.solve()
    gait2 = dict(prob["gait"])
    gait2["phase0"] = (gait2["phase0"] + cfg["q_init"] * cfg["dt_us"]) % W.PHASE_ONE
    o.g = orc.make_gait(gait2)
    m_shift, v_shift = orc.warm_shift(o.P, o.g, 1, o.mean, o.var)
    o.mean, o.var = m_shift, v_shift
    J, q, th, margin, kap = o.rollout()
    g.solve(shift=1, gait=gait2)
    Jg, qg = g.read(S.BUF_COST), g.read(S.BUF_FREQ)
    amb = check_frequencies(qg, q, margin)
    check_costs(Jg, J, kap, skip=amb)
    st, mo, _, _ = orc.mppi(J, th, cfg["lam"])
    mg, vg = g.state()
    tol = mppi_tolerance(J, th, kap, cfg["lam"], mo)
    # the first tick's GPU/oracle means differ within their tolerance, and that
    # difference enters the second tick's sampling mean linearly
    assert np.all(np.abs(mg - mo) <= tol + 2 * MEAN_ATOL), np.max(np.abs(mg - mo) - tol)
    np.testing.assert_allclose(vg, v_shift, rtol=1e-6)
    g.close()


@pytest.mark.parametrize("tile", [96, 160])
def test_spline_full_horizon_odd_tiles(cuda, tile):
    # 100 steps, 4 knots: 160-sample tiles take 43.5 KB of dynamic shared memory,
    # above 48 KB with the static block state (the launch opts in); 96 leaves
    # three warps per block.  dt = 1 ms keeps the 0.1 s horizon well conditioned.
    cfg = W.config("spline_k262144_h100")
    cfg.update(K=3001, method="mppi", compare_mppi=False, sigma_init=5.0, seed=tile, dt_us=1000)
    mppi_parity(cfg, W.problem(cfg), f"spline-T{tile}", tile=tile)


def test_spline_warm_shift(cuda):
    cfg = W.config("spline_k262144_h100")
    cfg.update(K=512, H=25, dt_us=20000, method="mppi", compare_mppi=False, sigma_init=5.0, seed=12)
    prob = W.problem(cfg)
    g = CudaRun(cfg, prob)
    g.solve()
    mg1, vg1 = g.state()
    r = g.solve(shift=1)
    # MPPI keeps the covariance, and a spline shift keeps the knot variances
    mg2, vg2 = g.state()
    np.testing.assert_allclose(vg2, vg1)
    assert r["status"] == S.OK
    g.close()


# ------------------------------------------------------------------ boundary behaviour

def test_host_memory_path_equals_device_path(cuda):
    cfg = W.config("adaptive_elite_k8192_h25")
    cfg.update(K=1024, iterations=2, seed=4)
    prob = W.problem(cfg)
    g = CudaRun(cfg, prob)
    rd = g.solve()
    md, vd = g.state()
    c2 = S.Controller(cfg)
    res = c2.solve_host(f32(prob["x0"]), f32(prob["xref"]), prob["gait"], f32(prob["f_ext"]), 0)
    cuda.cuda.synchronize()
    rh = S.parse_result(bytes(res))
    np.testing.assert_array_equal(rd["u0"], rh["u0"])
    assert rd["cost_min"] == rh["cost_min"]
    np.testing.assert_array_equal(md, c2.read(S.BUF_MEAN).cpu().numpy())
    np.testing.assert_array_equal(vd, c2.read(S.BUF_VAR).cpu().numpy())
    g.close()
    c2.close()


def test_maximum_sample_count(cuda):
    # K at its maximum (2^24), elite 1 %: sampled costs (first, middle, last and
    # scattered samples, including the last tile) match the oracle's one-sample
    # rollouts, and the multi-block selection returns exactly the K_e smallest
    # (cost, index) keys of the GPU's own costs in index order
    cfg = W.config("plain_mppi_k512_h12")
    K = S.MAX_K
    cfg.update(K=K, H=4, seed=24, method="elite", elite_count=W.elite_count(0.01, K), tile=256)
    prob = W.problem(cfg)
    g, o = CudaRun(cfg, prob, tile=256), OracleRun(cfg, prob)
    r = g.solve()
    Jg = g.read(S.BUF_COST)
    ks = [0, 1, 255, 256, K // 2, K // 2 + 77, K - 257, K - 256, K - 2, K - 1] + \
         np.random.default_rng(24).integers(0, K, size=30).tolist()
    gated = 0
    for k in ks:
        Jo = o.sample(int(k))[0]
        kap = o.kappa(int(k))
        if np.isfinite(Jo) and Jo < 3e38 and kap <= 1e-5:
            assert abs(float(Jg[k]) - Jo) <= max(1e-4, 100 * kap) * abs(Jo), (k, float(Jg[k]), Jo)
            gated += 1
    assert gated >= 0.75 * len(ks)  # a 4-step horizon keeps the rollouts well conditioned
    key = np.where(np.isfinite(Jg), Jg, np.inf).astype(np.float64)
    Ke = cfg["elite_count"]
    order = np.lexsort((np.arange(K), key))
    want = np.sort(order[:Ke])
    eg = g.read(S.BUF_ELITE)
    np.testing.assert_array_equal(eg, want)
    assert r["cost_min"] == float(key.min())
    g.close()


def test_checkpoint_resume_bit_exact(cuda):
    cfg = W.config("plain_mppi_k512_h12")
    prob = W.problem(cfg)
    g = CudaRun(cfg, prob)
    g.solve()
    blob = g.ctl.get_state()
    r1 = g.solve(shift=1)
    m1, _ = g.state()
    g.ctl.set_state(blob)
    r2 = g.solve(shift=1)
    m2, _ = g.state()
    np.testing.assert_array_equal(m1, m2)
    np.testing.assert_array_equal(r1["u0"], r2["u0"])
    fresh = S.Controller(cfg)
    fresh.set_state(blob)
    res = fresh.solve(g.x0, g.xref, prob["gait"], g.fext, 1)
    cuda.cuda.synchronize()
    np.testing.assert_array_equal(S.parse_result(res.cpu().numpy())["u0"], r1["u0"])
    g.close()
    fresh.close()


def test_all_costs_nonfinite_reports_divergence(cuda):
    cfg = W.config("plain_mppi_k512_h12")
    prob = W.problem(cfg)
    g = CudaRun(cfg, prob)
    g.solve()
    m0, v0 = g.state()
    x0 = g.x0.clone()
    x0[0] = float("nan")
    r = g.solve(shift=0, x0=x0)
    assert r["status"] == S.ERR_DIVERGED and r["n_finite"] == 0
    m1, v1 = g.state()
    np.testing.assert_array_equal(m0, m1)
    np.testing.assert_array_equal(v0, v1)
    cfg2 = dict(cfg, method="elite", elite_count=10)
    g2 = CudaRun(cfg2, prob)
    g2.solve()
    m0, v0 = g2.state()
    r = g2.solve(shift=0, x0=x0)
    assert r["status"] == S.ERR_DIVERGED
    m1, v1 = g2.state()
    np.testing.assert_array_equal(m0, m1)
    np.testing.assert_array_equal(v0, v1)
    g.close()
    g2.close()


def test_host_input_validation(cuda):
    cfg = W.config("plain_mppi_k512_h12")
    prob = W.problem(cfg)
    c = S.Controller(cfg)
    x0 = f32(prob["x0"]).copy()
    x0[3] = np.inf
    with pytest.raises(S.SBSError) as e:
        c.solve_host(x0, f32(prob["xref"]), prob["gait"], None, 0)
    assert e.value.status == S.ERR_INVALID_ARG
    bad = dict(prob["gait"], phase0=W.PHASE_ONE)
    with pytest.raises(S.SBSError):
        c.solve_host(f32(prob["x0"]), f32(prob["xref"]), bad, None, 0)
    c.close()


def test_fp32_peak_is_plausible(cuda):
    f = S.fp32_peak()
    assert 1e12 < f < 2e14
