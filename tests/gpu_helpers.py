"""Shared helpers of the GPU parity tests: run the CUDA path and the FP64 oracle
on the same seeded inputs and compare with the tolerances below.

Tolerances (derived from the arithmetic):
  * integers (Philox words, quantised frequencies, contact flags): exact; a
    frequency whose FP64 value lies within Q_MARGIN of a rounding boundary may
    round either way on the GPU and is checked against both candidates.  The GPU
    forms f = mu_f + sigma_f z in single precision from its own normal, which is
    within 3e-6 + 2e-6 |z| of the FP64 one (|z| <= 5.77 for 24-bit uniforms): at
    sigma_f <= 0.3 Hz that moves 1000 f by at most 4.4e-3 mHz, and the
    single-precision roundings of the fused multiply-add, the product by 1000 and
    the added half by at most 6e-4 mHz more; Q_MARGIN = 6e-3 mHz covers both.
  * normals: 3e-6 + 2e-6 |z| (hardware sine/cosine of the angle); force normals
    also the radius bound min(2 e / r, sqrt(2 e)) of the hardware base-2
    logarithm (ln error e at most 2^-22 ln 2 on [0.5, 1], 3 ulp below).
  * costs: relative error <= 1e-4 for samples whose conditioning estimate
    kappa (the oracle's relative cost change under per-step rounding-sized
    perturbations) is <= 1e-6, and <= max(1e-4, 100 kappa) up to kappa = 1e-5;
    samples above that are chaotic (tumbling rollouts) and only reported.
  * MPPI mean: 1e-4 m|g| plus the first-order propagation of those cost
    tolerances through the weights: (1/lambda) sum_i w_i |theta_i - m| tol_i J_i.
  * elite set: identical except samples whose cost is within its tolerance band
    of the threshold cost.
"""
import math

import numpy as np

import oracle as orc
from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

MG = 21.0 * 9.81
MEAN_ATOL = 1e-4 * MG
Q_MARGIN = 6e-3
KAPPA_STRICT = 1e-6
KAPPA_GATED = 1e-5


def dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def f32(a):
    return np.asarray(a, dtype=np.float32)


class CudaRun:
    """One controller on the GPU with device-resident inputs."""

    def __init__(self, cfg, prob, tile=0):
        import torch
        self.cfg, self.prob = cfg, prob
        self.ctl = S.Controller(cfg, tile=tile)
        self.x0 = dev(prob["x0"])
        self.xref = dev(prob["xref"])
        self.fext = dev(prob["f_ext"])
        self.feet = dev(prob["feet"]) if "feet" in prob else None
        self.torch = torch

    def solve(self, shift=0, gait=None, x0=None, feet=None):
        res = self.ctl.solve(self.x0 if x0 is None else x0, self.xref, gait or self.prob["gait"], self.fext, shift,
                             feet=self.feet if feet is None else feet)
        self.torch.cuda.synchronize()
        return S.parse_result(res.cpu().numpy())

    def read(self, which):
        out = self.ctl.read(which).cpu().numpy()
        self.torch.cuda.synchronize()
        return out

    def state(self):
        return self.read(S.BUF_MEAN), self.read(S.BUF_VAR)

    def close(self):
        self.ctl.close()


class OracleRun:
    """The oracle on the same (single-precision-rounded) inputs."""

    def __init__(self, cfg, prob):
        self.cfg, self.prob = cfg, prob
        self.P = orc.make_params(cfg)
        self.g = orc.make_gait(prob["gait"])
        self.x0 = np.float64(f32(prob["x0"]))
        self.xref = np.float64(f32(prob["xref"]))
        self.fext = np.float64(f32(prob["f_ext"]))
        self.feet = np.float64(f32(prob["feet"])) if "feet" in prob else None
        self.mean, self.var = orc.init_dist(self.P, self.g)
        self.iter = 0

    def rollout(self, want_theta=True, kappa=True, nthreads=8):
        J, q, th, margin = orc.rollout(self.P, self.g, self.x0, self.xref, self.fext, self.mean, self.var,
                                       self.iter, want_theta=want_theta, nthreads=nthreads, feet=self.feet)
        kap = None
        if kappa:
            kap = orc.cost_condition_all(self.P, self.g, self.x0, self.xref, self.fext, self.mean, self.var,
                                         self.iter, nthreads=nthreads, feet=self.feet)
        return J, q, th, margin, kap

    def sample(self, k, q_override=-1):
        return orc.rollout_sample(self.P, self.g, self.x0, self.xref, self.fext, self.mean, self.var,
                                  self.iter, k, q_override, feet=self.feet)

    def kappa(self, k):
        return orc.cost_condition(self.P, self.g, self.x0, self.xref, self.fext, self.mean, self.var,
                                  self.iter, k, feet=self.feet)[0]

    def solve(self, shift=0, nthreads=8):
        r = orc.solve(self.P, self.g, self.x0, self.xref, self.fext, shift, self.iter, self.mean, self.var,
                      nthreads=nthreads, feet=self.feet)
        self.mean, self.var = r["mean"], r["var"]
        self.iter += self.P.iterations
        return r


def alt_frequency(o, k):
    """The other rounding of sample k's frequency (from the oracle's FP64 value)."""
    z = orc.freq_normal(o.P.seed, o.P.ctrl, k, o.iter)
    f = min(o.P.f_max, max(o.P.f_min, o.mean[-1] + math.sqrt(o.var[-1]) * z))
    lo = math.floor(1000.0 * f)
    q, _ = orc.quantise_freq(o.mean[-1], math.sqrt(o.var[-1]), z, o.P.f_min, o.P.f_max)
    return lo + 1 if q == lo else lo


def cost_tolerance(kap):
    return np.maximum(1e-4, 100.0 * kap)


def check_frequencies(q_gpu, q_orc, margin):
    """Exact except at ambiguous roundings, where either neighbour is valid."""
    amb = margin < Q_MARGIN
    assert np.array_equal(q_gpu[~amb], q_orc[~amb])
    d = np.abs(q_gpu[amb].astype(np.int64) - q_orc[amb].astype(np.int64))
    assert np.all(d <= 1)
    return amb


def check_costs(J_gpu, J_orc, kap, skip=None):
    """Cost parity gated by conditioning; returns a report dict."""
    Jg = J_gpu.astype(np.float64)
    fin = np.isfinite(J_orc) & (J_orc < 3.0e38)
    sel = np.ones(J_orc.size, bool) if skip is None else ~skip
    strict = sel & fin & (kap <= KAPPA_STRICT)
    gated = sel & fin & (kap <= KAPPA_GATED)
    rel = np.abs(Jg - J_orc) / np.maximum(np.abs(J_orc), 1e-30)
    tol = cost_tolerance(kap)
    bad = gated & ~(rel <= tol)
    assert not bad.any(), f"{bad.sum()} costs outside tolerance: rel {rel[bad][:5]} kappa {kap[bad][:5]}"
    if strict.any():
        assert rel[strict].max() <= 1e-4
    # a sample the oracle finds finite and well conditioned is finite on the GPU too
    assert np.all(np.isfinite(Jg[gated]))
    return {"n": J_orc.size, "strict": int(strict.sum()), "gated": int(gated.sum()),
            "max_rel_strict": float(rel[strict].max()) if strict.any() else 0.0,
            "max_rel_gated": float(rel[gated].max()) if gated.any() else 0.0}


def mppi_tolerance(J, th, kap, lam, mean_ref):
    """Per-dimension tolerance of the MPPI mean: accumulation term plus the
    first-order effect of the cost tolerances through the weights."""
    fin = np.isfinite(J)
    beta = J[fin].min()
    w = np.where(fin, np.exp(-(np.where(fin, J, beta) - beta) / lam), 0.0)
    w /= w.sum()
    # non-finite samples have zero weight (their conditioning estimate is NaN)
    tolJ = np.where(fin, cost_tolerance(np.where(fin, kap, 0.0)) * np.abs(np.where(fin, J, 0.0)), 0.0)
    # a weight error moves the mean only along dimensions where the sample differs
    # from it: an unbounded tolerance (infinite conditioning) times a zero
    # distance adds nothing
    diff = np.abs(th - mean_ref[None, :])
    # the mean's derivative with respect to J_k is -(w_k / lam)(theta_k - mean): a
    # sample of zero weight moves it by nothing to first order, whatever its
    # cost tolerance (an unbounded one included)
    with np.errstate(invalid="ignore"):
        wt = np.where(w == 0.0, 0.0, w * tolJ)
        prop = np.where(diff == 0.0, 0.0, wt[:, None] * diff) / lam
    return MEAN_ATOL + prop.sum(axis=0)


def elite_band_ok(gpu_set, orc_J, Ke, kap, alt_J=None):
    """The GPU elite set against the oracle's costs (Alg. 1 Sorting).

    Samples whose cost no single-precision evaluation can reproduce (conditioning
    estimate above KAPPA_GATED, or a non-finite oracle cost) may enter or leave the
    set, and each one that does moves the K_e-th place.  So the set is compared on
    the reproducible samples: among them, the GPU's elite set must be a prefix of
    the oracle's cost order up to each sample's tolerance band, i.e. no
    reproducible sample outside the set is clearly cheaper than one inside it.  A
    sample with an ambiguous frequency counts with either of its two costs (alt_J).
    Returns the size of the symmetric difference with the oracle's own set."""
    key = np.where(np.isnan(orc_J), np.inf, orc_J)
    order = np.lexsort((np.arange(key.size), key))
    orc_set = set(order[:Ke].tolist())
    gset = set(int(i) for i in gpu_set)
    tol = cost_tolerance(kap)
    with np.errstate(invalid="ignore"):
        ok = np.isfinite(key) & (kap <= KAPPA_GATED)
    band = np.where(ok, tol * np.abs(np.where(ok, key, 0.0)) * 2, np.inf)
    lo_cost, hi_cost = key.copy(), key.copy()  # the range of a sample's admissible costs
    if alt_J is not None:
        for i, a in alt_J.items():
            lo_cost[i], hi_cost[i] = min(key[i], a), max(key[i], a)
    inside = np.array(sorted(i for i in gset if ok[i]), dtype=np.int64)
    outside = np.nonzero(ok & ~np.isin(np.arange(key.size), np.fromiter(gset, np.int64)))[0]
    if inside.size and outside.size:
        worst_in = np.max(lo_cost[inside] - band[inside])
        best_out = np.min(hi_cost[outside] + band[outside])
        i_in = inside[np.argmax(lo_cost[inside] - band[inside])]
        i_out = outside[np.argmin(hi_cost[outside] + band[outside])]
        assert worst_in <= best_out, (f"sample {i_out} (cost {key[i_out]}) is outside the GPU's elite set but "
                                      f"clearly cheaper than sample {i_in} (cost {key[i_in]}) inside it")
    return len(orc_set ^ gset)


def mppi_parity(cfg, prob, name, tile=0):
    """One MPPI solve against the oracle: frequencies, costs, mean, kept variance,
    result record."""
    g, o = CudaRun(cfg, prob, tile=tile), OracleRun(cfg, prob)
    J, q, th, margin, kap = o.rollout()
    r = g.solve()
    Jg, qg = g.read(S.BUF_COST), g.read(S.BUF_FREQ)
    amb = check_frequencies(qg, q, margin)
    rep = check_costs(Jg, J, kap, skip=amb)
    st, mo, esso, beta = orc.mppi(J, th, cfg["lam"])
    mg, vg = g.state()
    tol = mppi_tolerance(J, th, kap, cfg["lam"], mo)
    assert np.all(np.abs(mg - mo) <= tol), (name, np.max(np.abs(mg - mo) - tol))
    np.testing.assert_array_equal(vg, f32(o.var))  # MPPI keeps the covariance
    assert r["status"] == S.OK
    assert r["cost_min"] == float(np.min(Jg))  # its value is covered by the cost parity above
    # the reported count is the GPU's own; the oracle agrees on every sample except
    # chaotic ones (conditioning above the gate), which may overflow on one side only
    fin_g = np.isfinite(Jg)
    assert r["n_finite"] == int(fin_g.sum())
    odd = fin_g != (np.isfinite(J) & (J < 3e38))
    assert not np.any(odd & (kap <= KAPPA_GATED)), np.nonzero(odd)[0][:5]
    u0 = orc.first_control(o.P, o.g, mo)
    np.testing.assert_allclose(r["u0"], u0, atol=float(np.max(tol[:12])))
    g.close()
    return rep


def elite_parity(cfg, prob, name, tile=0):
    """One elite solve (one iteration) against the oracle: frequencies, costs,
    the elite set up to the threshold band, and the refit as the elite mean and
    floored biased variance of the selected samples."""
    g, o = CudaRun(cfg, prob, tile=tile), OracleRun(cfg, prob)
    J, q, th, margin, kap = o.rollout()
    r = g.solve()
    Jg, qg = g.read(S.BUF_COST), g.read(S.BUF_FREQ)
    amb = check_frequencies(qg, q, margin)
    rep = check_costs(Jg, J, kap, skip=amb)
    Ke = cfg["elite_count"]
    eg = g.read(S.BUF_ELITE)
    assert np.all(np.diff(eg) > 0) and eg.size == Ke, name
    alt = {int(i): o.sample(int(i), alt_frequency(o, int(i)))[0] for i in np.nonzero(amb)[0]}
    elite_band_ok(eg, J, Ke, kap, alt)
    mg, vg = g.state()
    thg = th.copy()
    if cfg.get("adaptive"):
        thg[:, -1] = qg / 1000.0
    sel = thg[eg]
    np.testing.assert_allclose(mg, sel.mean(axis=0), atol=MEAN_ATOL, rtol=1e-5)
    floor = np.full(thg.shape[1], cfg["sigma_min"] ** 2)
    if cfg.get("adaptive"):
        floor[-1] = cfg["sigma_f_min"] ** 2
    np.testing.assert_allclose(vg, np.maximum(sel.var(axis=0), floor), rtol=2e-4, atol=1e-6)
    assert r["status"] == S.OK and r["cost_min"] == float(np.min(Jg))
    g.close()
    return rep
