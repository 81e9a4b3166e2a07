"""Count the FLOPs of one sample's rollout in the FP64 oracle (its counting build)
and write the per-sample model the roofline uses.

    python oracle/count_flops.py            # writes profiles/oracle_flop_model.json

One sample of a controller with horizon H, P spline knots (0: one force per
step), S stance (leg, step) pairs over its horizon, and a sampled step
frequency (adaptive = 1) or not, costs

    F = c0 + cH H + cS S + cA adaptive          (P = 0)
    F = c0 + cH H + cS S + cA adaptive + cP P + cHP H P   (P > 0)

floating-point operations (add, sub, mul, div, sqrt; transcendentals apart)
when no friction-cone penalty term is active; each active term adds 2 (its
square and its sum), so the exact count lies in [F, F + 4 S].  The MPPI update
(Alg. 5) adds m0 + mK K + mF K_finite + mKD K D + mD D for K samples of
dimension D, K_finite of them with a finite cost.

The coefficients are solved from counted cases whose forces lie inside the
friction cone (zero variance, vertical mean forces), and every case is then
checked to equal the model exactly.  Only the oracle is called.
"""
import json
import os
import sys
from fractions import Fraction

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
from paper_2403_11383_b300 import workloads as W  # noqa: E402

OUT = os.path.join(ROOT, "profiles", "oracle_flop_model.json")


def stance_pairs(gait, q_mhz, dt_us, H):
    """S = number of (leg, step) pairs in stance over the horizon (Sec. IV-C)."""
    return sum(orc.stance(gait, i, q_mhz, dt_us, j) for i in range(4) for j in range(H))


def count_case(H, P, gname, phase0, adaptive, q_mhz=2000, dt_us=20000):
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(K=1, H=H, P=P, dt_us=dt_us, q_init=q_mhz, adaptive=adaptive)
    if adaptive:
        cfg.update(sigma_f_init=0.0)  # frequency fixed at its mean: a known schedule
    params = orc.make_params(cfg)
    gait = W.gait(gname, phase0)
    g = orc.make_gait(gait)
    D = orc.dim(params)
    nf = 12 * (P if P > 0 else H)
    mean = np.zeros(D)
    mean[2:nf:3] = 50.0  # vertical forces inside the cone: no penalty term active
    if adaptive:
        mean[-1] = q_mhz / 1000.0
    var = np.zeros(D)
    x0 = np.zeros(12)
    x0[2] = 0.30
    xref = W.reference(H, dt_us, x0, (0.3, 0.0))
    c, J = orc.count_rollout(params, g, x0, xref, np.zeros(3), mean, var, 0, 0)
    S = stance_pairs(gait, q_mhz, dt_us, H)
    return c, S


def _solve_exact(rows, rhs):
    """Integer coefficients from an exactly determined or overdetermined system
    (least squares in rationals, then checked to be integers)."""
    A = np.array(rows, dtype=np.float64)
    b = np.array(rhs, dtype=np.float64)
    sol, *_ = np.linalg.lstsq(A, b, rcond=None)
    coef = [int(round(v)) for v in sol]
    for r, y in zip(rows, rhs):
        assert sum(Fraction(a) * c for a, c in zip(r, coef)) == y, (r, y, coef)
    return coef


def fit_rollout(P_values=(0,), keys=("flop", "add", "mul", "div", "sqrt", "fn")):
    cases = []
    rng = np.random.default_rng(0)
    for P in P_values:
        for adaptive in (False, True):
            for H in ((1, 2, 3, 7, 12, 25, 50) if P == 0 else (4, 9, 12, 25, 40)):
                for gname in ("trot", "pace", "crawl"):
                    phase0 = int(rng.integers(0, W.PHASE_ONE))
                    c, S = count_case(H, P, gname, phase0, adaptive)
                    cases.append((H, P, S, int(adaptive), c))
    model = {}
    for key in keys:
        rows, rhs = [], []
        for H, P, S, A, c in cases:
            row = [1, H, S, A] + ([P, H * P] if P > 0 else [])
            rows.append(row)
            rhs.append(c[key])
        model[key] = _solve_exact(rows, rhs)
    return model, len(cases)


def fit_mppi():
    rows, rhs = [], []
    rng = np.random.default_rng(1)
    for K in (1, 2, 5, 17, 64):
        for D in (1, 12, 37):
            for nfin_frac in (1.0, 0.5):
                J = rng.uniform(0, 10, K)
                nfin = max(1, int(round(K * nfin_frac)))
                J[nfin:] = np.inf
                th = rng.normal(size=(K, D))
                c = orc.count_mppi(J, th, 0.5)
                rows.append([1, K, nfin, K * D, D])
                rhs.append(c["flop"])
    return _solve_exact(rows, rhs), len(rows)


def main():
    per_step, n0 = fit_rollout((0,))
    spline, n1 = fit_rollout((2, 4, 8))
    mppi, n2 = fit_mppi()
    out = {
        "what": "FP64 oracle operation counts (counting build, oracle/flop_count.cpp) per sample of one rollout and "
                "for the MPPI update; FLOP = add + mul + div + sqrt, transcendentals ('fn') apart",
        "command": "python oracle/count_flops.py",
        "per_step": {"terms": ["1", "H", "S", "adaptive"], "coef": per_step},
        "spline": {"terms": ["1", "H", "S", "adaptive", "P", "H*P"], "coef": spline},
        "mppi_flop": {"terms": ["1", "K", "K_finite", "K*D", "D"], "coef": mppi},
        "penalty_terms": "each active friction-penalty term adds 2 FLOP (at most 4 per stance leg-step); "
                         "the model counts none (a lower bound of the exact count)",
        "cases_checked": {"per_step": n0, "spline": n1, "mppi": n2},
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
