"""Controllers of the sample-sharding tests: every update (MPPI over many tile
groups, elite with the MPPI comparison, the histogram selection of a large K,
Naive with and without a frequency set), the spline policy, two samples per
thread, the extended model features, several iterations per tick."""
import numpy as np

from paper_2403_11383_b300 import workloads as W


def _cfg(**upd):
    def make():
        c = W.config("plain_mppi_k512_h12")
        c.update(upd, seed=2468)
        return c
    return make


CASES = {
    "mppi_k40000_groups": _cfg(K=40000, H=10, tile=128, lam=30.0),
    "mppi_adaptive_pair": _cfg(K=5000, H=25, tile=256, adaptive=True, lam=50.0, spt=2),
    "mppi_spline_p4": _cfg(K=3000, H=30, P=4, dt_us=10000, lam=30.0),
    "elite_spline_p4_pair": _cfg(K=6000, H=30, P=4, dt_us=10000, tile=256, method="elite", elite_count=60,
                                 adaptive=True, spt=2),
    "mppi_worldfeet_friction": _cfg(K=2048, H=25, world_feet=True, friction_project=True, lam=30.0),
    "elite_cmp_adaptive_it2": _cfg(K=8192, H=25, method="elite", elite_count=410, adaptive=True,
                                   compare_mppi=True, iterations=2),
    "elite_hist_k70000": _cfg(K=70000, H=8, tile=256, method="elite", elite_count=700),
    "naive_freqset": _cfg(K=3000, H=12, method="naive", q_init=1300, freq_set_mhz=(1300, 2000, 2400)),
    "naive_k777_t64": _cfg(K=777, H=12, tile=64, method="naive"),
}


def problem_tensors(prob):
    import torch

    def dev(a):
        return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
    feet = dev(prob["feet"]) if "feet" in prob else None
    return dev(prob["x0"]), dev(prob["xref"]), dev(prob["f_ext"]), feet


def ticks(cfg, prob, n=3):
    """(gait, shift) of n warm-started ticks."""
    for tick in range(n):
        g = dict(prob["gait"])
        g["phase0"] = (g["phase0"] + tick * cfg["q_init"] * cfg["dt_us"]) % W.PHASE_ONE
        yield g, (0 if tick == 0 else 1)
