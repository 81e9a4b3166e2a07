"""Seeded synthetic workloads for the SBS controller.

This module holds only configuration values and seeded input generators (initial
states, references, gait phases, instance mixes).  It contains none of the
controller's arithmetic, so both the CUDA path and the FP64 oracle can be fed
from it without sharing any computation.

Physical constants follow the quadruped of the paper's experiments (21 kg,
Sec. V) with the body inertia and foot positions of the single-robot workload;
the sample counts and horizons follow the paper's timing experiment (10 000
rollouts, N = 12, dt = 0.02 s, Sec. V-A) scaled to the five workloads below.
The paper publishes no dataset; every input is synthetic.
"""
from __future__ import annotations

import copy
import math

import numpy as np

PHASE_ONE = 1_000_000_000  # one gait cycle in units of 1e-9 cycle

# Per-leg phase offsets (legs FL, FR, RL, RR) and duty factors, in 1e-9 cycle.
GAITS = {
    "trot": {"offset": (0, 500_000_000, 500_000_000, 0), "duty": 600_000_000},
    "pace": {"offset": (0, 500_000_000, 0, 500_000_000), "duty": 600_000_000},
    "crawl": {"offset": (0, 500_000_000, 750_000_000, 250_000_000), "duty": 800_000_000},
}

MODEL = {
    "mass": 21.0,
    "inertia": (0.07, 0.26, 0.24),
    # body-frame foot positions relative to the CoM: FL, FR, RL, RR
    "foot": ((0.24, 0.13, -0.30), (0.24, -0.13, -0.30), (-0.24, 0.13, -0.30), (-0.24, -0.13, -0.30)),
    "gravity": (0.0, 0.0, -9.81),
}

COST = {
    # state order: p (3), roll/pitch/yaw (3), v (3), omega (3)
    "Q": (0.0, 0.0, 50.0, 10.0, 10.0, 1.0, 5.0, 5.0, 1.0, 0.1, 0.1, 0.1),
    "R": (1e-5, 1e-5, 1e-5),
    "w_fc": 1e-3,
    "mu": 0.5,
    "rho": 1.0,
    "f_nominal": 1.3,
}

BASE = {
    "P": 0,
    "method": "mppi",
    "iterations": 1,
    "elite_count": 1,
    "adaptive": False,
    "dt_us": 20_000,
    "q_init": 2000,  # 2.0 Hz in mHz
    "lam": 0.1,
    "f_min": 1.0,
    "f_max": 4.0,
    "sigma_init": 20.0,
    "sigma_min": 1.0,
    "sigma_f_init": 0.3,
    "sigma_f_min": 0.05,
    "compare_mppi": False,
    "model": MODEL,
    "cost": COST,
    "ctrl": 0,
    "gait": "trot",
    "v_ref": (0.3, 0.0),
    "f_ext": (0.0, 0.0, 0.0),
    "z_ref": 0.30,
}


def _cfg(**kw):
    c = copy.deepcopy(BASE)
    c.update(kw)
    return c


def elite_count(frac: float, K: int) -> int:
    return max(1, int(math.ceil(frac * K - 1e-9)))


def config(name: str) -> dict:
    """The controller configuration of one named workload."""
    if name == "plain_mppi_k512_h12":
        return _cfg(K=512, H=12, seed=0)
    if name == "adaptive_elite_k8192_h25":
        return _cfg(K=8192, H=25, seed=1, method="elite", iterations=5,
                    elite_count=elite_count(0.05, 8192), adaptive=True, compare_mppi=True,
                    f_ext=(0.0, 60.0, 0.0))
    if name == "spline_k262144_h100":
        # 256-sample tiles: 473 us per solve on a B300 against 494 (128), 509 (192),
        # 521 (160), 532 (96) and 557 (64)
        return _cfg(K=262144, H=100, P=4, dt_us=10_000, seed=4, method="elite",
                    elite_count=elite_count(0.01, 262144), adaptive=True, compare_mppi=True, tile=256)
    if name == "naive_freqset_k10000_h12":
        # the paper's gait-adaptation setting (Sec. V): 10 000 rollouts, N = 12,
        # dt = 0.02 s, trot, step frequency uniform over {1.3, 2.0, 2.4} Hz with one
        # force Gaussian per frequency, Naive optimiser, regulariser towards 1.3 Hz
        return _cfg(K=10_000, H=12, seed=5, method="naive", q_init=1300,
                    freq_set_mhz=(1300, 2000, 2400), v_ref=(0.5, 0.0))
    if name == "worldfeet_mppi_k4096_h25":
        # stance feet fixed on the ground with footholds placed at touchdown
        # (Sec. IV-D) over a 0.5 s horizon: every leg touches down at least once
        return _cfg(K=4096, H=25, seed=6, world_feet=True, v_ref=(0.5, 0.0))
    raise KeyError(name)


SINGLE = ("plain_mppi_k512_h12", "adaptive_elite_k8192_h25", "spline_k262144_h100", "naive_freqset_k10000_h12",
          "worldfeet_mppi_k4096_h25")


def initial_state(rng: np.random.Generator, z: float = 0.30) -> np.ndarray:
    """Nominal standing state plus a U(-0.05, 0.05) perturbation per component."""
    x = np.zeros(12)
    x[2] = z
    return x + rng.uniform(-0.05, 0.05, size=12)


def reference(H: int, dt_us: int, x0: np.ndarray, v_ref, z_ref: float = 0.30) -> np.ndarray:
    """Constant-velocity reference over the horizon: planar position advancing at
    v_ref from x0, fixed height, level attitude, zero angular velocity."""
    dt = dt_us * 1e-6
    xr = np.zeros((H, 12))
    for j in range(H):
        xr[j, 0] = x0[0] + v_ref[0] * j * dt
        xr[j, 1] = x0[1] + v_ref[1] * j * dt
        xr[j, 2] = z_ref
        xr[j, 6] = v_ref[0]
        xr[j, 7] = v_ref[1]
    return xr


def initial_feet(rng: np.random.Generator, x0: np.ndarray, model: dict = MODEL) -> np.ndarray:
    """Ground (x, y) of the 4 feet at t_0: under the nominal foot offsets from the
    CoM, plus U(-0.02, 0.02) m per coordinate (a robot mid-stride)."""
    off = np.asarray(model["foot"], dtype=np.float64)[:, :2]
    return (x0[None, :2] + off + rng.uniform(-0.02, 0.02, size=(4, 2))).ravel()


def gait(name: str, phase0: int) -> dict:
    g = GAITS[name]
    return {"offset": tuple(g["offset"]), "duty": g["duty"], "phase0": int(phase0) % PHASE_ONE}


def problem(cfg: dict, seed: int | None = None) -> dict:
    """Seeded inputs of one solve: x0, x_ref, gait (with a random phase), f_ext."""
    rng = np.random.default_rng(cfg["seed"] if seed is None else seed)
    x0 = initial_state(rng, cfg["z_ref"])
    phase0 = int(rng.integers(0, PHASE_ONE))
    out = {
        "x0": x0,
        "xref": reference(cfg["H"], cfg["dt_us"], x0, cfg["v_ref"], cfg["z_ref"]),
        "gait": gait(cfg["gait"], phase0),
        "f_ext": np.asarray(cfg["f_ext"], dtype=np.float64),
    }
    if cfg.get("world_feet"):
        out["feet"] = initial_feet(rng, x0, cfg["model"])
    return out


# Samples per tile of the batched workloads.  A 256-sample tile halves the
# per-tile work (record lookup, staging, tile-end reductions, partial rows) at the
# same occupancy as 128 and makes the 256-controller tick 1.4 % faster; single
# small controllers keep the library default of 128 for more blocks per solve.
BATCH_TILE = 256


def batch_mix(n: int = 256, seed: int = 2, Ks=(256, 1024, 4096, 16384), Hs=(10, 25, 50),
              methods=("mppi", "elite"), gaits=("trot", "pace", "crawl"), adaptive=False):
    """Uneven independent controllers: K, H, gait, method and a planar velocity
    reference drawn per instance, each with its own initial state and phase."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        K = int(rng.choice(Ks))
        H = int(rng.choice(Hs))
        method = str(rng.choice(methods))
        gname = str(rng.choice(gaits))
        v = tuple(float(a) for a in rng.uniform(-0.5, 0.5, size=2))
        c = _cfg(K=K, H=H, seed=seed, ctrl=i, method=method, gait=gname, v_ref=v,
                 elite_count=elite_count(0.05, K) if method == "elite" else 1,
                 adaptive=adaptive, tile=BATCH_TILE)
        x0 = initial_state(rng, c["z_ref"])
        phase0 = int(rng.integers(0, PHASE_ONE))
        prob = {"x0": x0, "xref": reference(H, c["dt_us"], x0, v, c["z_ref"]),
                "gait": gait(gname, phase0), "f_ext": np.zeros(3)}
        out.append((c, prob))
    return out


def batch_config(n: int = 256, seed: int = 2):
    """The batched workload: 256 controllers, K in {256, 1024, 4096, 16384},
    H in {10, 25, 50}, trot/pace/crawl, MPPI or elite (5 %)."""
    return batch_mix(n, seed)


def serving_mix(n: int = 2048, seed: int = 3):
    """The serving workload's robots: K in {1024, 4096, 16384}, H in {12, 25, 50},
    adaptive step frequency, MPPI; each robot also gets a control rate."""
    mix = batch_mix(n, seed, Ks=(1024, 4096, 16384), Hs=(12, 25, 50), methods=("mppi",),
                    gaits=("trot",), adaptive=True)
    rng = np.random.default_rng(seed + 1000)
    rates = rng.choice((50, 100, 200), size=n)
    return mix, rates
