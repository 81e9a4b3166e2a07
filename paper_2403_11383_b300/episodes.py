"""Closed-loop episodes: SBS controllers walking a simulated quadruped under random
external wrenches, the setting of the paper's closed-loop comparison (Sec. V-B,
Table I: success rate and cost over 50 episodes with random +-20 N/Nm wrenches)
on a single-rigid-body world instead of MuJoCo.

The world (`Body`) is an FP64 single rigid body whose stance feet stay on the
ground: each leg's contact follows the gait phase, which advances at the step
frequency the controller last chose (gait adaptation, Sec. IV-C); a leg that
touches down lands at the foothold of the leg control framework (Sec. IV-D,
Eq. (foothold)); stance legs apply the controller's first control (held over the
control period, projected onto the friction cone: the ground cannot pull or
slip); swing legs apply nothing.  A random wrench (uniform in +-W per force and
torque component) acts on the CoM, redrawn every 2 s.  An episode fails when
roll or pitch leaves +-0.8 rad or the CoM height leaves [0.12, 0.6] m.

All robots of a run are solved together by one batched launch per control tick
(sbs_batch_solve); every controller keeps its distribution on the device.

    python -m paper_2403_11383_b300.episodes --episodes 50 --seconds 10 --wrench 5
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import sbs as S
from . import workloads as W

VARIANTS = {
    # the paper's Naive controller on a fixed trot at the nominal 1.3 Hz
    "naive_fixed": dict(method="naive", q_init=1300),
    # the same with gait adaptation: step frequency from {1.3, 2.0, 2.4} Hz (Sec. V)
    "naive_adaptive": dict(method="naive", q_init=1300, freq_set_mhz=(1300, 2000, 2400)),
    # MPPI on the fixed trot
    "mppi_fixed": dict(method="mppi", q_init=1300),
}


class Body:
    """Vectorised FP64 world: n single rigid bodies with feet on the ground z = 0."""

    def __init__(self, n, model, gait, rng, q_mhz):
        self.n = n
        self.m = float(model["mass"])
        self.I = np.asarray(model["inertia"], dtype=np.float64)
        self.off = np.asarray(model["foot"], dtype=np.float64)  # [4, 3] body-frame foot offsets
        self.g = np.asarray(model["gravity"], dtype=np.float64)
        self.offset = np.asarray(gait["offset"], dtype=np.int64)
        self.duty = int(gait["duty"])
        self.x = np.zeros((n, 12))
        self.x[:, 2] = 0.30
        self.x += rng.uniform(-0.02, 0.02, size=(n, 12))
        self.feet = self.x[:, None, :2] + self.off[None, :, :2]  # under the nominal feet
        self.phase = rng.integers(0, W.PHASE_ONE, size=n).astype(np.int64)
        self.q = np.full(n, float(q_mhz))
        self.prev = self.stance()

    def stance(self):
        return ((self.phase[:, None] + self.offset[None, :]) % W.PHASE_ONE) < self.duty

    @staticmethod
    def rotation(rpy):
        sr, cr = np.sin(rpy[:, 0]), np.cos(rpy[:, 0])
        sp, cp = np.sin(rpy[:, 1]), np.cos(rpy[:, 1])
        sy, cy = np.sin(rpy[:, 2]), np.cos(rpy[:, 2])
        return np.stack([np.stack([cy * cp, cy * sp * sr - sy * cr, cy * sp * cr + sy * sr], -1),
                         np.stack([sy * cp, sy * sp * sr + cy * cr, sy * sp * cr - cy * sr], -1),
                         np.stack([-sp, cp * sr, cp * cr], -1)], -2)  # [n, 3, 3] body to world

    def land(self, legs, vd):
        """Footholds of the legs touching down now (Sec. IV-D): the hip, R (offset x,
        offset y, 0) from the CoM, plus (T_st / 2) v^d + sqrt(z / g) (v - v^d)."""
        R = self.rotation(self.x[:, 3:6])
        hips = np.einsum("nij,kj->nki", R, np.concatenate([self.off[:, :2], np.zeros((4, 1))], 1))[:, :, :2]
        tst = (self.duty / W.PHASE_ONE) / (self.q / 1000.0)
        s = np.sqrt(np.maximum(self.x[:, 2], 0.0) / -self.g[2])
        shift = 0.5 * tst[:, None] * vd + s[:, None] * (self.x[:, 6:8] - vd)
        new = self.x[:, None, :2] + hips + shift[:, None, :]
        self.feet = np.where(legs[:, :, None], new, self.feet)

    @staticmethod
    def friction(G, mu):
        """Forces the ground can carry: the orthogonal projection onto the cone."""
        s = np.hypot(G[..., 0], G[..., 1])
        t = G[..., 2]
        lam = (mu * s + t) / (1.0 + mu * mu)
        k = np.where(s > 0, mu * lam / np.where(s > 0, s, 1.0), 0.0)
        out = np.stack([k * G[..., 0], k * G[..., 1], lam], -1)
        out = np.where((s <= mu * t)[..., None], G, out)
        return np.where((mu * s <= -t)[..., None], 0.0, out)

    def step(self, u, wrench, h, vd, mu):
        """Advance h seconds under the first-control forces u [n, 12] and the world
        wrench [n, 6] (force, torque); contacts and footholds follow the gait.
        (A fallen body may overflow; it is no longer counted.)"""
        with np.errstate(all="ignore"):
            self._step(u, wrench, h, vd, mu)

    def _step(self, u, wrench, h, vd, mu):
        st = self.stance()
        self.land(st & ~self.prev, vd)
        self.prev = st
        G = self.friction(u.reshape(-1, 4, 3), mu) * st[:, :, None]
        x = self.x
        R = self.rotation(x[:, 3:6])
        rpy, v, w = x[:, 3:6], x[:, 6:9], x[:, 9:12]
        lever = np.concatenate([self.feet - x[:, None, :2], np.broadcast_to(-x[:, None, 2:3], (self.n, 4, 1))], -1)
        tau_w = np.cross(lever, G).sum(axis=1) + wrench[:, 3:]
        tau = np.einsum("nji,nj->ni", R, tau_w)  # body frame
        wd = (tau - np.cross(w, self.I[None, :] * w)) / self.I[None, :]
        sr, cr = np.sin(rpy[:, 0]), np.cos(rpy[:, 0])
        tp, cp = np.tan(rpy[:, 1]), np.cos(rpy[:, 1])
        rates = np.stack([w[:, 0] + sr * tp * w[:, 1] + cr * tp * w[:, 2], cr * w[:, 1] - sr * w[:, 2],
                          (sr * w[:, 1] + cr * w[:, 2]) / cp], -1)
        acc = (G.sum(axis=1) + wrench[:, :3]) / self.m + self.g[None, :]
        self.x = x + h * np.concatenate([v, rates, acc, wd], axis=1)
        self.phase = (self.phase + np.round(self.q * h * 1e6).astype(np.int64)) % W.PHASE_ONE

    def fallen(self):
        x = np.nan_to_num(self.x, nan=np.inf)
        return ~np.isfinite(x).all(axis=1) | (np.abs(x[:, 3]) > 0.8) | (np.abs(x[:, 4]) > 0.8) | \
            (x[:, 2] < 0.12) | (x[:, 2] > 0.6)


def run(variant="naive_adaptive", episodes=32, seconds=10.0, wrench=5.0, K=10_000, H=12, substeps=4,
        v_ref=(0.5, 0.0), seed=0, P=0, sigma=10.0, friction_project=False):
    """Run `episodes` robots for `seconds` in closed loop; returns a summary dict.
    P: spline knots per force axis (0: one force per step); sigma: the sampling
    standard deviation of each force component, N (the paper gives none; 5-10 N
    keeps this world's robots walking, 20 N makes the first controls too noisy)."""
    import torch
    base = W.config("naive_freqset_k10000_h12")
    base.update(K=K, H=H, P=P, world_feet=True, v_ref=tuple(v_ref), sigma_init=sigma,
                friction_project=friction_project)
    base.pop("freq_set_mhz", None)
    base.update(VARIANTS[variant])
    rng = np.random.default_rng(seed)
    cfgs = []
    for e in range(episodes):
        c = dict(base)
        c.update(seed=seed, ctrl=e)
        cfgs.append(c)
    ctls = [S.Controller(c) for c in cfgs]
    n = episodes
    body = Body(n, base["model"], W.GAITS[base["gait"]], rng, base["q_init"])
    batch = S.Batch(n, sum(c.workspace_bytes() + 256 for c in ctls))
    dt = base["dt_us"] * 1e-6
    steps = int(round(seconds / dt))
    vd = np.broadcast_to(np.asarray(v_ref, dtype=np.float64), (n, 2))
    x0 = torch.empty((n, 12), dtype=torch.float32, device="cuda")
    xref = torch.empty((n, H, 12), dtype=torch.float32, device="cuda")
    feet = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    fext = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    res = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    alive = np.ones(n, dtype=bool)
    survived = np.full(n, float(seconds))
    cost_sum, cost_n, freq_sum = 0.0, 0, 0.0
    Q = np.asarray(base["cost"]["Q"], dtype=np.float64)
    wrench_now = np.zeros((n, 6))
    solve_ms = []
    jj = np.arange(H)
    for k in range(steps):
        t = k * dt
        if k % int(round(2.0 / dt)) == 0:  # a new wrench every 2 s
            wrench_now = rng.uniform(-wrench, wrench, size=(n, 6))
        # controller inputs: the measured state, a reference advancing at v_ref from here
        xr = np.zeros((n, H, 12))
        xr[:, :, 0] = body.x[:, None, 0] + v_ref[0] * jj[None, :] * dt
        xr[:, :, 1] = body.x[:, None, 1] + v_ref[1] * jj[None, :] * dt
        xr[:, :, 2] = base["z_ref"]
        xr[:, :, 6] = v_ref[0]
        xr[:, :, 7] = v_ref[1]
        xs = np.where(alive[:, None], body.x, 0.0)
        xs[~alive, 2] = base["z_ref"]  # a fallen robot's controller keeps solving a standing state
        x0.copy_(torch.from_numpy(xs.astype(np.float32)))
        xref.copy_(torch.from_numpy(xr.astype(np.float32)))
        feet.copy_(torch.from_numpy(np.where(alive[:, None], body.feet.reshape(n, 8), 0.0).astype(np.float32)))
        probs = []
        for e in range(n):
            g = {"offset": tuple(int(o) for o in body.offset), "duty": body.duty, "phase0": int(body.phase[e])}
            probs.append(ctls[e].problem(x0[e], xref[e], g, fext[e], 0 if k == 0 else 1, feet=feet[e]))
        t0 = time.perf_counter()
        batch.solve(ctls, probs, res)
        out = np.frombuffer(res.cpu().numpy().tobytes(), dtype=S.RESULT_DTYPE)
        solve_ms.append((time.perf_counter() - t0) * 1e3)
        u = np.asarray(out["u0"], dtype=np.float64)
        if "freq_set_mhz" in base:  # gait adaptation: the body walks at the chosen frequency
            body.q = np.where(alive, out["q_freq"].astype(np.float64), body.q)
        freq_sum += float(body.q[alive].sum()) / 1000.0
        err = np.where(alive[:, None], body.x - xr[:, 0, :], 0.0)
        cost_sum += float((Q[None, :] * err * err).sum(axis=1).sum())
        cost_n += int(alive.sum())
        for _ in range(substeps):
            body.step(u, wrench_now, dt / substeps, vd, base["cost"]["mu"])
        fell = alive & body.fallen()
        survived[fell] = t + dt
        alive &= ~fell
        if not alive.any():
            break
    batch.close()
    for c in ctls:
        c.close()
    return {"variant": variant, "episodes": n, "seconds": seconds, "wrench": wrench, "K": K, "H": H, "P": P,
            "sigma": sigma,
            "success_rate": float(alive.mean()), "mean_survival_s": float(survived.mean()),
            "mean_tracking_cost": cost_sum / max(cost_n, 1), "mean_frequency_hz": freq_sum / max(cost_n, 1),
            "batched_solve_ms_p50": float(np.median(solve_ms))}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--variants", default="naive_fixed,naive_adaptive,mppi_fixed")
    ap.add_argument("--episodes", type=int, default=50)
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--wrench", type=float, default=5.0, help="wrench bound per component, N and Nm")
    ap.add_argument("--sigma", type=float, default=10.0, help="sampling standard deviation per force, N")
    ap.add_argument("--K", type=int, default=10_000)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    for v in a.variants.split(","):
        print(json.dumps(run(v, a.episodes, a.seconds, a.wrench, a.K, seed=a.seed, sigma=a.sigma)), flush=True)


if __name__ == "__main__":
    main()
