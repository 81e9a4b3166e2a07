"""Closed-loop serving workload: simulated robots issuing controller solves.

Each robot runs its own SBS controller (its distribution and RNG counter stay
on the device between solves) and issues a solve at its control rate with
Poisson jitter, at most one outstanding at a time: a robot whose previous solve
is still running issues its next one as soon as the result is back.  Between
solves the robot is advanced by a simulated body: a single rigid body under the
last first-control forces on its stance legs, its gait phase advancing at the
controller's step frequency, and random horizontal pushes of 0-80 N.  A robot
that falls (attitude or height out of range) is reset.  The simulated body is
the robots' world, not part of the controller.

run() drives a Server (continuous batching, or plain one-solve-at-a-time) for a
fixed wall-clock window and reports solves/s, sample-steps/s and the server's
submit-to-result latency percentiles.
"""
from __future__ import annotations

import time

import numpy as np

from . import sbs as S
from . import workloads as W


class Plant:
    """Vectorised simulated robots (FP64 explicit Euler, at most two substeps per
    control interval: a coarse world model whose job is to move the state the
    controllers see)."""

    def __init__(self, n, model, rng):
        self.n = n
        self.rng = rng
        self.m = model["mass"]
        self.I = np.asarray(model["inertia"], dtype=np.float64)
        self.foot = np.asarray(model["foot"], dtype=np.float64)  # [4, 3]
        self.g = np.asarray(model["gravity"], dtype=np.float64)
        self.x = np.zeros((n, 12))
        self.reset(np.arange(n))
        self.push = np.zeros((n, 3))
        self.push_change = rng.exponential(2.0, size=n)

    def reset(self, idx):
        self.x[idx] = 0.0
        self.x[idx, 2] = 0.30
        self.x[idx] += self.rng.uniform(-0.02, 0.02, size=(len(idx), 12))

    def _deriv(self, x, u, stance):
        with np.errstate(all="ignore"):  # fallen robots are reset after the step
            return self._deriv_raw(x, u, stance)

    def _deriv_raw(self, x, u, stance):
        # Eq. (1) with body-fixed lever arms, component by component (vectorised over robots)
        sr, cr = np.sin(x[:, 3]), np.cos(x[:, 3])
        sp, cp = np.sin(x[:, 4]), np.cos(x[:, 4])
        sy, cy = np.sin(x[:, 5]), np.cos(x[:, 5])
        # body-to-world R = Rz(yaw) Ry(pitch) Rx(roll)
        r00, r01, r02 = cy * cp, cy * sp * sr - sy * cr, cy * sp * cr + sy * sr
        r10, r11, r12 = sy * cp, sy * sp * sr + cy * cr, sy * sp * cr - cy * sr
        r20, r21, r22 = -sp, cp * sr, cp * cr
        G = u.reshape(-1, 4, 3) * stance[:, :, None]
        gx, gy, gz = G[:, :, 0], G[:, :, 1], G[:, :, 2]  # [n, 4] world forces per leg
        bx = r00[:, None] * gx + r10[:, None] * gy + r20[:, None] * gz  # R^T G per leg
        by = r01[:, None] * gx + r11[:, None] * gy + r21[:, None] * gz
        bz = r02[:, None] * gx + r12[:, None] * gy + r22[:, None] * gz
        fx, fy, fz = self.foot[:, 0], self.foot[:, 1], self.foot[:, 2]
        t0 = (fy * bz - fz * by).sum(axis=1)
        t1 = (fz * bx - fx * bz).sum(axis=1)
        t2 = (fx * by - fy * bx).sum(axis=1)
        w0, w1, w2 = x[:, 9], x[:, 10], x[:, 11]
        I0, I1, I2 = self.I
        out = np.empty_like(x)
        out[:, 0:3] = x[:, 6:9]
        tp = sp / cp
        out[:, 3] = w0 + sr * tp * w1 + cr * tp * w2
        out[:, 4] = cr * w1 - sr * w2
        out[:, 5] = (sr * w1 + cr * w2) / cp
        out[:, 6] = (gx.sum(axis=1) + self.push_sel[:, 0]) / self.m + self.g[0]
        out[:, 7] = (gy.sum(axis=1) + self.push_sel[:, 1]) / self.m + self.g[1]
        out[:, 8] = (gz.sum(axis=1) + self.push_sel[:, 2]) / self.m + self.g[2]
        out[:, 9] = (t0 - (w1 * I2 * w2 - w2 * I1 * w1)) / I0
        out[:, 10] = (t1 - (w2 * I0 * w0 - w0 * I2 * w2)) / I1
        out[:, 11] = (t2 - (w0 * I1 * w1 - w1 * I0 * w0)) / I2
        return out

    def advance(self, idx, dt, u, phase, q, offset, duty, now):
        """Advance robots idx by dt seconds; phase (uint32 1e-9 cycle) advances too."""
        if len(idx) == 0:
            return phase
        change = now >= self.push_change[idx]
        if change.any():
            ci = idx[change]
            mag = self.rng.uniform(0.0, 80.0, size=len(ci)) * (self.rng.random(len(ci)) < 0.5)
            ang = self.rng.uniform(0, 2 * np.pi, size=len(ci))
            self.push[ci] = np.stack([mag * np.cos(ang), mag * np.sin(ang), np.zeros(len(ci))], -1)
            self.push_change[ci] = now + self.rng.exponential(2.0, size=len(ci))
        self.push_sel = self.push[idx]
        x = self.x[idx]
        dt = np.broadcast_to(np.asarray(dt, dtype=np.float64), (len(idx),))
        nsub = int(min(2, max(1, np.ceil(dt.max() / 0.005))))  # per-robot step dt / nsub
        h = dt / nsub
        ph = phase.astype(np.int64)
        dph = np.round(q * h * 1e6).astype(np.int64)
        for _ in range(nsub):
            st = ((ph[:, None] + offset) % W.PHASE_ONE) < duty[:, None]
            x = x + h[:, None] * self._deriv(x, u, st)
            ph = (ph + dph) % W.PHASE_ONE
        bad = ~np.isfinite(x).all(axis=1) | (np.abs(x[:, 3]) > 1.0) | (np.abs(x[:, 4]) > 1.0) | \
            (x[:, 2] < 0.1) | (x[:, 2] > 1.0)
        self.x[idx] = x
        if bad.any():
            self.reset(idx[bad])
        return ph.astype(np.uint32)


class Robots:
    """The serving mix: one controller and one simulated body per robot."""

    def __init__(self, n=2048, seed=3):
        mix, rates = W.serving_mix(n, seed)
        self.cfgs = [c for c, _ in mix]
        self.n = n
        # device memory from the library's own allocator: the dispatcher thread must
        # never wait for the Python interpreter to allocate
        self.ctls = [S.Controller(c, use_torch_allocator=False) for c in self.cfgs]
        self.handles = np.array([c.handle.value for c in self.ctls], dtype=np.uint64)
        self.K = np.array([c["K"] for c in self.cfgs])
        self.H = np.array([c["H"] for c in self.cfgs])
        self.dt = np.array([c["dt_us"] * 1e-6 for c in self.cfgs])
        self.period = 1.0 / rates
        self.v_ref = np.array([c["v_ref"] for c in self.cfgs])
        self.offset = np.array([p["gait"]["offset"] for _, p in mix], dtype=np.int64)
        self.duty = np.array([p["gait"]["duty"] for _, p in mix], dtype=np.int64)
        self.phase = np.array([p["gait"]["phase0"] for _, p in mix], dtype=np.uint32)
        self.q = np.array([c["q_init"] for c in self.cfgs], dtype=np.float64)
        self.rng = np.random.default_rng(seed + 7)
        self.plant = Plant(n, W.MODEL, self.rng)
        self.u = np.zeros((n, 12))
        self.x0 = np.zeros((n, 12), dtype=np.float32)
        self.xref = np.zeros((n, 50 * 12), dtype=np.float32)  # room for the longest horizon
        self.probs = np.zeros(n, dtype=S.PROBLEM_DTYPE)
        self.probs["host_memory"] = 1
        self.probs["x0"] = self.x0.ctypes.data + np.arange(n, dtype=np.uint64) * 48
        self.probs["xref"] = self.xref.ctypes.data + np.arange(n, dtype=np.uint64) * (50 * 12 * 4)
        self.probs["offset"] = self.offset.astype(np.uint32)
        self.probs["duty"] = self.duty.astype(np.uint32)
        self._steps = np.arange(50, dtype=np.float64)

    def prepare(self, idx, now, last_update, anchor, first):
        """Advance robots idx to `now` and fill their request records."""
        dt = now - last_update[idx]
        self.phase[idx] = self.plant.advance(idx, dt, self.u[idx], self.phase[idx], self.q[idx], self.offset[idx],
                                             self.duty[idx], now)
        last_update[idx] = now
        x = self.plant.x[idx]
        self.x0[idx] = x.astype(np.float32)
        # constant-velocity reference from the current state (planar velocity, height 0.30 m, level)
        H = 50
        t = self._steps[None, :] * self.dt[idx, None]  # [n, H] step times
        ref = np.zeros((len(idx), H, 12), dtype=np.float32)
        ref[:, :, 0] = x[:, 0:1] + self.v_ref[idx, 0:1] * t
        ref[:, :, 1] = x[:, 1:2] + self.v_ref[idx, 1:2] * t
        ref[:, :, 2] = 0.30
        ref[:, :, 6] = self.v_ref[idx, 0:1]
        ref[:, :, 7] = self.v_ref[idx, 1:2]
        self.xref[idx] = ref.reshape(len(idx), -1)
        shift = np.floor((now - anchor[idx]) / self.dt[idx]).astype(np.int64)
        shift = np.minimum(shift, self.H[idx])
        anchor[idx] += shift * self.dt[idx]
        shift[first[idx]] = 0
        self.probs["phase0"][idx] = self.phase[idx]
        self.probs["shift"][idx] = shift.astype(np.int32)
        return self.probs[idx]


def run(plain=False, n=2048, duration=4.0, warmup=1.0, slots=4, budget=8 << 30, seed=3, robots=None,
        samples_per_thread=2, theta_mode=S.THETA_REGENERATE, max_batch=192):
    """Serve n robots for warmup + duration seconds; statistics of the measured window.
    samples_per_thread, theta_mode, max_batch: the batched server's launch settings
    and requests per tick (None: all robots); plain solves take the same deviation
    mode with one sample per thread.  The defaults are the fastest of a sweep on
    B300 for this mix (2 s windows): regenerated deviations with 160-192 requests
    per tick served 199 k solves/s, stored deviations (ticks capped by the budget,
    about 185 requests) 182-186 k, regenerated without a cap (about 300 per tick,
    the slots no longer overlapping) 129-147 k."""
    import torch
    R = robots if robots is not None else Robots(n, seed)
    n = R.n
    if plain:  # plain solves use each controller's own workspace: allocate it before serving
        for c in R.ctls:
            c.prepare()
            c.set_theta_mode(theta_mode)
            c.set_samples_per_thread(1)
    server = S.Server(slots=1 if plain else slots, max_batch=max_batch or n, max_pending=4 * n, budget_bytes=budget,
                      plain=plain, samples_per_thread=samples_per_thread, theta_mode=theta_mode)
    rng = np.random.default_rng(seed + 11)
    outstanding = np.zeros(n, dtype=bool)
    tickets = np.zeros(n, dtype=np.uint64)
    t_sub = np.zeros(n)
    first = np.ones(n, dtype=bool)
    t0 = time.perf_counter()
    next_due = t0 + rng.uniform(0, 1, size=n) * R.period
    last_update = np.full(n, t0)
    anchor = np.full(n, t0)
    measuring, m_start = False, None
    done_n, done_ss, missed = 0, 0, 0
    rates = np.rint(1.0 / R.period).astype(np.int64)
    by_rate = {int(r): [0, 0] for r in np.unique(rates)}  # solves done, deadlines missed
    lat_host = []
    while True:
        now = time.perf_counter()
        if not measuring and now - t0 >= warmup:
            measuring, m_start = True, now
            server.stats(reset=True)
            done_n, done_ss, missed = 0, 0, 0
            by_rate = {r: [0, 0] for r in by_rate}
            lat_host = []
        if measuring and now - m_start >= duration:
            break
        out = np.nonzero(outstanding)[0]
        if len(out):
            st, res = server.poll(tickets[out])
            ok = st == S.OK
            if ok.any():
                fin = out[ok]
                r = res[ok]
                R.u[fin] = np.where(np.isfinite(r["u0"]), r["u0"], 0.0)
                good = r["status"] == S.OK
                R.q[fin[good]] = np.clip(r["q_freq"][good], 1000, 4000)
                outstanding[fin] = False
                lat = now - t_sub[fin]
                if measuring:
                    done_n += len(fin)
                    done_ss += int((R.K[fin] * R.H[fin]).sum())
                    late = lat > R.period[fin]
                    missed += int(late.sum())
                    for r in by_rate:
                        sel = rates[fin] == r
                        by_rate[r][0] += int(sel.sum())
                        by_rate[r][1] += int((late & sel).sum())
                    lat_host.extend(lat.tolist())
            bad = st == S.ERR_INVALID_ARG
            if bad.any():
                raise RuntimeError("server lost a ticket")
        due = np.nonzero(~outstanding & (next_due <= now))[0]
        if len(due):
            recs = R.prepare(due, now, last_update, anchor, first)
            tickets[due] = server.submit(R.handles[due], recs)
            outstanding[due] = True
            first[due] = False
            t_sub[due] = now
            gap = rng.exponential(1.0, size=len(due)) * R.period[due]
            next_due[due] = np.maximum(next_due[due] + gap, now)
        else:
            time.sleep(0)
    elapsed = time.perf_counter() - m_start
    stats = server.stats()
    # drain
    while outstanding.any():
        out = np.nonzero(outstanding)[0]
        st, _ = server.poll(tickets[out])
        outstanding[out[st == S.OK]] = False
        time.sleep(0.001)
    server.close()
    torch.cuda.synchronize()
    lat_host = np.sort(np.array(lat_host)) if lat_host else np.zeros(1)
    return {"mode": "plain" if plain else "batched", "robots": n, "seconds": elapsed,
            "solves_per_s": done_n / elapsed, "sample_steps_per_s": done_ss / elapsed,
            "latency_ms": {"p50": stats["p50_us"] / 1e3, "p99": stats["p99_us"] / 1e3, "max": stats["max_us"] / 1e3,
                           "kind": "server: submit to result on the host"},
            "host_latency_ms": {"p50": 1e3 * lat_host[len(lat_host) // 2],
                                "p99": 1e3 * lat_host[min(len(lat_host) - 1, int(0.99 * len(lat_host)))]},
            "deadline_miss_frac": missed / max(done_n, 1),
            "by_rate_hz": {str(r): {"robots": int((rates == r).sum()), "solves_per_s": d / elapsed,
                                    "offered_solves_per_s": float(r * (rates == r).sum()),
                                    "deadline_miss_frac": m / max(d, 1)} for r, (d, m) in by_rate.items()},
            "launch": {"samples_per_thread": 1 if plain else samples_per_thread,
                       "sampled_deviations": "regenerate" if theta_mode == S.THETA_REGENERATE else "store"},
            "mean_batch": stats["mean_batch"],
            "ticks": stats["ticks"], "admission_waits": stats["admission_waits"], "budget_bytes": budget,
            "offered_solves_per_s": float((1.0 / R.period).sum())}
