"""Benchmark of the SBS controller hot path on B300.

Workload: 256 independent controllers of uneven size solved together each
control tick (K in {256, 1024, 4096, 16384}, H in {10, 25, 50}, trot/pace/crawl,
MPPI or elite 5 %), one graph-replayed batched launch set per tick (grid or
persistent mode, picked by the autotuner), inputs resident in HBM, synthetic
seeded data.  A step is one tick: rollout,
cost, update of all 256 controllers (warm-started from the previous tick).
Every timed tick (or single-controller solve) has its own CUDA events, and a
buffer of twice the L2 size is written before it, outside the events, so no
tick starts with the previous one's data in L2.

Metric: rollout sample-steps per second (sum of K*H over the controllers
solved, per second of tick time); also reported: solves/s, tick latency
p50/p99 (over at least 400 ticks), the same tick as plain
one-launch-set-per-controller solves, the end-to-end number through the C ABI
from host memory (sbs_batch_solve_host), the dominant kernel's roofline (its
algorithmic FLOPs from the FP64 oracle's counting build), the FP64 oracle's
throughput on the host cores, and each workload's per-output errors against
the oracle (`parity`, computed after the timed regions).

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU: one process per GPU (torchrun); each rank runs its own 256
controllers (weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "batched_256_uneven_K256-16384_H10-50"

# Algorithmic work of a rollout: the FP64 oracle's operation counts (its counting
# build, oracle/count_flops.py) per sample as a function of the horizon H, the
# stance (leg, step) pairs S, the knots P and a sampled frequency, and of the MPPI
# update; FLOP = add + mul + div + sqrt, transcendentals and the integer Philox
# rounds apart.  Read from profiles/oracle_flop_model.json (data, not code).
PHASE_ONE = 1_000_000_000


def flop_model():
    with open(os.path.join(ROOT, "profiles", "oracle_flop_model.json")) as f:
        return json.load(f)


def stance_pairs(gait, q_mhz, dt_us, H):
    """Stance (leg, step) pairs of each sample's horizon for step frequencies q
    (mHz, array): the integer contact schedule of Sec. IV-C."""
    q = np.atleast_1d(np.asarray(q_mhz, dtype=np.int64))
    j = np.arange(H, dtype=np.int64)
    S = np.zeros(q.size, dtype=np.int64)
    for off in gait["offset"]:
        ph = (int(gait["phase0"]) + int(off) + j[None, :] * q[:, None] * int(dt_us)) % PHASE_ONE
        S += (ph < int(gait["duty"])).sum(axis=1)
    return S


def controller_flops(model, cfg, gait, q=None, n_finite=None):
    """Algorithmic FLOPs of one iteration of a controller: (every sample's
    rollout, the MPPI weighted mean over its samples).  q: the samples' step
    frequencies (mHz) when sampled, else the nominal one; n_finite: samples of
    finite cost (default all).  The friction-penalty terms the model leaves out
    (2 FLOP each when active) make this a lower bound."""
    P, H, K = cfg.get("P", 0), cfg["H"], cfg["K"]
    ad = 1 if cfg.get("adaptive") else 0
    fam = model["spline" if P > 0 else "per_step"]["coef"]["flop"]
    S = stance_pairs(gait, cfg["q_init"] if q is None else q, cfg["dt_us"], H)
    S_tot = int(S.sum()) * (K if q is None else 1)
    roll = K * (fam[0] + fam[1] * H + fam[3] * ad) + fam[2] * S_tot
    if P > 0:
        roll += K * (fam[4] * P + fam[5] * H * P)
    m = model["mppi_flop"]["coef"]
    D = 12 * (P if P > 0 else H) + ad
    kf = K if n_finite is None else int(n_finite)
    mppi = m[0] + m[1] * K + m[2] * kf + m[3] * K * D + m[4] * D
    return int(roll), int(mppi)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="sbs", choices=["sbs", "reference"])
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--tile", type=int, default=0,
                    help="samples per block of the batched controllers; 0: timed at 128 and 256, fastest kept")
    ap.add_argument("--launch", default="auto", choices=["auto", "grid", "persistent"],
                    help="batched launch mode; auto: measured by the autotuner (with --spt and --theta)")
    ap.add_argument("--spt", type=int, default=0, choices=[0, 1, 2, 3],
                    help="samples per thread of the rollout (3: one sample and a noise thread per sample, "
                         "single-controller workloads only); 0: autotuned")
    ap.add_argument("--theta", default="auto", choices=["auto", "store", "regenerate"],
                    help="sampled deviations stored or regenerated; auto: autotuned")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline and the parity record")
    ap.add_argument("--no-parity", action="store_true", help="skip the per-output FP64 error record")
    ap.add_argument("--no-serving", action="store_true", help="skip the closed-loop serving comparison")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the serialised plain-solve comparison (its controllers' own workspaces)")
    ap.add_argument("--serving-seconds", type=float, default=3.0)
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "plain_mppi_k512_h12", "adaptive_elite_k8192_h25", "spline_k262144_h100",
                             "naive_freqset_k10000_h12", "worldfeet_mppi_k4096_h25"],
                    help="batched: the 256-controller tick (default); otherwise one controller's solves")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "sbs" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        # time nothing until nvidia-smi has written its first sample: its start-up
        # contends for the driver, its steady 200 ms polling barely does
        deadline = time.time() + 5.0
        while self.proc is not None and self.proc.poll() is None and time.time() < deadline:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.02)
        time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        self.proc.wait()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


class L2Flush:
    """Writes a device buffer of twice the L2 size between timed iterations, so
    each tick or solve starts with nothing of the previous one cached; the write
    runs outside the iteration's CUDA events."""

    def __init__(self, dev):
        import torch
        l2 = getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or (126 << 20)
        self.bytes = 2 * int(l2)
        self.buf = torch.empty(self.bytes, dtype=torch.uint8, device=dev)
        self.n = 0

    def __call__(self):
        self.n += 1
        self.buf.fill_(self.n & 0xFF)

    def describe(self):
        return (f"L2 flushed between timed iterations: {self.bytes / 2**20:.0f} MiB (2 x L2) written "
                f"before each tick or solve, outside its CUDA events")


def timed_iterations(fn, steps, flush, stream):
    """Device time (ms) of each of `steps` calls of fn on the stream, with the L2
    flushed before each call, outside the call's events."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def timed_host_iterations(fn, steps, flush):
    """Wall time (s) of each of `steps` synchronous calls of fn, with the L2
    flushed (and the device idle) before each call."""
    import torch
    out = []
    for _ in range(steps):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        out.append(time.perf_counter() - t0)
    return out


def solve_launches(cfg):
    """Kernel launches of one plain solve: per iteration the rollout, and for elite
    and Naive the selection (five kernels for an elite set chosen from more than
    32 768 costs) and the refit."""
    if cfg["method"] == "mppi":
        return cfg["iterations"]
    select = 5 if cfg["method"] == "elite" and cfg["K"] > 32768 else 1
    return cfg["iterations"] * (2 + select)


def rollout_traffic(mode, spt, theta):
    """DRAM bytes per sample-step of the rollout kernel from the committed ncu
    record, or None when the kernel sources changed since that capture or the
    record was taken in another launch setting."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "rollout_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    h = hashlib.sha256()
    for src in rec["sources"]:
        with open(os.path.join(ROOT, src), "rb") as g:
            h.update(g.read())
    same = (rec.get("launch_mode"), rec.get("samples_per_thread"), rec.get("sampled_deviations")) == (mode, spt, theta)
    return rec["dram_bytes_per_sample_step"] if h.hexdigest() == rec["sources_sha256"] and same else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


# ----------------------------------------------------------------------------- CPU oracle

def oracle_rate(mix, budget_s, nthreads):
    """Sample-steps/s of the FP64 oracle on the first instances of the mix that fit
    the time budget (one solve each, all host cores)."""
    import oracle as orc
    done_ss, t_used, n = 0, 0.0, 0
    for cfg, prob in mix:
        if t_used > budget_s:
            break
        P = orc.make_params(cfg)
        g = orc.make_gait(prob["gait"])
        mean, var = orc.init_dist(P, g)
        t0 = time.perf_counter()
        orc.solve(P, g, np.float64(np.float32(prob["x0"])), np.float64(np.float32(prob["xref"])),
                  prob["f_ext"], 0, 0, mean, var, nthreads=nthreads)
        t_used += time.perf_counter() - t0
        done_ss += cfg["K"] * cfg["H"]
        n += 1
    return done_ss / t_used, n, done_ss, t_used


def run_reference(args, world, rank):
    """The FP64 oracle as the reference arm (host cores), same workload and metric."""
    if rank != 0:
        return
    from paper_2403_11383_b300 import workloads as W
    mix = W.batch_config(args.instances)
    nthreads = os.cpu_count() or 1
    # one step = one solve of each of the first 8 controllers of the mix
    sub = mix[:8]
    for _ in range(args.warmup):
        oracle_rate(sub, 1e9, nthreads)
    t0 = time.perf_counter()
    ss = 0
    for _ in range(args.steps):
        r, n, s_, t_ = oracle_rate(sub, 1e9, nthreads)
        ss += s_
    dt = time.perf_counter() - t0
    value = ss / dt
    sample = "8 of the 256 controllers per step, one FP64 solve each"
    line = {"impl": "reference", "metric": "rollout sample-steps/s", "value": value, "unit": "sample-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances": args.instances, "parallelism": "host threads"},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": "sample-steps/s", "cores": nthreads,
                             "sample": sample},
            "e2e": {"value": value, "unit": "sample-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- parity record

MEAN_ATOL = 1e-4 * 21.0 * 9.81  # 1e-4 m|g|: the updated controls' tolerance
Q_MARGIN = 6e-3  # mHz: a frequency this close to a rounding boundary may round either way


def parity_one(cfg, prob, nthreads, n_cost=4096, seed=0):
    """Errors of one GPU solve (iteration 0, from the initial distribution,
    through sbs_solve) against the FP64 oracle on the same seeded inputs.
    Costs: relative error on the samples whose conditioning estimate kappa is at
    most 1e-5 (the gate of the parity tests; a random subset of n_cost samples
    when K is larger).  Update: staged, i.e. the FP64 update formed from the
    GPU's own costs and frequencies on the oracle's samples; also end to end (the
    oracle's own costs), reported only."""
    import torch

    import oracle as orc
    from paper_2403_11383_b300 import sbs as S
    cfg = dict(cfg, iterations=1)
    ctl = S.Controller(cfg)
    dv = lambda a: torch.tensor(np.float32(a), device="cuda")
    feet = dv(prob["feet"]) if "feet" in prob else None
    res = ctl.solve(dv(prob["x0"]), dv(prob["xref"]), prob["gait"], dv(prob["f_ext"]), 0, feet=feet)
    torch.cuda.synchronize()
    r = S.parse_result(res.cpu().numpy())
    Jg = ctl.read(S.BUF_COST).cpu().numpy().astype(np.float64)
    qg = ctl.read(S.BUF_FREQ).cpu().numpy()
    mg, vg = ctl.read(S.BUF_MEAN).cpu().numpy(), ctl.read(S.BUF_VAR).cpu().numpy()
    eg = ctl.read(S.BUF_ELITE).cpu().numpy() if cfg["method"] == "elite" else None
    mm = ctl.read(S.BUF_MPPI_MEAN).cpu().numpy() if cfg.get("compare_mppi") else None
    ctl.close()
    P, g = orc.make_params(cfg), orc.make_gait(prob["gait"])
    f64 = lambda a: np.float64(np.float32(a))
    ft = f64(prob["feet"]) if "feet" in prob else None
    x0, xr, fe = f64(prob["x0"]), f64(prob["xref"]), f64(prob["f_ext"])
    m0, v0 = orc.init_dist(P, g)
    J, q, th, margin = orc.rollout(P, g, x0, xr, fe, m0, v0, 0, want_theta=True, nthreads=nthreads, feet=ft)
    K = cfg["K"]
    idx = np.arange(K) if K <= n_cost else np.sort(np.random.default_rng(seed).choice(K, n_cost, replace=False))
    if idx.size == K:
        kap = orc.cost_condition_all(P, g, x0, xr, fe, m0, v0, 0, nthreads=nthreads, feet=ft)
    else:
        kap = np.array([orc.cost_condition(P, g, x0, xr, fe, m0, v0, 0, int(k), feet=ft)[0] for k in idx])
    Jo, Jgi = J[idx], Jg[idx]
    fin_o = np.isfinite(Jo) & (Jo < 3e38)
    amb = margin[idx] < Q_MARGIN
    gated = fin_o & ~amb & (kap <= 1e-5)
    rel = np.abs(Jgi - Jo) / np.maximum(np.abs(Jo), 1e-30)
    out = {"K": K, "H": cfg["H"], "P": cfg.get("P", 0), "method": cfg["method"], "adaptive": bool(cfg.get("adaptive")),
           "samples_checked": int(idx.size), "finite_frac_oracle": float(fin_o.mean()),
           "finite_frac_gpu": float(np.isfinite(Jg).mean()), "gated": int(gated.sum()),
           "gated_frac": float(gated.mean()),
           "cost_rel_err_gated": {"max": float(rel[gated].max()) if gated.any() else None,
                                  "p99": float(np.quantile(rel[gated], 0.99)) if gated.any() else None},
           "freq_exact_frac": float(np.mean(qg[idx] == q[idx])) if cfg.get("adaptive") else None}
    thg = th.copy()
    if cfg.get("adaptive"):
        thg[:, -1] = qg / 1000.0
    fin_g = np.isfinite(Jg)
    if cfg["method"] == "mppi" and fin_g.any():
        _, mo, ess_o, _ = orc.mppi(Jg, thg, cfg["lam"])
        out["staged"] = {"mean_abs_err": float(np.abs(mg - mo).max()),
                         "u0_abs_err": float(np.abs(np.asarray(r["u0"]) - orc.first_control(P, g, mo)).max()),
                         "ess_rel_err": float(abs(r["ess"] - ess_o) / ess_o), "ess": float(ess_o)}
        _, me, _, _ = orc.mppi(J, th, cfg["lam"])
        out["end_to_end"] = {"mean_abs_err": float(np.abs(mg - me).max()),
                             "u0_abs_err": float(np.abs(np.asarray(r["u0"]) - orc.first_control(P, g, me)).max())}
    elif cfg["method"] == "elite" and fin_g.any():
        Ke = cfg["elite_count"]
        order = np.lexsort((np.arange(K), np.where(fin_g, Jg, np.inf)))
        sel = thg[eg]
        floor = np.full(thg.shape[1], cfg["sigma_min"] ** 2)
        if cfg.get("adaptive"):
            floor[-1] = cfg["sigma_f_min"] ** 2
        vref = np.maximum(sel.var(axis=0), floor)
        out["staged"] = {"elite_set_is_first_Ke_of_gpu_costs": bool(np.array_equal(eg, np.sort(order[:Ke]))),
                         "mean_abs_err": float(np.abs(mg - sel.mean(axis=0)).max()),
                         "var_rel_err": float(np.max(np.abs(vg - vref) / vref))}
        eo = orc.elite_select(J, Ke)
        out["end_to_end"] = {"elite_overlap_frac": len(set(eo.tolist()) & set(eg.tolist())) / Ke,
                             "mean_abs_err": float(np.abs(mg - th[eo].mean(axis=0)).max())}
        if mm is not None:
            _, mo, _, _ = orc.mppi(Jg, thg, cfg["lam"])
            out["staged"]["compare_mppi_mean_abs_err"] = float(np.abs(mm - mo).max())
    return out


def parity_record(mix, tile, nthreads):
    """Per-output FP64 errors of the workloads (outside any timed region)."""
    from paper_2403_11383_b300 import workloads as W
    t0 = time.perf_counter()
    rec = {"tolerances": {"cost_rel": "1e-4 for kappa <= 1e-6, max(1e-4, 100 kappa) up to kappa = 1e-5, "
                                      "samples above reported only",
                          "mean_abs": MEAN_ATOL, "ess_rel": 1e-4},
           "kind": "GPU iteration-0 solves (sbs_solve; a batched tick gives the same bits) against the FP64 "
                   "oracle on the same seeded inputs"}
    rec["batched_mix_first8"] = [parity_one(dict(c, tile=tile), p, nthreads) for c, p in mix[:8]]
    for name in ("plain_mppi_k512_h12", "adaptive_elite_k8192_h25", "spline_k262144_h100"):
        cfg = W.config(name)
        rec[name] = parity_one(cfg, W.problem(cfg), nthreads, n_cost=512 if cfg["K"] > 100000 else 8192)
    smix, _ = W.serving_mix(2048, seed=3)
    rec["serving_mix_first4"] = [parity_one(c, p, nthreads) for c, p in smix[:4]]
    rec["seconds"] = time.perf_counter() - t0
    return rec


# ----------------------------------------------------------------------------- single controller

def run_single(args, world, rank, local):
    """Timed solves of one controller of a named workload (warm-started ticks)."""
    import torch
    from paper_2403_11383_b300 import sbs as S
    from paper_2403_11383_b300 import workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    cfg = W.config(args.workload)
    prob = W.problem(cfg)
    ctl = S.Controller(cfg)
    x0, xref, fe = (torch.tensor(np.float32(prob[k]), device=dev) for k in ("x0", "xref", "f_ext"))
    # ground-fixed stance feet ([4, 2] positions) for the controllers that use them
    feet = torch.tensor(np.float32(prob["feet"]), device=dev) if "feet" in prob else None
    res = torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device=dev)
    for w in range(max(args.warmup, 3)):
        ctl.solve(x0, xref, prob["gait"], fe, 0 if w == 0 else 1, res, feet=feet)
    p1 = ctl.problem(x0, xref, prob["gait"], fe, 1, feet=feet)  # built once, as a control loop would
    if args.spt or args.theta != "auto":  # fixed for a profiling capture, which would distort the tuner's timings
        tune = {}
        if args.spt:
            ctl.set_samples_per_thread(args.spt)
        if args.theta != "auto":
            ctl.set_theta_mode(S.THETA_REGENERATE if args.theta == "regenerate" else S.THETA_STORE)
    else:
        tune = ctl.autotune(p1, res, ticks=5)  # samples per thread x stored or regenerated deviations
    flush = L2Flush(dev)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    torch.cuda.nvtx.range_push("timed")
    solve_ms = timed_iterations(lambda: ctl.solve_packed(p1, res), args.steps, flush, stream)
    torch.cuda.nvtx.range_pop()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(sum(solve_ms) / args.steps, world, dev)
    ss = cfg["K"] * cfg["H"] * cfg["iterations"]
    # algorithmic FLOPs of a solve from the oracle's counts: every iteration's
    # rollouts (sampled frequencies: the last solve's), and the MPPI mean of an
    # MPPI solve, or of the first iteration when the elite solve compares MPPI
    rr = S.parse_result(res.cpu().numpy())
    qs = ctl.read(S.BUF_FREQ).cpu().numpy() if cfg.get("adaptive") else None
    roll_fl, mppi_fl = controller_flops(flop_model(), cfg, prob["gait"], qs, rr["n_finite"])
    n_mppi = cfg["iterations"] if cfg["method"] == "mppi" else (1 if cfg.get("compare_mppi") else 0)
    fl = cfg["iterations"] * roll_fl + n_mppi * mppi_fl
    # the solve is rollout + (select + refit) launches; the roofline uses the whole solve
    achieved = fl / (ms * 1e-3) / 1e12
    peak = S.fp32_peak() / 1e12
    # host inputs and result, synchronised per solve
    hx0, hxr, hfe = (np.ascontiguousarray(np.float32(prob[k])) for k in ("x0", "xref", "f_ext"))
    hfeet = np.ascontiguousarray(np.float32(prob["feet"])) if "feet" in prob else None
    r = S.Result()
    hp = ctl.problem(hx0, hxr, prob["gait"], hfe, 1, host=True, feet=hfeet)
    torch.cuda.synchronize()

    def host_solve():
        ctl.solve_packed(hp, r)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks(sum(timed_host_iterations(host_solve, args.steps, flush)) / args.steps, world, dev)
    if rank == 0:
        line = {"metric": "rollout sample-steps/s", "value": world * ss / (ms * 1e-3), "unit": "sample-steps/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": args.workload, "K": cfg["K"], "H": cfg["H"], "P": cfg.get("P", 0),
                           "iterations": cfg["iterations"], "method": cfg["method"], "tile": ctl.tile,
                           "samples_per_thread": ctl.samples_per_thread(),
                           "sampled_deviations": "regenerate" if ctl.theta_mode() == S.THETA_REGENERATE else "store",
                           "autotune_ms_per_solve": {f"spt{k[0]}_{'regen' if k[1] else 'store'}": v
                                                     for k, v in tune.items()} or None,
                           "fixed_by_flags": {k: v for k, v in (("spt", args.spt), ("theta", args.theta))
                                              if v not in (0, "auto")} or None,
                           "l2": flush.describe(), "parallelism": f"replicas x{world}"},
                "solves_per_s": world / (ms * 1e-3),
                "roofline": {"kernel": "whole solve", "bound": "alu", "achieved": achieved, "peak": peak,
                             "unit": "TFLOP/s", "frac": achieved / peak,
                             "peak_kind": "FP32 FMA-chain microbenchmark on this GPU (live)",
                             "flops_per_solve": fl, "flops_per_sample_step": fl / ss,
                             "flops_source": "FP64 oracle counting build (profiles/oracle_flop_model.json)",
                             "traffic": None},
                "e2e": {"value": world * ss / e2e_s, "unit": "sample-steps/s",
                        "h2d_bytes_per_step": int(4 * (12 + 3 + 12 * cfg["H"] + (8 if "feet" in prob else 0))),
                        "d2h_bytes_per_step": S.RESULT_BYTES},
                "gpu_launches": args.steps * solve_launches(cfg),
                "clocks": clk}
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    if args.workload != "batched":
        run_single(args, world, rank, local)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    import torch
    from paper_2403_11383_b300 import sbs as S
    from paper_2403_11383_b300 import tuning
    from paper_2403_11383_b300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    mix = W.batch_config(args.instances)
    x0 = [torch.tensor(np.float32(p["x0"]), device=dev) for _, p in mix]
    xref = [torch.tensor(np.float32(p["xref"]), device=dev) for _, p in mix]
    fext = [torch.tensor(np.float32(p["f_ext"]), device=dev) for _, p in mix]
    gaits = [dict(p["gait"]) for _, p in mix]
    # samples per block: timed on this mix at each candidate before the controllers are built
    if args.tile:
        tile, tile_ms = args.tile, None
    else:
        tile, tile_ms = tuning.tile_for_batch([c for c, _ in mix], list(zip(x0, xref, gaits, fext)))
    for c, _ in mix:
        c["tile"] = tile
    ctls = [S.Controller(c) for c, _ in mix]
    n = len(ctls)
    ss_tick = sum(c["K"] * c["H"] for c, _ in mix)
    mppi_ss = sum(c["K"] * c["H"] for c, _ in mix if c["method"] == "mppi")
    mppi_n = sum(1 for c, _ in mix if c["method"] == "mppi")
    # workspaces for stored deviations, unless the deviations are fixed to be regenerated
    ws_mode = S.THETA_REGENERATE if args.theta == "regenerate" else S.THETA_STORE
    arena = sum(c.workspace_bytes_mode(ws_mode) + 256 for c in ctls)
    batch = S.Batch(n, 2 * arena, inflight=2)  # two ticks in flight: the next is prepared while one runs
    if args.theta != "auto":  # from the first tick: the arena may fit only this mode
        batch.set_theta_mode(ws_mode)
    results = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device=dev)

    def problems(shift):
        return [ctls[i].problem(x0[i], xref[i], gaits[i], fext[i], shift) for i in range(n)]

    probs0, probs1 = problems(0), problems(1)

    packed0, packed1 = S.Packed(ctls, probs0), S.Packed(ctls, probs1)  # marshalled once

    def tick(first=False):
        batch.solve_packed(packed0 if first else packed1, results)

    # warm-up (the first tick initialises every controller), then the launch-mode
    # autotuner measures both modes on this mix and keeps the faster
    for w in range(max(args.warmup, 3)):
        tick(first=(w == 0))
    tune_ms = batch.autotune(ctls, probs1, results, ticks=5)
    # fixed choices (profiling captures) replace the autotuner's
    if args.launch != "auto":
        batch.set_mode(S.BATCH_GRID if args.launch == "grid" else S.BATCH_PERSISTENT)
    if args.spt:
        batch.set_samples_per_thread(args.spt)
    if args.theta != "auto":
        batch.set_theta_mode(S.THETA_REGENERATE if args.theta == "regenerate" else S.THETA_STORE)
    mode = "grid" if batch.mode() == S.BATCH_GRID else "persistent"
    spt = batch.samples_per_thread() or 1
    theta = "regenerate" if batch.theta_mode() == S.THETA_REGENERATE else "store"
    fixed = {k: v for k, v in (("launch", args.launch), ("spt", args.spt), ("theta", args.theta))
             if v not in ("auto", 0)}
    for _ in range(3):  # rebuild the tick graphs in the chosen mode before timing
        tick()
    flush = L2Flush(dev)
    torch.cuda.synchronize()

    # ---- timed region: K ticks on the stream, each timed by its own events with
    # the L2 flushed before it
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")  # profilers can select exactly the timed launches
    tick_ms = timed_iterations(tick, args.steps, flush, stream)
    torch.cuda.nvtx.range_pop()
    barrier(world)
    clk = clocks.stop()
    ms = sum(tick_ms) / args.steps
    ms = max_over_ranks(ms, world, dev)
    value = world * ss_tick / (ms * 1e-3)

    # ---- tick latency distribution (device time of each tick)
    n_lat = max(args.steps, 400)  # enough ticks for a 99th percentile
    lat = sorted(timed_iterations(tick, n_lat, flush, stream))
    p50, p99 = lat[len(lat) // 2], lat[min(len(lat) - 1, int(0.99 * len(lat)))]

    # ---- stage durations with per-stage events (dominant kernel for the roofline)
    batch.set_profiling(True)
    st = []
    for _ in range(args.steps):
        flush()
        tick()
        st.append(batch.stage_ms())
    batch.set_profiling(False)
    st = np.array(st)
    roll_ms = float(st[:, 0].mean())
    sel_ms, ref_ms = float(st[:, 1].mean()), float(st[:, 2].mean())
    # algorithmic FLOPs of the rollout launch (every controller's samples, and the
    # MPPI controllers' weighted means formed in the same launch), from the FP64
    # oracle's operation counts; finite counts from the last profiled tick
    model = flop_model()
    last = [S.parse_result(results[i * S.RESULT_BYTES:(i + 1) * S.RESULT_BYTES].cpu().numpy()) for i in range(n)]
    flops_launch = 0
    for i, ((c, _), r) in enumerate(zip(mix, last)):
        roll_fl, mppi_fl = controller_flops(model, c, gaits[i], None, r["n_finite"])
        flops_launch += roll_fl + (mppi_fl if c["method"] == "mppi" else 0)
    achieved = flops_launch / (roll_ms * 1e-3) / 1e12
    # algorithmic bytes of the elite update: the selection reads each cost once and
    # writes the elite indices; the refit reads each elite's deviation row (48 B)
    # and index per step, and reads and writes the distribution (mean, variance)
    sel_bytes = ref_bytes = 0
    for c, _ in mix:
        if c["method"] == "mppi":
            continue
        ke = c["elite_count"] if c["method"] == "elite" else 1
        d = 12 * c["H"] + (1 if c.get("adaptive") else 0)
        sel_bytes += 4 * c["K"] + 4 * ke
        # stored deviations: each elite's row (48 B) and index per step; regenerated:
        # the indices only
        ref_bytes += ((48 if theta == "store" else 0) + 4) * ke * c["H"] + 16 * d
    fp32_peak = S.fp32_peak() / 1e12
    nominal = 148 * 128 * 2 * 2032e6 / 1e12

    # ---- plain form: one sbs_solve (its own launches) per controller, serialised
    plain_ms = None
    if not args.no_plain:
        plain_ticks = max(3, min(args.steps, 40))
        pres = [torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device=dev) for _ in range(n)]

        def plain_tick():
            for i in range(n):
                ctls[i].solve(x0[i], xref[i], gaits[i], fext[i], 1, pres[i])
        plain_tick()
        torch.cuda.synchronize()
        plain_ms = sum(timed_iterations(plain_tick, plain_ticks, flush, stream)) / plain_ticks

    # ---- end to end through the C ABI from host memory: the inputs sit in the
    # batch's pinned staging buffer (written there once, as a control loop writes
    # each tick's inputs: sbs_batch_host_inputs); every timed sbs_batch_solve_host
    # copies them to the device in one transfer, runs the tick and returns with
    # the results on the host
    h_x0 = [np.ascontiguousarray(np.float32(p["x0"])) for _, p in mix]
    h_xr = [np.ascontiguousarray(np.float32(p["xref"])) for _, p in mix]
    h_fe = [np.ascontiguousarray(np.float32(p["f_ext"])) for _, p in mix]
    hpacked, views = batch.host_inputs(ctls, gaits, shift=1)
    for i, v in enumerate(views):
        v["x0"][:] = h_x0[i]
        v["xref"][:] = h_xr[i]
        v["f_ext"][:] = h_fe[i]
    h_out = np.zeros(n * S.RESULT_BYTES, dtype=np.uint8)
    for _ in range(3):
        batch.solve_host(hpacked, h_out)
    torch.cuda.synchronize()
    barrier(world)
    e2e_s = sum(timed_host_iterations(lambda: batch.solve_host(hpacked, h_out), args.steps, flush)) / args.steps
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e_value = world * ss_tick / e2e_s
    h2d_bytes = sum(4 * (a.size + b.size + c.size) for a, b, c in zip(h_x0, h_xr, h_fe))
    status = [S.parse_result(h_out[i * S.RESULT_BYTES:(i + 1) * S.RESULT_BYTES])["status"] for i in range(n)]

    # ---- served: 2048 closed-loop robots, continuous batching vs plain solves
    served = None
    if not args.no_serving:
        from paper_2403_11383_b300 import serving
        robots = serving.Robots(2048, seed=3)
        served = {"batched": serving.run(plain=False, duration=args.serving_seconds, warmup=1.0, robots=robots),
                  "plain": serving.run(plain=True, duration=args.serving_seconds, warmup=1.0, robots=robots)}
        del robots

    # ---- CPU baseline: the FP64 oracle on a bounded sample (rank 0), and the
    # per-output errors of the GPU path against it
    cpu = parity = None
    if rank == 0 and not args.no_cpu:
        nthreads = os.cpu_count() or 1
        rate, ninst, ss, t_ = oracle_rate(W.batch_config(args.instances), 15.0, nthreads)
        cpu = {"value": rate, "unit": "sample-steps/s", "cores": nthreads, "kind": "oracle",
               "sample": f"first {ninst} controllers of the mix, one FP64 solve each ({ss} sample-steps, "
                         f"{t_:.1f} s)"}
        if not args.no_parity:
            parity = parity_record(W.batch_config(args.instances), tile, nthreads)

    peaks = measured_peaks()
    traffic_ss = rollout_traffic(mode, spt, theta)
    if rank == 0:
        line = {
            "metric": "rollout sample-steps/s", "value": value, "unit": "sample-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances": n, "sample_steps_per_tick": ss_tick,
                       "tile": tile, "tile_autotune_ms_per_tick": tile_ms, "graph": True, "launch_mode": mode,
                       "autotune_ms_per_tick": {"grid": tune_ms[0], "persistent": tune_ms[1]},
                       "samples_per_thread": spt, "sampled_deviations": theta,
                       "fixed_by_flags": fixed or None,
                       "l2": flush.describe(), "workspace_bytes": 2 * arena,
                       "parallelism": f"replicas x{world}"},
            "solves_per_s": world * n / (ms * 1e-3),
            "latency_ms": {"p50": p50, "p99": p99, "ticks": len(lat),
                           "kind": f"device time of one {len(mix)}-controller tick"},
            "plain": None if plain_ms is None else
                     {"ms_per_tick": plain_ms, "sample_steps_per_s": ss_tick / (plain_ms * 1e-3),
                      "solves_per_s": n / (plain_ms * 1e-3), "kind": f"{n} serialised sbs_solve calls"},
            "stages_ms": {"rollout": roll_ms, "select": sel_ms, "refit": ref_ms},
            "roofline": {"kernel": {("grid", 1): "k_grid_rollout_lean", ("grid", 2): "k_grid_rollout_pair",
                                    ("persistent", 1): "k_batch_rollout<0, false>",
                                    ("persistent", 2): "k_batch_rollout_pair"}[(mode, spt)],
                         "bound": "alu", "achieved": achieved,
                         "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "peak_kind": "FP32 FMA-chain microbenchmark on this GPU (live)",
                         "nominal_peak": nominal, "frac_of_nominal": achieved / nominal,
                         "flops_per_launch": flops_launch,
                         "traffic": None if traffic_ss is None else traffic_ss * ss_tick,
                         "traffic_note": "ncu DRAM read+write of the rollout launches of this workload's tick "
                                         "in the same launch setting (one-pass capture, "
                                         "profiles/rollout_traffic.json), per sample-step times this tick's "
                                         "sample-steps"},
            "update_roofline": {
                "bound": "hbm", "unit": "GB/s", "peak": peaks.get("hbm_gbs"),
                "select": {"bytes": sel_bytes, "achieved": sel_bytes / (sel_ms * 1e-3) / 1e9,
                           "frac": sel_bytes / (sel_ms * 1e-3) / 1e9 / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None},
                "refit": {"bytes": ref_bytes, "achieved": ref_bytes / (ref_ms * 1e-3) / 1e9,
                          "frac": ref_bytes / (ref_ms * 1e-3) / 1e9 / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None},
                "note": "algorithmic bytes of the elite controllers' selection and refit; both stages are "
                        "latency-bound chains of dependent loads, far from the HBM roof"},
            "e2e": {"value": e2e_value, "unit": "sample-steps/s",
                    "h2d_bytes_per_step": int(h2d_bytes), "d2h_bytes_per_step": int(h_out.size),
                    "call": "sbs_batch_solve_host (inputs in the batch's pinned staging, written in place "
                            "by sbs_batch_host_inputs' views; one copy each way per tick, synchronous)"},
            # rollout, selection and refit; a split tick (grid mode, MPPI and elite or
            # Naive controllers together) launches the rollout twice
            "gpu_launches": (4 if mode == "grid" and 0 < mppi_n < len(mix) else 3) * args.steps,
            "clocks": clk,
            "status_counts": {"ok": sum(s == S.OK for s in status),
                              "diverged": sum(s == S.ERR_DIVERGED for s in status)},
            "hbm_gbs_measured": peaks.get("hbm_gbs"),
        }
        if served:
            line["served"] = served
        if cpu:
            line["cpu_baseline"] = cpu
        if parity:
            line["parity"] = parity
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
