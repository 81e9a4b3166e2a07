"""Benchmark of the SBS controller hot path on B300.

Workload: 256 independent controllers of uneven size solved together each
control tick (K in {256, 1024, 4096, 16384}, H in {10, 25, 50}, trot/pace/crawl,
MPPI or elite 5 %), one graph-replayed batched launch set per tick (grid or
persistent mode, picked by the autotuner), inputs resident in HBM, synthetic
seeded data.  A step is one tick: rollout,
cost, update of all 256 controllers (warm-started from the previous tick).

Metric: rollout sample-steps per second (sum of K*H over the controllers
solved, per second of tick time); also reported: solves/s, tick latency
p50/p99, the same tick as plain one-launch-set-per-controller solves, the
end-to-end number with host inputs/outputs, the dominant kernel's roofline and
the FP64 oracle's throughput on the host cores.

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

# Algorithmic FP32 work per sample-step of the per-step policy (counted from the
# kernel's formulation, FMA = 2): Box-Muller arithmetic 36, sampling 24, stage
# cost 128, SRBD Euler step 201; MPPI partial sums add 24.  Transcendentals
# (26 per sample-step) and the integer Philox rounds are not counted.
FLOPS_ROLLOUT = 36 + 24 + 128 + 201
FLOPS_MPPI_PARTIAL = 24


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="sbs", choices=["sbs", "reference"])
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--tile", type=int, default=0,
                    help="samples per block of the batched controllers; 0: timed at 128 and 256, fastest kept")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-serving", action="store_true", help="skip the closed-loop serving comparison")
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


def solve_launches(cfg):
    """Kernel launches of one plain solve: per iteration the rollout, and for elite
    and Naive the selection (five kernels for an elite set chosen from more than
    32 768 costs) and the refit."""
    if cfg["method"] == "mppi":
        return cfg["iterations"]
    select = 5 if cfg["method"] == "elite" and cfg["K"] > 32768 else 1
    return cfg["iterations"] * (2 + select)


def rollout_traffic():
    """DRAM bytes per sample-step of the rollout kernel from the committed ncu
    record, or None when the kernel sources changed since that capture."""
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
    return rec["dram_bytes_per_sample_step"] if h.hexdigest() == rec["sources_sha256"] else None


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


# ----------------------------------------------------------------------------- single controller

def flops_per_sample_step(cfg):
    """Algorithmic FP32 work per sample-step of one controller (FMA = 2).
    Per-step policy: see FLOPS_ROLLOUT.  Spline policy: per step the basis
    evaluation (2 P FLOP per force) replaces Box-Muller and sampling, and the
    knot noise (Box-Muller 6 FLOP per pair, 12 P normals; sampling 2 FLOP per
    knot value) is counted once per sample, i.e. divided by H."""
    P, H = cfg.get("P", 0), cfg["H"]
    base = 128 + 201  # stage cost + SRBD Euler step
    if P > 0:
        per = base + 12 * 2 * P + (6 * 6 * P + 2 * 12 * P) / H
        part = (2 * 12 * P) / H  # MPPI partials from the knot deviations
    else:
        per = FLOPS_ROLLOUT
        part = FLOPS_MPPI_PARTIAL
    mppi = cfg["method"] == "mppi" or cfg.get("compare_mppi")
    return per + (part if mppi else 0.0)


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
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        ctl.solve_packed(p1, res)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    ss = cfg["K"] * cfg["H"] * cfg["iterations"]
    fl = flops_per_sample_step(cfg) * ss
    # the solve is rollout + (select + refit) launches; the roofline uses the whole solve
    achieved = fl / (ms * 1e-3) / 1e12
    peak = S.fp32_peak() / 1e12
    # host inputs and result, synchronised per solve
    hx0, hxr, hfe = (np.ascontiguousarray(np.float32(prob[k])) for k in ("x0", "xref", "f_ext"))
    hfeet = np.ascontiguousarray(np.float32(prob["feet"])) if "feet" in prob else None
    r = S.Result()
    hp = ctl.problem(hx0, hxr, prob["gait"], hfe, 1, host=True, feet=hfeet)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctl.solve_packed(hp, r)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)
    if rank == 0:
        line = {"metric": "rollout sample-steps/s", "value": world * ss / (ms * 1e-3), "unit": "sample-steps/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": args.workload, "K": cfg["K"], "H": cfg["H"], "P": cfg.get("P", 0),
                           "iterations": cfg["iterations"], "method": cfg["method"], "tile": ctl.tile,
                           "parallelism": f"replicas x{world}"},
                "solves_per_s": world / (ms * 1e-3),
                "roofline": {"kernel": "whole solve", "bound": "alu", "achieved": achieved, "peak": peak,
                             "unit": "TFLOP/s", "frac": achieved / peak,
                             "peak_kind": "FP32 FMA-chain microbenchmark on this GPU (live)",
                             "flops_per_sample_step": flops_per_sample_step(cfg), "traffic": None},
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
    arena = sum(c.workspace_bytes() + 256 for c in ctls)
    batch = S.Batch(n, 2 * arena, inflight=2)  # two ticks in flight: the next is prepared while one runs
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
    mode = "grid" if batch.mode() == S.BATCH_GRID else "persistent"
    for _ in range(3):  # rebuild the tick graphs in the chosen mode before timing
        tick()
    torch.cuda.synchronize()

    # ---- timed region: K ticks back to back on the stream
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # profilers can select exactly the timed launches
    e0.record(stream)
    for _ in range(args.steps):
        tick()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world, dev)
    value = world * ss_tick / (ms * 1e-3)

    # ---- tick latency distribution (device time of each tick)
    lat = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ev:
        a.record(stream)
        tick()
        b.record(stream)
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(b) for a, b in ev)
    p50, p99 = lat[len(lat) // 2], lat[min(len(lat) - 1, int(0.99 * len(lat)))]

    # ---- stage durations with per-stage events (dominant kernel for the roofline)
    batch.set_profiling(True)
    st = []
    for _ in range(args.steps):
        tick()
        st.append(batch.stage_ms())
    batch.set_profiling(False)
    st = np.array(st)
    roll_ms = float(st[:, 0].mean())
    sel_ms, ref_ms = float(st[:, 1].mean()), float(st[:, 2].mean())
    flops_launch = ss_tick * FLOPS_ROLLOUT + mppi_ss * FLOPS_MPPI_PARTIAL
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
        ref_bytes += (48 + 4) * ke * c["H"] + 16 * d
    fp32_peak = S.fp32_peak() / 1e12
    nominal = 148 * 128 * 2 * 2032e6 / 1e12

    # ---- plain form: one sbs_solve (its own launches) per controller, serialised
    plain_ticks = max(3, min(args.steps, 40))
    pres = [torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device=dev) for _ in range(n)]
    for i in range(n):
        ctls[i].solve(x0[i], xref[i], gaits[i], fext[i], 1, pres[i])
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(plain_ticks):
        for i in range(n):
            ctls[i].solve(x0[i], xref[i], gaits[i], fext[i], 1, pres[i])
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / plain_ticks

    # ---- end to end: inputs from pinned host memory, results back to the host
    h_in = torch.empty(sum(12 + x.numel() + 3 for x in xref), dtype=torch.float32).pin_memory()
    off = 0
    views = []
    for i in range(n):
        nn_ = 12 + xref[i].numel() + 3
        h_in[off:off + 12] = x0[i].cpu()
        h_in[off + 12:off + 12 + xref[i].numel()] = xref[i].cpu().ravel()
        h_in[off + 12 + xref[i].numel():off + nn_] = fext[i].cpu()
        views.append((off, nn_))
        off += nn_
    d_in = torch.empty_like(h_in, device=dev)
    eprobs = []
    for i, (o, nn_) in enumerate(views):
        xi = d_in[o:o + 12]
        ri = d_in[o + 12:o + 12 + xref[i].numel()]
        fi = d_in[o + 12 + xref[i].numel():o + nn_]
        eprobs.append(ctls[i].problem(xi, ri, gaits[i], fi, 1))
    epacked = S.Packed(ctls, eprobs)
    h_out = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8).pin_memory()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        d_in.copy_(h_in, non_blocking=True)
        batch.solve_packed(epacked, results)
        h_out.copy_(results, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e_value = world * ss_tick / e2e_s
    status = [S.parse_result(h_out[i * S.RESULT_BYTES:(i + 1) * S.RESULT_BYTES].numpy())["status"] for i in range(n)]

    # ---- served: 2048 closed-loop robots, continuous batching vs plain solves
    served = None
    if not args.no_serving:
        from paper_2403_11383_b300 import serving
        robots = serving.Robots(2048, seed=3)
        served = {"batched": serving.run(plain=False, duration=args.serving_seconds, warmup=1.0, robots=robots),
                  "plain": serving.run(plain=True, duration=args.serving_seconds, warmup=1.0, robots=robots)}
        del robots

    # ---- CPU baseline: the FP64 oracle on a bounded sample (rank 0)
    cpu = None
    if rank == 0 and not args.no_cpu:
        nthreads = os.cpu_count() or 1
        rate, ninst, ss, t_ = oracle_rate(W.batch_config(args.instances), 15.0, nthreads)
        cpu = {"value": rate, "unit": "sample-steps/s", "cores": nthreads, "kind": "oracle",
               "sample": f"first {ninst} controllers of the mix, one FP64 solve each ({ss} sample-steps, "
                         f"{t_:.1f} s)"}

    peaks = measured_peaks()
    traffic_ss = rollout_traffic()
    if rank == 0:
        line = {
            "metric": "rollout sample-steps/s", "value": value, "unit": "sample-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances": n, "sample_steps_per_tick": ss_tick,
                       "tile": tile, "tile_autotune_ms_per_tick": tile_ms, "graph": True, "launch_mode": mode,
                       "autotune_ms_per_tick": {"grid": tune_ms[0], "persistent": tune_ms[1]},
                       "l2": "per-tick working set above L2 (sampled deviations "
                       f"{arena / 1e9:.2f} GB)", "workspace_bytes": 2 * arena, "parallelism": f"replicas x{world}"},
            "solves_per_s": world * n / (ms * 1e-3),
            "latency_ms": {"p50": p50, "p99": p99, "kind": f"device time of one {len(mix)}-controller tick"},
            "plain": {"ms_per_tick": plain_ms, "sample_steps_per_s": ss_tick / (plain_ms * 1e-3),
                      "solves_per_s": n / (plain_ms * 1e-3), "kind": "256 serialised sbs_solve calls"},
            "stages_ms": {"rollout": roll_ms, "select": sel_ms, "refit": ref_ms},
            "roofline": {"kernel": "k_grid_rollout_lean" if mode == "grid" else "k_batch_rollout<0, false>", "bound": "alu", "achieved": achieved,
                         "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "peak_kind": "FP32 FMA-chain microbenchmark on this GPU (live)",
                         "nominal_peak": nominal, "frac_of_nominal": achieved / nominal,
                         "flops_per_launch": flops_launch,
                         "traffic": None if traffic_ss is None else traffic_ss * ss_tick,
                         "traffic_note": "ncu DRAM read+write of the two rollout launches of this workload's tick "
                                         "(one-pass capture, profiles/rollout_traffic.json), per sample-step "
                                         "times this tick's sample-steps"},
            "update_roofline": {
                "bound": "hbm", "unit": "GB/s", "peak": peaks.get("hbm_gbs"),
                "select": {"bytes": sel_bytes, "achieved": sel_bytes / (sel_ms * 1e-3) / 1e9,
                           "frac": sel_bytes / (sel_ms * 1e-3) / 1e9 / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None},
                "refit": {"bytes": ref_bytes, "achieved": ref_bytes / (ref_ms * 1e-3) / 1e9,
                          "frac": ref_bytes / (ref_ms * 1e-3) / 1e9 / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None},
                "note": "algorithmic bytes of the elite controllers' selection and refit; both stages are "
                        "latency-bound chains of dependent loads, far from the HBM roof"},
            "e2e": {"value": e2e_value, "unit": "sample-steps/s",
                    "h2d_bytes_per_step": int(h_in.numel() * 4), "d2h_bytes_per_step": int(h_out.numel())},
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
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
