"""bench.py run as a user runs it: every named workload and a small batched tick
print one JSON line that keeps the benchmark contract (keys, units, the kernel
launch count the library makes, host bytes of the end-to-end leg)."""
import json
import os
import subprocess
import sys

import pytest

from paper_2403_11383_b300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
STEPS, WARMUP = 5, 3


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", str(STEPS), "--warmup",
                          str(WARMUP), "--no-cpu", *args], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def _common(d):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["metric"] == "rollout sample-steps/s" and d["unit"] == "sample-steps/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == STEPS and d["n_gpus"] == 1
    r = d["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and 0 < r["frac"] < 1.5
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert d["e2e"]["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0


@pytest.mark.parametrize("name", W.SINGLE)
def test_single_workload_line(name):
    d = _run("--workload", name)
    _common(d)
    cfg = W.config(name)
    assert d["config"]["workload"] == name and d["config"]["K"] == cfg["K"] and d["config"]["H"] == cfg["H"]
    # per solve: the rollout, plus the selection (five kernels above 32 768 costs) and refit
    per = 1 if cfg["method"] == "mppi" else 2 + (5 if cfg["method"] == "elite" and cfg["K"] > 32768 else 1)
    assert d["gpu_launches"] == STEPS * cfg["iterations"] * per
    feet = 8 if cfg.get("world_feet") else 0
    assert d["e2e"]["h2d_bytes_per_step"] == 4 * (12 + 3 + 12 * cfg["H"] + feet)


def test_single_workload_fixed_setting():
    # a profiling capture fixes the launch setting instead of timing the others
    d = _run("--workload", "plain_mppi_k512_h12", "--spt", "3", "--theta", "regenerate")
    _common(d)
    c = d["config"]
    assert c["samples_per_thread"] == 3 and c["sampled_deviations"] == "regenerate"
    assert c["fixed_by_flags"] == {"spt": 3, "theta": "regenerate"} and c["autotune_ms_per_solve"] is None


def test_small_batched_line():
    d = _run("--instances", "8", "--tile", "256", "--no-serving")
    _common(d)
    assert d["config"]["instances"] == 8 and d["config"]["tile"] == 256
    mix = W.batch_mix(8)
    mppi = sum(1 for c, _ in mix if c["method"] == "mppi")
    split = d["config"]["launch_mode"] == "grid" and 0 < mppi < len(mix)
    assert d["gpu_launches"] == (4 if split else 3) * STEPS
    assert set(d["stages_ms"]) == {"rollout", "select", "refit"}
    # the end-to-end leg copies x0, the reference and f_ext of every controller in
    # and one result record per controller out
    assert d["e2e"]["h2d_bytes_per_step"] == sum(4 * (12 + 12 * c["H"] + 3) for c, _ in mix)
    assert d["e2e"]["d2h_bytes_per_step"] == 8 * 80
    assert d["latency_ms"]["ticks"] >= 400


@pytest.mark.parametrize("name", ["plain_mppi_k512_h12", "adaptive_elite_k8192_h25"])
def test_parity_record_within_tolerances(name):
    # the bench's per-output error record on two workloads: the staged update
    # errors meet the parity tests' tolerances
    import bench
    cfg = W.config(name)
    rec = bench.parity_one(cfg, W.problem(cfg), os.cpu_count() or 1)
    assert rec["gated"] > 0 and rec["cost_rel_err_gated"]["max"] <= 1e-3
    assert rec["staged"]["mean_abs_err"] <= bench.MEAN_ATOL
    if cfg["method"] == "mppi":
        assert rec["staged"]["ess_rel_err"] <= 1e-4
    else:
        assert rec["staged"]["elite_set_is_first_Ke_of_gpu_costs"]
        assert rec["staged"]["var_rel_err"] <= 2e-4
        assert rec["staged"]["compare_mppi_mean_abs_err"] <= bench.MEAN_ATOL
