"""Failures injected on the host, without a GPU: a refusing device allocator,
invalid requests, and the multi-process launch path of bench.py (gloo,
world size 2)."""
import ctypes as C
import json
import os
import socket
import subprocess
import sys

import pytest

from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class Refusing:
    """An allocator that refuses every request and counts them."""

    def __init__(self):
        self.calls = 0
        self._a = S.ALLOC_FN(self._alloc)
        self._f = S.FREE_FN(self._free)
        self.struct = S.Allocator(self._a, self._f, None)

    def _alloc(self, n, ctx):
        self.calls += 1
        return None

    def _free(self, p, ctx):
        raise AssertionError("nothing was allocated")


def test_refusing_allocator_gives_oom_and_no_handle():
    S.lib()
    ref = Refusing()
    c = S.make_config(W.config("plain_mppi_k512_h12"))
    h = C.c_void_p()
    st = S.lib().sbs_create(C.byref(c), C.byref(ref.struct), C.byref(h))
    assert st == S.ERR_OOM and not h.value and ref.calls == 1
    b = C.c_void_p()
    st = S.lib().sbs_batch_create(4, 1, 1 << 20, C.byref(ref.struct), C.byref(b))
    assert st in (S.ERR_OOM, S.ERR_CUDA) and not b.value


def test_allocator_without_functions_is_rejected():
    S.lib()
    c = S.make_config(W.config("plain_mppi_k512_h12"))
    bad = S.Allocator()
    h = C.c_void_p()
    assert S.lib().sbs_create(C.byref(c), C.byref(bad), C.byref(h)) == S.ERR_INVALID_ARG


def test_server_and_batch_argument_checks():
    L = S.lib()
    cfg = S.ServerConfig(0, 1, 1, 0, 1 << 20)
    s = C.c_void_p()
    assert L.sbs_server_create(C.byref(cfg), None, C.byref(s)) == S.ERR_INVALID_ARG
    cfg = S.ServerConfig(2, 0, 1, 0, 1 << 20)
    assert L.sbs_server_create(C.byref(cfg), None, C.byref(s)) == S.ERR_INVALID_ARG
    b = C.c_void_p()
    assert L.sbs_batch_create(4, 0, 1 << 20, None, C.byref(b)) == S.ERR_INVALID_ARG
    assert L.sbs_batch_create(4, 9, 1 << 20, None, C.byref(b)) == S.ERR_INVALID_ARG
    assert L.sbs_batch_set_mode(None, 0) == S.ERR_INVALID_ARG
    assert L.sbs_server_submit(None, 1, None, None, None) == S.ERR_INVALID_ARG
    assert L.sbs_server_poll(None, 1, None, None, None) == S.ERR_INVALID_ARG
    assert L.sbs_solve_mppi_static(None, None, None, None, 0, None, None) == S.ERR_INVALID_ARG


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_bench_reference_arm_two_ranks_gloo():
    # two ranks on the CPU: rank 0 alone runs and prints one JSON line, rank 1 exits 0
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--instances", "8"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["n_gpus"] == 2
    assert rec["cpu_baseline"]["kind"] == "oracle"


def test_bench_rank_helpers_gloo(tmp_path):
    # the max-over-ranks reduction bench.py uses for its timing, on two gloo ranks
    code = r'''
import os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
r = int(os.environ["RANK"])
bench.barrier(2)
v = bench.max_over_ranks(1.0 + r, 2, None)
assert v == 2.0, v
print("ok", r)
dist.destroy_process_group()
'''
    path = tmp_path / "rank_probe.py"
    path.write_text(code)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), str(path), ROOT]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.count("ok") == 2
