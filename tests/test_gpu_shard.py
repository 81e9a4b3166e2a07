"""Sample sharding of one controller (sbs_shard_rollout / sbs_shard_update):
the sharded solve gives the unsharded solve's bits on every rank.

In one process: `world` handles of the same controller act as the ranks, and the
exchange is a sum of their buffers on the GPU (int32 words, as the collective
computes it).  Each rank's buffer writes only words no other rank writes, which
is what makes the sum exact.  Then a real world-size-2 gloo group of two
processes on the one GPU (the kernels of the two ranks never wait on each
other: the exchange runs on the host between an iteration's launches)."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from shard_cases import CASES, problem_tensors, ticks  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    S.lib()
    return torch


def _controller(cfg):
    c = S.Controller(cfg, cfg.get("tile", 0))
    if cfg.get("spt"):
        c.set_samples_per_thread(cfg["spt"])
    return c


def _bufs(cfg):
    b = [S.BUF_MEAN, S.BUF_VAR, S.BUF_COST, S.BUF_FREQ]
    if cfg["method"] != "mppi":
        b.append(S.BUF_ELITE)
    if cfg.get("compare_mppi"):
        b.append(S.BUF_MPPI_MEAN)
    return b


@pytest.mark.parametrize("world", [1, 2, 3, 7])
@pytest.mark.parametrize("name", list(CASES))
def test_sharded_equals_unsharded(name, world):
    import torch
    cfg = CASES[name]()
    prob = W.problem(cfg)
    x0, xr, fe, feet = problem_tensors(prob)
    ref = _controller(cfg)
    ranks = [_controller(cfg) for _ in range(world)]
    nbytes = ranks[0].shard_exchange_bytes()
    assert nbytes % 4 == 0
    xb = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(world)]
    res = [torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device="cuda") for _ in range(world)]
    ntiles = ranks[0].shard_tiles()
    spans = [S.shard_range(ntiles, r, world) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == ntiles
    for tick, (g, shift) in enumerate(ticks(cfg, prob)):
        rr = ref.solve(x0, xr, g, fe, shift, feet=feet)
        probs = [c.problem(x0, xr, g, fe, shift, feet=feet) for c in ranks]
        for it in range(cfg.get("iterations", 1)):
            for r, c in enumerate(ranks):
                c.shard_rollout(probs[r], r, world, xb[r])
            words = torch.stack([b.view(torch.int32) for b in xb])
            # each word written by at most one rank
            assert int((words != 0).sum(0).max()) <= 1, f"{name}: ranks' buffers overlap"
            total = words.sum(0, dtype=torch.int32)
            for r, c in enumerate(ranks):
                xb[r].view(torch.int32).copy_(total)
                c.shard_update(xb[r], res[r])
        torch.cuda.synchronize()
        want = rr.cpu().numpy()
        for r, c in enumerate(ranks):
            np.testing.assert_array_equal(res[r].cpu().numpy(), want, err_msg=f"{name} tick {tick} rank {r}")
            for b in _bufs(cfg):
                np.testing.assert_array_equal(c.read(b).cpu().numpy(), ref.read(b).cpu().numpy(),
                                              err_msg=f"{name} tick {tick} rank {r} buffer {b}")
        assert S.parse_result(want)["status"] == S.OK
    for c in ranks + [ref]:
        c.close()


def test_shard_refusals():
    import torch
    cfg = CASES["naive_k777_t64"]()
    prob = W.problem(cfg)
    x0, xr, fe, _ = problem_tensors(prob)
    c = _controller(cfg)
    p = c.problem(x0, xr, prob["gait"], fe, 0)
    xb = torch.empty(c.shard_exchange_bytes(), dtype=torch.uint8, device="cuda")
    res = torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.SBSError):  # rank outside the world
        c.shard_rollout(p, 2, 2, xb)
    with pytest.raises(S.SBSError):  # an update with no rollout
        c.shard_update(xb, res)
    with pytest.raises(S.SBSError):  # misaligned exchange buffer
        c.shard_rollout(p, 0, 1, xb[4:])
    c.shard_rollout(p, 0, 1, xb)
    with pytest.raises(S.SBSError):  # a second rollout before the update
        c.shard_rollout(p, 0, 1, xb)
    with pytest.raises(S.SBSError):  # an unsharded solve meanwhile
        c.solve(x0, xr, prob["gait"], fe, 0)
    c.shard_update(xb, res)
    c.solve(x0, xr, prob["gait"], fe, 1)  # usable again
    torch.cuda.synchronize()
    c.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("name", ["mppi_k40000_groups", "elite_cmp_adaptive_it2", "naive_freqset"])
def test_two_process_gloo(name, tmp_path):
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "tests", "shard_worker.py"), "gpu",
                                       name, str(tmp_path / f"r{r}.npz")], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    outs = []
    for p in procs:
        try:
            out, _ = p.communicate(timeout=600)
        except subprocess.TimeoutExpired:
            p.kill()
            out, _ = p.communicate()
        outs.append(out)
    for r, p in enumerate(procs):
        assert p.returncode == 0, f"rank {r}:\n{outs[r][-3000:]}"
    a, b = np.load(tmp_path / "r0.npz"), np.load(tmp_path / "r1.npz")
    assert a["tiles"][1] == b["tiles"][0]
    for tick in range(3):
        for key in ("res", "mean", "cost"):
            np.testing.assert_array_equal(a[f"{key}{tick}"], a[f"ref_{key}{tick}"], err_msg=f"rank 0 {key} {tick}")
            np.testing.assert_array_equal(b[f"{key}{tick}"], a[f"ref_{key}{tick}"], err_msg=f"rank 1 {key} {tick}")
