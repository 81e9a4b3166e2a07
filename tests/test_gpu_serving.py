"""The request loop: results served with continuous batching equal each
controller's own plain solve; requests arriving while ticks run are admitted
into free slots; admission by budget; order per controller; a short closed-loop
serving run."""
import numpy as np
import pytest

from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import serving
from paper_2403_11383_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup(n=6, seed=5):
    mix, _ = W.serving_mix(n, seed)
    cfgs = [dict(c, K=[512, 1000, 300][i % 3], H=[12, 25, 10][i % 3]) for i, (c, _) in enumerate(mix)]
    probs = [W.problem(c) for c in cfgs]
    return cfgs, probs


def _records(ctls, probs, shift, bufs):
    recs = np.zeros(len(ctls), dtype=S.PROBLEM_DTYPE)
    for i, (c, p) in enumerate(zip(ctls, probs)):
        x0 = np.ascontiguousarray(p["x0"], dtype=np.float32)
        xr = np.ascontiguousarray(p["xref"], dtype=np.float32)
        bufs.extend([x0, xr])
        recs[i]["x0"], recs[i]["xref"], recs[i]["f_ext"] = x0.ctypes.data, xr.ctypes.data, 0
        recs[i]["offset"] = p["gait"]["offset"]
        recs[i]["duty"], recs[i]["phase0"] = p["gait"]["duty"], p["gait"]["phase0"]
        recs[i]["shift"], recs[i]["host_memory"] = shift, 1
    return recs


def _wait(server, tickets, timeout=30.0):
    import time
    t0 = time.time()
    out = np.zeros(len(tickets), dtype=S.RESULT_DTYPE)
    left = np.ones(len(tickets), bool)
    while left.any():
        st, res = server.poll(tickets[left])
        idx = np.nonzero(left)[0]
        ok = st == S.OK
        out[idx[ok]] = res[ok]
        left[idx[ok]] = False
        assert not (st == S.ERR_INVALID_ARG).any()
        assert time.time() - t0 < timeout
    return out


@pytest.mark.parametrize("spt,theta", [(0, S.THETA_STORE), (2, S.THETA_REGENERATE)])
def test_served_results_equal_plain_solves(spt, theta):
    # in the library's default launch settings and in those the serving run uses
    # (two samples per thread, regenerated deviations): the same bits
    import torch
    cfgs, probs = _setup()
    served = [S.Controller(c) for c in cfgs]
    plain = [S.Controller(c) for c in cfgs]
    srv = S.Server(slots=2, max_batch=16, budget_bytes=1 << 30, samples_per_thread=spt, theta_mode=theta)
    handles = np.array([c.handle.value for c in served], dtype=np.uint64)
    for rnd in range(3):
        bufs = []
        recs = _records(served, probs, 0 if rnd == 0 else 1, bufs)
        t = srv.submit(handles, recs)
        res = _wait(srv, t)
        for i, c in enumerate(plain):
            r = c.solve_host(np.float32(probs[i]["x0"]), np.float32(probs[i]["xref"]), probs[i]["gait"], None,
                             0 if rnd == 0 else 1)
            torch.cuda.synchronize()
            want = np.frombuffer(bytes(r), dtype=S.RESULT_DTYPE)[0]
            assert res[i].tobytes() == want.tobytes()
    for a, b in zip(served, plain):
        np.testing.assert_array_equal(a.read(S.BUF_MEAN).cpu().numpy(), b.read(S.BUF_MEAN).cpu().numpy())
    srv.close()


def test_served_extended_features_equal_plain_solves():
    # ground-fixed feet, the frequency set, the friction projection and the terminal
    # cost go through the server's staging (feet included) and the extended kernels
    import torch
    base = W.config("worldfeet_mppi_k4096_h25")
    cfgs = [dict(base, K=700, seed=61, ctrl=0),
            dict(base, K=900, H=12, seed=61, ctrl=1, friction_project=True,
                 cost=dict(base["cost"], w_terminal=3.0)),
            dict(W.config("naive_freqset_k10000_h12"), K=1200, world_feet=True, seed=61, ctrl=2)]
    probs = [W.problem(c) for c in cfgs]
    served = [S.Controller(c) for c in cfgs]
    plain = [S.Controller(c) for c in cfgs]
    srv = S.Server(slots=2, max_batch=8, budget_bytes=1 << 30)
    handles = np.array([c.handle.value for c in served], dtype=np.uint64)
    for rnd in range(2):
        bufs = []
        recs = _records(served, probs, 0 if rnd == 0 else 1, bufs)
        for i, p in enumerate(probs):
            f = np.ascontiguousarray(p["feet"], dtype=np.float32)
            bufs.append(f)
            recs[i]["feet"] = f.ctypes.data
        res = _wait(srv, srv.submit(handles, recs))
        for i, c in enumerate(plain):
            r = c.solve_host(np.float32(probs[i]["x0"]), np.float32(probs[i]["xref"]), probs[i]["gait"], None,
                             0 if rnd == 0 else 1, feet=np.float32(probs[i]["feet"]))
            torch.cuda.synchronize()
            want = np.frombuffer(bytes(r), dtype=S.RESULT_DTYPE)[0]
            assert res[i].tobytes() == want.tobytes()
    srv.close()


def test_requests_of_one_controller_are_served_in_order():
    cfgs, probs = _setup(2)
    c = S.Controller(cfgs[0])
    srv = S.Server(slots=3, max_batch=8, budget_bytes=1 << 30)
    bufs = []
    recs = np.concatenate([_records([c], [probs[0]], s, bufs) for s in (0, 1, 1)])
    t = srv.submit(np.array([c.handle.value] * 3, dtype=np.uint64), recs)
    res = _wait(srv, t)
    its = res["iter_lo"]
    assert its.tolist() == [0, 1, 2]
    st = srv.stats()
    assert st["ticks"] == 3 and st["completed"] == 3
    srv.close()


def test_admission_by_budget_and_full_queue():
    cfgs, probs = _setup(4)
    ctls = [S.Controller(c) for c in cfgs]
    need = max(c.workspace_bytes() for c in ctls)
    # room for one controller per tick: ticks of one
    srv = S.Server(slots=2, max_batch=8, budget_bytes=2 * (need + 4096))
    bufs = []
    t = srv.submit(np.array([c.handle.value for c in ctls], dtype=np.uint64), _records(ctls, probs, 0, bufs))
    res = _wait(srv, t)
    assert (res["status"] == S.OK).all()
    st = srv.stats()
    assert st["ticks"] >= 2 and st["admission_waits"] >= 1
    srv.close()
    tiny = S.Server(slots=1, max_batch=8, budget_bytes=8192)
    with pytest.raises(S.SBSError) as e:
        tiny.submit(np.array([ctls[0].handle.value], dtype=np.uint64), _records(ctls[:1], probs[:1], 0, bufs))
    assert e.value.status == S.ERR_BUDGET
    tiny.close()
    # a server that regenerates the deviations admits by the smaller workspace: the
    # same budget holds every request in one tick
    need_r = sum(c.workspace_bytes_mode(S.THETA_REGENERATE) + 256 for c in ctls)
    assert need_r < need
    srv = S.Server(slots=1, max_batch=8, budget_bytes=need_r + 4096, theta_mode=S.THETA_REGENERATE)
    t = srv.submit(np.array([c.handle.value for c in ctls], dtype=np.uint64), _records(ctls, probs, 1, bufs))
    res = _wait(srv, t)
    assert (res["status"] == S.OK).all() and srv.stats()["ticks"] == 1
    srv.close()
    small = S.Server(slots=1, max_batch=8, max_pending=2, budget_bytes=1 << 30)
    with pytest.raises(S.SBSError) as e:
        small.submit(np.array([c.handle.value for c in ctls[:3]], dtype=np.uint64), _records(ctls[:3], probs[:3], 0, bufs))
    assert e.value.status == S.PENDING
    small.close()


def test_continuous_batching_admits_while_ticks_run():
    # the first tick is long (4 spline controllers of 2^21 samples over 128 steps,
    # ~20 ms on the GPU), so the second batch arrives while it runs
    cfgs, _ = _setup(8)
    cfgs = [dict(c, K=1 << 21, H=128, P=4) if i < 4 else dict(c, K=4096, H=12) for i, c in enumerate(cfgs)]
    probs = [W.problem(c) for c in cfgs]
    ctls = [S.Controller(c) for c in cfgs]
    srv = S.Server(slots=2, max_batch=64, budget_bytes=8 << 30)
    bufs = []
    h = np.array([c.handle.value for c in ctls], dtype=np.uint64)
    import time
    rec1 = _records(ctls[:4], probs[:4], 0, bufs)
    rec2 = _records(ctls[4:], probs[4:], 0, bufs)
    t1 = srv.submit(h[:4], rec1)
    t0 = time.time()
    while srv.stats()["ticks"] < 1:  # the first tick is on the GPU ...
        assert time.time() - t0 < 10
    t2 = srv.submit(h[4:], rec2)  # ... when these arrive
    r = _wait(srv, np.concatenate([t1, t2]))
    assert (r["iter_lo"] == 0).all()
    st = srv.stats()
    assert st["completed"] == 8 and st["ticks"] >= 2
    assert st["max_inflight"] >= 2  # the second tick was issued while the first still ran
    srv.close()


def test_short_closed_loop_serving_run():
    R = serving.Robots(64, seed=9)
    out = serving.run(plain=False, duration=1.0, warmup=0.3, robots=R)
    assert out["solves_per_s"] > 100
    assert out["latency_ms"]["p50"] > 0 and out["latency_ms"]["p99"] >= out["latency_ms"]["p50"]
    assert out["mean_batch"] >= 1
