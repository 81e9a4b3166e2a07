"""Batched ticks: every controller's result in a mix of uneven controllers
equals its own plain sbs_solve (same tile size), in both launch modes, over
warm-started ticks; budget admission and the launch-mode autotuner."""
import numpy as np
import pytest

from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _mix():
    base = W.config("plain_mppi_k512_h12")
    specs = [
        dict(K=1000, H=7, gait="trot", method="mppi"),
        dict(K=4096, H=25, gait="pace", method="elite", elite_count=205),
        dict(K=300, H=12, gait="crawl", method="naive"),
        dict(K=2048, H=10, gait="trot", method="mppi", adaptive=True),
        dict(K=777, H=50, gait="pace", method="elite", elite_count=39, adaptive=True),
        dict(K=16384, H=12, gait="trot", method="mppi"),
        dict(K=129, H=3, gait="crawl", method="elite", elite_count=7),
        dict(K=5000, H=33, gait="trot", method="mppi", adaptive=True, compare_mppi=True),
        dict(K=2500, H=12, gait="trot", method="naive", freq_set_mhz=(1300, 2000, 2400)),
        dict(K=1500, H=25, gait="pace", method="mppi", world_feet=True),
        dict(K=1024, H=12, gait="trot", method="elite", elite_count=52, friction_project=True),
    ]
    out = []
    for i, sp in enumerate(specs):
        c = dict(base)
        c.update(sp)
        c.update(seed=100 + i, ctrl=i)
        out.append((c, W.problem(c)))
    return out


def _tensors(prob):
    import torch
    d = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
    return d(prob["x0"]), d(prob["xref"]), d(prob["f_ext"]), (d(prob["feet"]) if "feet" in prob else None)


def _gait(prob, tick, cfg):
    g = dict(prob["gait"])
    g["phase0"] = (g["phase0"] + tick * cfg["q_init"] * cfg["dt_us"]) % W.PHASE_ONE
    return g


def _state(ctl):
    return ctl.read(S.BUF_MEAN).cpu().numpy(), ctl.read(S.BUF_VAR).cpu().numpy()


@pytest.mark.parametrize("mode", [S.BATCH_GRID, S.BATCH_PERSISTENT])
def test_batch_equals_plain(mode):
    import torch
    mix = _mix()
    plain = [S.Controller(c) for c, _ in mix]
    batched = [S.Controller(c) for c, _ in mix]
    tens = [_tensors(p) for _, p in mix]
    n = len(mix)
    b = S.Batch(n, sum(c.workspace_bytes() + 256 for c in batched))
    b.set_mode(mode)
    assert b.mode() == mode
    res = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for tick in range(3):
        shift = 0 if tick == 0 else 1
        probs = []
        plain_res = []
        for i, (c, p) in enumerate(mix):
            x0, xr, fe, ft = tens[i]
            g = _gait(p, tick, c)
            plain_res.append(plain[i].solve(x0, xr, g, fe, shift, feet=ft).clone())
            probs.append(batched[i].problem(x0, xr, g, fe, shift, feet=ft))
        b.solve(batched, probs, res)
        torch.cuda.synchronize()
        for i in range(n):
            rp = S.parse_result(plain_res[i].cpu().numpy())
            rb = S.parse_result(res[i * S.RESULT_BYTES:(i + 1) * S.RESULT_BYTES].cpu().numpy())
            assert rb["status"] == rp["status"]
            np.testing.assert_array_equal(rb["u0"], rp["u0"])
            assert rb["cost_min"] == rp["cost_min"] and rb["ess"] == rp["ess"]
            assert rb["q_freq"] == rp["q_freq"] and rb["n_finite"] == rp["n_finite"] and rb["iter"] == rp["iter"]
            mp, vp = _state(plain[i])
            mb, vb = _state(batched[i])
            np.testing.assert_array_equal(mb, mp)
            np.testing.assert_array_equal(vb, vp)
            if mix[i][0].get("compare_mppi"):
                np.testing.assert_array_equal(batched[i].read(S.BUF_MPPI_MEAN).cpu().numpy(),
                                              plain[i].read(S.BUF_MPPI_MEAN).cpu().numpy())
    b.close()


@pytest.mark.parametrize("inflight", [1, 2])
def test_changing_controller_sets(inflight):
    # ticks over changing subsets of the mix, as a request loop makes them: the
    # tick's graph splits its rollout when elite or Naive and MPPI controllers meet,
    # and keeps one launch otherwise, so consecutive ticks of a slot rebuild or
    # update it; every result and state equals the controller's own plain solve
    import torch
    mix = _mix()
    n = len(mix)
    plain = [S.Controller(c) for c, _ in mix]
    batched = [S.Controller(c) for c, _ in mix]
    tens = [_tensors(p) for _, p in mix]
    mppi = [i for i, (c, _) in enumerate(mix) if c["method"] == "mppi"]
    upd = [i for i, (c, _) in enumerate(mix) if c["method"] != "mppi"]
    subsets = [list(range(n)), mppi, upd, list(range(n)), list(range(6)), upd[:2] + mppi[:1], list(range(n))]
    b = S.Batch(n, inflight * sum(c.workspace_bytes() + 256 for c in batched), inflight=inflight)
    b.set_mode(S.BATCH_GRID)
    res = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ticks = [0] * n
    for sub in subsets:
        probs, plain_res = [], []
        for i in sub:
            c, p = mix[i]
            x0, xr, fe, ft = tens[i]
            shift = 0 if ticks[i] == 0 else 1
            g = _gait(p, ticks[i], c)
            plain_res.append(plain[i].solve(x0, xr, g, fe, shift, feet=ft).clone())
            probs.append(batched[i].problem(x0, xr, g, fe, shift, feet=ft))
            ticks[i] += 1
        out = res[:len(sub) * S.RESULT_BYTES]
        b.solve([batched[i] for i in sub], probs, out)
        torch.cuda.synchronize()
        for r, i in enumerate(sub):
            rp = S.parse_result(plain_res[r].cpu().numpy())
            rb = S.parse_result(out[r * S.RESULT_BYTES:(r + 1) * S.RESULT_BYTES].cpu().numpy())
            assert rb["status"] == rp["status"], (sub, i)
            np.testing.assert_array_equal(rb["u0"], rp["u0"])
            assert rb["cost_min"] == rp["cost_min"] and rb["q_freq"] == rp["q_freq"] and rb["iter"] == rp["iter"]
            mp, vp = _state(plain[i])
            mb, vb = _state(batched[i])
            np.testing.assert_array_equal(mb, mp)
            np.testing.assert_array_equal(vb, vp)
    b.close()


@pytest.mark.parametrize("mode", [S.BATCH_GRID, S.BATCH_PERSISTENT])
@pytest.mark.parametrize("P", [3, 8])
def test_spline_batch_equals_plain(P, mode):
    # a batch of spline controllers (one knot count per batch): uneven K and H, MPPI,
    # elite and Naive, so the tick splits its rollout; two warm-started ticks
    import torch
    base = W.config("spline_k262144_h100")
    specs = [dict(K=3000, H=25, method="mppi", compare_mppi=False), dict(K=1500, H=12, method="elite"),
             dict(K=700, H=40, method="naive", compare_mppi=False), dict(K=4097, H=20, method="mppi"),
             dict(K=257, H=8, method="elite", adaptive=False)]
    mix = []
    for i, sp in enumerate(specs):
        c = dict(base)
        c.update(P=P, dt_us=20000, sigma_init=5.0, tile=128, seed=200 + i, ctrl=i, **sp)
        if c["method"] == "elite":
            c["elite_count"] = W.elite_count(0.03, c["K"])
        mix.append((c, W.problem(c)))
    n = len(mix)
    plain = [S.Controller(c) for c, _ in mix]
    batched = [S.Controller(c) for c, _ in mix]
    tens = [_tensors(p) for _, p in mix]
    b = S.Batch(n, sum(c.workspace_bytes() + 256 for c in batched))
    b.set_mode(mode)
    res = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for tick in range(2):
        probs, plain_res = [], []
        for i, (c, p) in enumerate(mix):
            x0, xr, fe, ft = tens[i]
            g = _gait(p, tick, c)
            plain_res.append(plain[i].solve(x0, xr, g, fe, min(tick, 1)).clone())
            probs.append(batched[i].problem(x0, xr, g, fe, min(tick, 1)))
        b.solve(batched, probs, res)
        torch.cuda.synchronize()
        for i in range(n):
            rp = S.parse_result(plain_res[i].cpu().numpy())
            rb = S.parse_result(res[i * S.RESULT_BYTES:(i + 1) * S.RESULT_BYTES].cpu().numpy())
            assert rb["status"] == rp["status"], i
            np.testing.assert_array_equal(rb["u0"], rp["u0"])
            assert rb["cost_min"] == rp["cost_min"] and rb["q_freq"] == rp["q_freq"]
            mp, vp = _state(plain[i])
            mb, vb = _state(batched[i])
            np.testing.assert_array_equal(mb, mp)
            np.testing.assert_array_equal(vb, vp)
    b.close()


def test_same_alone_and_in_the_mix():
    # one controller solved in a batch of one and inside a batch of eight
    import torch
    mix = _mix()
    k = 4
    alone = S.Controller(mix[k][0])
    inmix = [S.Controller(c) for c, _ in mix]
    tens = [_tensors(p) for _, p in mix]
    b1 = S.Batch(1, alone.workspace_bytes() + 256)
    b8 = S.Batch(len(mix), sum(c.workspace_bytes() + 256 for c in inmix))
    r1 = torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    r8 = torch.empty(len(mix) * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for tick in range(2):
        x0, xr, fe, ft = tens[k]
        g = _gait(mix[k][1], tick, mix[k][0])
        b1.solve([alone], [alone.problem(x0, xr, g, fe, min(tick, 1), feet=ft)], r1)
        probs = [inmix[i].problem(*tens[i][:2], _gait(mix[i][1], tick, mix[i][0]), tens[i][2], min(tick, 1),
                                  feet=tens[i][3])
                 for i in range(len(mix))]
        b8.solve(inmix, probs, r8)
    torch.cuda.synchronize()
    a, m = _state(alone), _state(inmix[k])
    np.testing.assert_array_equal(a[0], m[0])
    np.testing.assert_array_equal(a[1], m[1])
    assert bytes(r1.cpu().numpy()) == bytes(r8[k * S.RESULT_BYTES:(k + 1) * S.RESULT_BYTES].cpu().numpy())


def test_packed_closed_loop_equals_solve():
    # one Packed object edited in place (gait phase, shift) tick after tick gives
    # the same bits as packing fresh problems on every call
    import torch
    mix = _mix()
    a = [S.Controller(c) for c, _ in mix]
    p = [S.Controller(c) for c, _ in mix]
    tens = [_tensors(pr) for _, pr in mix]
    n = len(mix)
    ba = S.Batch(n, sum(c.workspace_bytes() + 256 for c in a))
    bp = S.Batch(n, 2 * sum(c.workspace_bytes() + 256 for c in p), inflight=2)  # split between two ticks
    ra = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    rp = torch.empty_like(ra)
    packed = S.Packed(p, [p[i].problem(*tens[i][:2], mix[i][1]["gait"], tens[i][2], 0, feet=tens[i][3])
                          for i in range(n)])
    for tick in range(3):
        probs = [a[i].problem(*tens[i][:2], _gait(mix[i][1], tick, mix[i][0]), tens[i][2], min(tick, 1),
                              feet=tens[i][3]) for i in range(n)]
        ba.solve(a, probs, ra)
        for i in range(n):
            packed.problems[i].gait.phase0 = _gait(mix[i][1], tick, mix[i][0])["phase0"]
            packed.problems[i].shift = min(tick, 1)
        bp.solve_packed(packed, rp)
        torch.cuda.synchronize()
        assert bytes(ra.cpu().numpy()) == bytes(rp.cpu().numpy())
    for i in range(n):
        np.testing.assert_array_equal(_state(a[i])[0], _state(p[i])[0])
        np.testing.assert_array_equal(_state(a[i])[1], _state(p[i])[1])
    ba.close()
    bp.close()


@pytest.mark.parametrize("host", [False, True])
def test_controller_solve_packed_equals_solve(host):
    # a Problem built once and edited in place gives the bits of per-call solves
    import torch
    c, pr = _mix()[1]
    a, p = S.Controller(c), S.Controller(c)
    f32 = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.float32))
    if host:
        x0, xr, fe = f32(pr["x0"]), f32(pr["xref"]), f32(pr["f_ext"])
    else:
        x0, xr, fe, _ = _tensors(pr)
    prob = p.problem(x0, xr, pr["gait"], fe, 0, host=host)
    for tick in range(3):
        g = _gait(pr, tick, c)
        prob.gait.phase0, prob.shift = g["phase0"], min(tick, 1)
        if host:
            ra = a.solve_host(x0, xr, g, fe, min(tick, 1))
            rp = p.solve_packed(prob, S.Result())
            torch.cuda.synchronize()
            assert bytes(ra) == bytes(rp)
        else:
            ra = a.solve(x0, xr, g, fe, min(tick, 1))
            rp = p.solve_packed(prob, torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device="cuda"))
            torch.cuda.synchronize()
            assert bytes(ra.cpu().numpy()) == bytes(rp.cpu().numpy())
    np.testing.assert_array_equal(_state(a)[0], _state(p)[0])
    np.testing.assert_array_equal(_state(a)[1], _state(p)[1])


def test_batch_replans_when_the_controllers_change():
    # one batch object alternates between two lists of controllers (the launch
    # plan is cached per list of handles); every tick equals the plain solves, and
    # a list with a duplicate is still rejected after a plan was cached
    import torch
    mix = _mix()
    lists = [[0, 1, 2, 3, 4, 5], [6, 7, 8, 9, 10, 1]]
    batched = {i: S.Controller(c) for i, (c, _) in enumerate(mix)}
    plain = {i: S.Controller(c) for i, (c, _) in enumerate(mix)}
    tens = [_tensors(p) for _, p in mix]
    b = S.Batch(len(mix), sum(c.workspace_bytes() + 256 for c in batched.values()))
    ticks = {i: 0 for i in batched}
    for rnd in range(4):
        idx = lists[rnd % 2]
        res = torch.empty(len(idx) * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
        probs, want = [], []
        for i in idx:
            x0, xr, fe, ft = tens[i]
            g = _gait(mix[i][1], ticks[i], mix[i][0])
            sh = min(ticks[i], 1)
            want.append(plain[i].solve(x0, xr, g, fe, sh, feet=ft).clone())
            probs.append(batched[i].problem(x0, xr, g, fe, sh, feet=ft))
            ticks[i] += 1
        b.solve([batched[i] for i in idx], probs, res)
        torch.cuda.synchronize()
        for k in range(len(idx)):
            assert bytes(res[k * S.RESULT_BYTES:(k + 1) * S.RESULT_BYTES].cpu().numpy()) == \
                bytes(want[k].cpu().numpy())
    with pytest.raises(S.SBSError) as e:
        b.solve([batched[0], batched[1], batched[0]], probs[:3], res)
    assert e.value.status == S.ERR_INVALID_ARG
    b.close()


def test_tile_tuner_times_every_candidate():
    from paper_2403_11383_b300 import tuning
    mix = _mix()
    tens = [_tensors(p) for _, p in mix]
    best, ms = tuning.tile_for_batch([c for c, _ in mix], [(t[0], t[1], p["gait"], t[2], t[3]) for t, (_, p) in
                                                           zip(tens, mix)], tiles=(64, 128, 256), ticks=2)
    assert set(ms) == {64, 128, 256} and all(v > 0 for v in ms.values())
    assert best == min(ms, key=ms.get)


def test_two_batches_on_two_streams_at_once():
    # two batches of independent controllers ticking concurrently on two streams
    # give the bits of the same ticks run one after the other: no state is shared
    # between batches
    import torch
    mix = _mix()
    half = len(mix) // 2
    groups = [list(range(half)), list(range(half, len(mix)))]
    tens = [_tensors(p) for _, p in mix]

    def run(concurrent):
        ctls = [S.Controller(c) for c, _ in mix]
        batches, packs, outs = [], [], []
        for g in groups:
            cs = [ctls[i] for i in g]
            batches.append(S.Batch(len(g), 2 * sum(c.workspace_bytes() + 256 for c in cs), inflight=2))
            packs.append([S.Packed(cs, [ctls[i].problem(*tens[i][:2], mix[i][1]["gait"], tens[i][2], sh,
                                                        feet=tens[i][3]) for i in g]) for sh in (0, 1)])
            outs.append(torch.empty(len(g) * S.RESULT_BYTES, dtype=torch.uint8, device="cuda"))
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        for tick in range(3):
            for k in range(2):
                if concurrent:
                    with torch.cuda.stream(streams[k]):
                        batches[k].solve_packed(packs[k][min(tick, 1)], outs[k], stream=streams[k])
                else:
                    batches[k].solve_packed(packs[k][min(tick, 1)], outs[k])
                    torch.cuda.synchronize()
            torch.cuda.synchronize()
        res = [bytes(o.cpu().numpy()) for o in outs]
        states = [_state(c) for c in ctls]
        for b in batches:
            b.close()
        return res, states

    ra, sa = run(False)
    rb, sb = run(True)
    assert ra == rb
    for (ma, va), (mb, vb) in zip(sa, sb):
        np.testing.assert_array_equal(ma, mb)
        np.testing.assert_array_equal(va, vb)


def test_checkpoint_resume_in_the_batch():
    # controllers saved after a batched tick and restored into fresh handles
    # continue in a batch with the same bits as the uninterrupted ones
    import torch
    mix = _mix()
    n = len(mix)
    tens = [_tensors(p) for _, p in mix]
    a = [S.Controller(c) for c, _ in mix]
    ba = S.Batch(n, sum(c.workspace_bytes() + 256 for c in a))
    res = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    probs = lambda cs, tick: [cs[i].problem(*tens[i][:2], _gait(mix[i][1], tick, mix[i][0]), tens[i][2],
                                            min(tick, 1), feet=tens[i][3]) for i in range(n)]
    ba.solve(a, probs(a, 0), res)
    torch.cuda.synchronize()
    blobs = [c.get_state() for c in a]
    ba.solve(a, probs(a, 1), res)
    torch.cuda.synchronize()
    want = bytes(res.cpu().numpy())
    fresh = [S.Controller(c) for c, _ in mix]
    for c, blob in zip(fresh, blobs):
        c.set_state(blob)
    bf = S.Batch(n, sum(c.workspace_bytes() + 256 for c in fresh))
    rf = torch.empty_like(res)
    bf.solve(fresh, probs(fresh, 1), rf)
    torch.cuda.synchronize()
    assert bytes(rf.cpu().numpy()) == want
    for i in range(n):
        np.testing.assert_array_equal(_state(a[i])[0], _state(fresh[i])[0])
        np.testing.assert_array_equal(_state(a[i])[1], _state(fresh[i])[1])
    ba.close()
    bf.close()


def test_large_elite_set_batch_equals_plain():
    # more than 2048 elites: 1024 virtual lanes, refit by 1024-thread blocks in a
    # plain solve and by 128-thread blocks in eight passes in a batch, same bits
    import torch
    base = W.config("plain_mppi_k512_h12")
    specs = [dict(K=65536, H=5, method="elite", elite_count=3277),
             dict(K=40000, H=6, method="elite", elite_count=2500, adaptive=True),
             dict(K=4096, H=8, method="elite", elite_count=205)]
    mix = []
    for i, sp in enumerate(specs):
        c = dict(base)
        c.update(sp)
        c.update(seed=300 + i, ctrl=i)
        mix.append((c, W.problem(c)))
    plain = [S.Controller(c) for c, _ in mix]
    batched = [S.Controller(c) for c, _ in mix]
    tens = [_tensors(p) for _, p in mix]
    n = len(mix)
    # two selections over more than 32 768 costs need 2 x 65 792 counter words,
    # workspace / 8192 of which the batch holds
    b = S.Batch(n, max(sum(c.workspace_bytes() + 256 for c in batched), 2 << 30))
    res = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for tick in range(2):
        probs, want = [], []
        for i, (c, p) in enumerate(mix):
            x0, xr, fe, _ = tens[i]
            g = _gait(p, tick, c)
            want.append(plain[i].solve(x0, xr, g, fe, min(tick, 1)).clone())
            probs.append(batched[i].problem(x0, xr, g, fe, min(tick, 1)))
        b.solve(batched, probs, res)
        torch.cuda.synchronize()
        for i in range(n):
            assert bytes(res[i * S.RESULT_BYTES:(i + 1) * S.RESULT_BYTES].cpu().numpy()) == \
                bytes(want[i].cpu().numpy())
            np.testing.assert_array_equal(_state(batched[i])[0], _state(plain[i])[0])
            np.testing.assert_array_equal(_state(batched[i])[1], _state(plain[i])[1])
    b.close()


@pytest.mark.parametrize("theta", [S.THETA_STORE, S.THETA_REGENERATE])
@pytest.mark.parametrize("mode", [S.BATCH_GRID, S.BATCH_PERSISTENT])
def test_multi_step_refit_items_equal_plain(mode, theta):
    # batched refit items of several steps (elite sets up to 2048): one item of a
    # whole 128-step horizon, items that end in a short one and a frequency item,
    # two-step items at 2048 elites, and one step per item just above 2048 and at
    # H = 1; beside an MPPI controller, so the grid-mode tick is split
    import torch
    base = W.config("plain_mppi_k512_h12")
    specs = [dict(K=64, H=128, dt_us=1000, method="elite", elite_count=1),
             dict(K=130, H=13, method="elite", elite_count=7),
             dict(K=2000, H=128, dt_us=1000, method="elite", elite_count=100, adaptive=True),
             dict(K=40960, H=6, method="elite", elite_count=2048),
             dict(K=40980, H=3, method="elite", elite_count=2049, adaptive=True),
             dict(K=6000, H=1, method="elite", elite_count=300),
             dict(K=3000, H=20, method="mppi")]
    mix = []
    for i, sp in enumerate(specs):
        c = dict(base)
        c.update(sp)
        c.update(seed=700 + i, ctrl=i)
        mix.append((c, W.problem(c)))
    plain = [S.Controller(c) for c, _ in mix]
    batched = [S.Controller(c) for c, _ in mix]
    for ctl in plain + batched:
        ctl.set_theta_mode(theta)
    tens = [_tensors(p) for _, p in mix]
    n = len(mix)
    # two selections over more than 32 768 costs: their counter words need a 2 GB arena
    b = S.Batch(n, max(sum(c.workspace_bytes() + 256 for c in batched), 2 << 30))
    b.set_mode(mode)
    b.set_theta_mode(theta)
    res = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    for tick in range(3):
        probs, want = [], []
        for i, (c, p) in enumerate(mix):
            x0, xr, fe, _ = tens[i]
            g = _gait(p, tick, c)
            want.append(plain[i].solve(x0, xr, g, fe, min(tick, 1)).clone())
            probs.append(batched[i].problem(x0, xr, g, fe, min(tick, 1)))
        b.solve(batched, probs, res)
        torch.cuda.synchronize()
        for i in range(n):
            assert bytes(res[i * S.RESULT_BYTES:(i + 1) * S.RESULT_BYTES].cpu().numpy()) == \
                bytes(want[i].cpu().numpy()), (i, tick)
            np.testing.assert_array_equal(_state(batched[i])[0], _state(plain[i])[0])
            np.testing.assert_array_equal(_state(batched[i])[1], _state(plain[i])[1])
    b.close()


def test_budget_admission_rejects_without_side_effects():
    import torch
    mix = _mix()[:3]
    ctls = [S.Controller(c) for c, _ in mix]
    tens = [_tensors(p) for _, p in mix]
    need = sum(c.workspace_bytes() + 256 for c in ctls)
    b = S.Batch(3, need - 4096)
    res = torch.empty(3 * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    probs = [ctls[i].problem(*tens[i][:2], mix[i][1]["gait"], tens[i][2], 0) for i in range(3)]
    with pytest.raises(S.SBSError) as e:
        b.solve(ctls, probs, res)
    assert e.value.status == S.ERR_BUDGET
    # the controllers were not touched: their first solve still initialises them
    b2 = S.Batch(3, need)
    b2.solve(ctls, probs, res)
    torch.cuda.synchronize()
    for i in range(3):
        assert S.parse_result(res[i * S.RESULT_BYTES:(i + 1) * S.RESULT_BYTES].cpu().numpy())["iter"] == 0


def test_batch_rejects_duplicates_and_mixed_tiles():
    import torch
    mix = _mix()[:2]
    a = S.Controller(mix[0][0])
    c128 = S.Controller(mix[1][0])
    c64 = S.Controller(mix[1][0], tile=64)
    tens = [_tensors(p) for _, p in mix]
    b = S.Batch(4, 1 << 28)
    res = torch.empty(4 * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    pa = a.problem(*tens[0][:2], mix[0][1]["gait"], tens[0][2], 0)
    with pytest.raises(S.SBSError):
        b.solve([a, a], [pa, pa], res)
    with pytest.raises(S.SBSError):
        b.solve([c128, c64], [c128.problem(*tens[1][:2], mix[1][1]["gait"], tens[1][2], 0),
                              c64.problem(*tens[1][:2], mix[1][1]["gait"], tens[1][2], 0)], res)


def test_autotune_picks_a_mode_and_results_stay_valid():
    import torch
    mix = _mix()
    ctls = [S.Controller(c) for c, _ in mix]
    tens = [_tensors(p) for _, p in mix]
    b = S.Batch(len(mix), sum(c.workspace_bytes() + 256 for c in ctls))
    res = torch.empty(len(mix) * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    probs = [ctls[i].problem(*tens[i][:2], mix[i][1]["gait"], tens[i][2], 0, feet=tens[i][3])
             for i in range(len(mix))]
    g_ms, p_ms = b.autotune(ctls, probs, res, ticks=2)
    assert g_ms > 0 and p_ms > 0
    assert b.mode() == (S.BATCH_GRID if g_ms <= p_ms else S.BATCH_PERSISTENT)
    b.solve(ctls, probs, res)
    torch.cuda.synchronize()
    for i in range(len(mix)):
        r = S.parse_result(res[i * S.RESULT_BYTES:(i + 1) * S.RESULT_BYTES].cpu().numpy())
        # autotune ticks: 2 launch modes x 2 deviation modes (stored, regenerated) x
        # (1 + 2); this mix has extended features, so one sample per thread only
        assert r["status"] in (S.OK, S.ERR_DIVERGED) and r["iter"] == 12


def test_batch_host_memory_equals_device():
    # sbs_batch_solve_host: the same ticks from host arrays (one staged copy in, one
    # out) give the bits of device-memory ticks, over warm-started ticks, with
    # ground-fixed feet and external forces among the inputs
    import torch
    mix = _mix()
    dev_c = [S.Controller(c) for c, _ in mix]
    host_c = [S.Controller(c) for c, _ in mix]
    tens = [_tensors(p) for _, p in mix]
    host = []
    for _, p in mix:
        a = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.float32))
        host.append((a(p["x0"]), a(p["xref"]), a(p["f_ext"]), a(p["feet"]) if "feet" in p else None))
    n = len(mix)
    bd = S.Batch(n, sum(c.workspace_bytes() + 256 for c in dev_c))
    bh = S.Batch(n, 2 * sum(c.workspace_bytes() + 256 for c in host_c), inflight=2)
    res_d = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    res_h = np.zeros(n * S.RESULT_BYTES, dtype=np.uint8)
    for tick in range(3):
        shift = 0 if tick == 0 else 1
        pd, ph = [], []
        for i, (c, p) in enumerate(mix):
            g = _gait(p, tick, c)
            x0, xr, fe, ft = tens[i]
            pd.append(dev_c[i].problem(x0, xr, g, fe, shift, feet=ft))
            hx, hr, hf, hft = host[i]
            ph.append(host_c[i].problem(hx, hr, g, hf, shift, host=True, feet=hft))
        bd.solve(dev_c, pd, res_d)
        bh.solve_host(S.Packed(host_c, ph), res_h)  # returns with the results on the host
        torch.cuda.synchronize()
        np.testing.assert_array_equal(res_h, res_d.cpu().numpy())
        for i in range(n):
            md, vd = _state(dev_c[i])
            mh, vh = _state(host_c[i])
            np.testing.assert_array_equal(mh, md)
            np.testing.assert_array_equal(vh, vd)
    # device pointers are refused by the host entry point
    with pytest.raises(S.SBSError):
        bh.solve_host(S.Packed(host_c, pd), res_h)
    bd.close()
    bh.close()


def test_host_inputs_in_place_equal_gathered():
    # inputs written into the batch's pinned staging (sbs_batch_host_inputs) give the
    # bits of the same inputs gathered from the caller's arrays, over warm ticks
    import torch
    mix = W.batch_mix(8, seed=41)
    for c, _ in mix:
        c["tile"] = 128
    ta = [S.Controller(c) for c, _ in mix]
    tb = [S.Controller(c) for c, _ in mix]
    n = len(mix)
    ba = S.Batch(n, sum(c.workspace_bytes() + 256 for c in ta))
    bb = S.Batch(n, sum(c.workspace_bytes() + 256 for c in tb))
    gaits = [p["gait"] for _, p in mix]
    h = [tuple(np.ascontiguousarray(np.float32(p[k])) for k in ("x0", "xref", "f_ext")) for _, p in mix]
    pb = S.Packed(tb, [tb[i].problem(h[i][0], h[i][1], gaits[i], h[i][2], 1, host=True) for i in range(n)])
    pa, views = ba.host_inputs(ta, gaits, shift=1)
    ra = np.zeros(n * S.RESULT_BYTES, dtype=np.uint8)
    rb = np.zeros_like(ra)
    rng = np.random.default_rng(5)
    for tick in range(3):
        for i in range(n):
            x0 = (h[i][0] + np.float32(0.01) * rng.standard_normal(12).astype(np.float32)).astype(np.float32)
            h[i][0][:] = x0  # the gathered side reads the caller's arrays
            views[i]["x0"][:] = x0
            views[i]["xref"][:] = h[i][1]
            views[i]["f_ext"][:] = h[i][2]
        ba.solve_host(pa, ra)
        bb.solve_host(pb, rb)
        np.testing.assert_array_equal(ra, rb)
        for i in range(n):
            np.testing.assert_array_equal(ta[i].read(S.BUF_MEAN).cpu().numpy(), tb[i].read(S.BUF_MEAN).cpu().numpy())
    ba.close()
    bb.close()
