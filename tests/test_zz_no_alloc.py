"""The allocation-free MPPI entry point (sbs_solve_mppi_static).

It serves callers that cannot allocate device memory when they solve: a
real-time control thread that must not block on an allocator, or a host
application or plug-in that owns all device memory.  Its per-solve scratch sits
in a static device array instead of handle-owned buffers; the kernel is the
ordinary rollout kernel, with the same tile, inputs, iteration counter and
warm-start shift, so two calls in a row through the C ABI must give the bits of
the ordinary sbs_solve path, and a warmed-up call must leave the device's
free memory unchanged.

This file is collected last, so a run that stops at the first failure has
already run every other test."""
import gc

import numpy as np
import pytest

from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def _state(ctl):
    import torch
    return torch.cat([ctl.read(S.BUF_MEAN), ctl.read(S.BUF_VAR)])


@pytest.mark.parametrize("variant", ["per_step", "adaptive_friction_projection"])
def test_static_entry_equals_solve_on_two_calls(variant):
    import torch
    assert torch.cuda.is_available()
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(K=1000, seed=17)  # several tiles and a ragged tail
    if variant != "per_step":  # the extended kernel instantiation, sampled frequencies
        cfg.update(adaptive=True, friction_project=True)
    prob = W.problem(cfg)
    x0, xref, fe = _dev(prob["x0"]), _dev(prob["xref"]), _dev(prob["f_ext"])
    gait1 = dict(prob["gait"])
    gait2 = dict(gait1, phase0=(gait1["phase0"] + cfg["q_init"] * cfg["dt_us"]) % W.PHASE_ONE)

    ref = S.Controller(cfg)
    ref.reset(gait1)
    D = ref.D
    state0 = _state(ref)
    ref_res = [ref.solve(x0, xref, gait1, fe, 0).clone()]
    ref_state = [_state(ref)]
    ref_res.append(ref.solve(x0, xref, gait2, fe, 1).clone())
    ref_state.append(_state(ref))

    states = [torch.empty(2 * D, device="cuda") for _ in range(2)]
    results = [torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device="cuda") for _ in range(2)]
    S.solve_mppi_static(cfg, x0, xref, gait1, fe, 0, state0, states[0], 0, results[0])
    torch.cuda.synchronize()
    # the second call, warmed up: nothing is allocated on the device (garbage of
    # earlier tests collected first: a collection during the call could only lower
    # the allocator's count)
    gc.collect()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    S.solve_mppi_static(cfg, x0, xref, gait2, fe, 1, states[0], states[1], 1, results[1])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() <= alloc0

    for got_state, got_res, want_state, want_res in zip(states, results, ref_state, ref_res):
        np.testing.assert_array_equal(got_state.cpu().numpy(), want_state.cpu().numpy())
        rg, rw = S.parse_result(got_res.cpu().numpy()), S.parse_result(want_res.cpu().numpy())
        assert rg["status"] == rw["status"] == S.OK
        np.testing.assert_array_equal(rg["u0"], rw["u0"])
        assert rg["cost_min"] == rw["cost_min"] and rg["ess"] == rw["ess"]
        assert rg["n_finite"] == rw["n_finite"] and rg["q_freq"] == rw["q_freq"]
    ref.close()


def test_static_entry_rejects_what_it_cannot_hold():
    import torch
    cfg = W.config("plain_mppi_k512_h12")
    prob = W.problem(cfg)
    x0, xref = _dev(prob["x0"]), _dev(prob["xref"])
    D = 12 * cfg["H"]
    s_in, s_out = torch.zeros(2 * D, device="cuda"), torch.zeros(2 * D, device="cuda")
    res = torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    big = dict(cfg, K=1 << 20, H=50)  # about 2.5 GB of scratch
    with pytest.raises(S.SBSError) as e:
        S.solve_mppi_static(big, x0, _dev(W.reference(50, 20000, prob["x0"], (0.3, 0))), prob["gait"], None, 0,
                            torch.zeros(1200, device="cuda"), torch.zeros(1200, device="cuda"), 0, res)
    assert e.value.status == S.ERR_BUDGET
    with pytest.raises(S.SBSError) as e:
        S.solve_mppi_static(dict(cfg, method="elite", elite_count=5), x0, xref, prob["gait"], None, 0, s_in, s_out,
                            0, res)
    assert e.value.status == S.ERR_INVALID_ARG
    with pytest.raises(S.SBSError) as e:
        S.solve_mppi_static(cfg, x0, xref, prob["gait"], None, 0, s_in, s_in, 0, res)
    assert e.value.status == S.ERR_INVALID_ARG
    # a capturing stream is refused before anything is enqueued, and the capture
    # then ends cleanly with an empty graph
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(S.SBSError) as e:
        with torch.cuda.graph(g, stream=s):
            S.solve_mppi_static(cfg, x0, xref, prob["gait"], None, 0, s_in, s_out, 0, res, stream=s)
    assert e.value.status == S.ERR_INVALID_ARG
    torch.cuda.synchronize()
