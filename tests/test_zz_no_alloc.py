"""The allocation-free MPPI entry point (sbs_solve_mppi_static) for callers that
cannot allocate device memory when they solve: called through the C ABI twice
in a row (a cold solve, then a warm-started one), it must agree with the
ordinary sbs_solve path within the parity tolerance of the other tests."""
import numpy as np
import pytest

from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

pytestmark = pytest.mark.gpu

MEAN_ATOL = 1e-4 * 21.0 * 9.81


def test_static_entry_matches_solve_on_two_calls():
    import torch
    assert torch.cuda.is_available()
    cfg = W.config("plain_mppi_k512_h12")
    cfg.update(K=1000, seed=17)  # several tiles and a ragged tail
    prob = W.problem(cfg)
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
    x0, xref, fe = dev(prob["x0"]), dev(prob["xref"]), dev(prob["f_ext"])
    gait1 = dict(prob["gait"])
    gait2 = dict(gait1, phase0=(gait1["phase0"] + cfg["q_init"] * cfg["dt_us"]) % W.PHASE_ONE)

    ref = S.Controller(cfg)
    ref.reset(gait1)
    D = ref.D
    state0 = torch.cat([ref.read(S.BUF_MEAN), ref.read(S.BUF_VAR)])
    ref_res = [ref.solve(x0, xref, gait1, fe, 0).clone()]
    ref_state = [torch.cat([ref.read(S.BUF_MEAN), ref.read(S.BUF_VAR)])]
    ref_res.append(ref.solve(x0, xref, gait2, fe, 1).clone())
    ref_state.append(torch.cat([ref.read(S.BUF_MEAN), ref.read(S.BUF_VAR)]))

    state1 = torch.empty(2 * D, device="cuda")
    state2 = torch.empty(2 * D, device="cuda")
    res1 = torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    res2 = torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    S.solve_mppi_static(cfg, x0, xref, gait1, fe, 0, state0, state1, 0, res1)
    S.solve_mppi_static(cfg, x0, xref, gait2, fe, 1, state1, state2, 1, res2)
    torch.cuda.synchronize()

    for got_state, got_res, want_state, want_res in ((state1, res1, ref_state[0], ref_res[0]),
                                                     (state2, res2, ref_state[1], ref_res[1])):
        g, w = got_state.cpu().numpy(), want_state.cpu().numpy()
        np.testing.assert_allclose(g[:D], w[:D], atol=MEAN_ATOL, rtol=0)
        np.testing.assert_allclose(g[D:], w[D:], rtol=1e-6)
        rg, rw = S.parse_result(got_res.cpu().numpy()), S.parse_result(want_res.cpu().numpy())
        assert rg["status"] == rw["status"] == S.OK
        np.testing.assert_allclose(rg["u0"], rw["u0"], atol=MEAN_ATOL)
        assert rg["cost_min"] == pytest.approx(rw["cost_min"], rel=1e-4)
        assert rg["n_finite"] == rw["n_finite"]
    ref.close()


def test_static_entry_rejects_what_it_cannot_hold():
    import torch
    cfg = W.config("plain_mppi_k512_h12")
    prob = W.problem(cfg)
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
    x0, xref = dev(prob["x0"]), dev(prob["xref"])
    D = 12 * cfg["H"]
    s_in, s_out = torch.zeros(2 * D, device="cuda"), torch.zeros(2 * D, device="cuda")
    res = torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    big = dict(cfg, K=1 << 20, H=50)  # about 2.5 GB of scratch
    with pytest.raises(S.SBSError) as e:
        S.solve_mppi_static(big, x0, dev(W.reference(50, 20000, prob["x0"], (0.3, 0))), prob["gait"], None, 0,
                            torch.zeros(1200, device="cuda"), torch.zeros(1200, device="cuda"), 0, res)
    assert e.value.status == S.ERR_BUDGET
    with pytest.raises(S.SBSError) as e:
        S.solve_mppi_static(dict(cfg, method="elite", elite_count=5), x0, xref, prob["gait"], None, 0, s_in, s_out,
                            0, res)
    assert e.value.status == S.ERR_INVALID_ARG
    with pytest.raises(S.SBSError) as e:
        S.solve_mppi_static(cfg, x0, xref, prob["gait"], None, 0, s_in, s_in, 0, res)
    assert e.value.status == S.ERR_INVALID_ARG
