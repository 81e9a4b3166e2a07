"""The batched workload exactly as bench.py times it: 256 controllers of uneven K,
H, gait and method, 256-sample tiles, grid launches replayed from a graph, two
ticks in flight and packed arguments.  Every controller's two ticks (an
initialising one, then warm-started ones) equal its own plain solve bit for bit,
and the largest MPPI and elite controllers of the mix, solved plainly at the same
tile, match the FP64 oracle within the parity gates: so the timed batched tick
computes what the oracle computes."""
import numpy as np
import pytest

from gpu_helpers import KAPPA_GATED, OracleRun, elite_parity, mppi_parity
from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mix():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    m = W.batch_config(256)
    assert all(c["tile"] == W.BATCH_TILE for c, _ in m)
    return m


def _state(ctl):
    return ctl.read(S.BUF_MEAN).cpu().numpy(), ctl.read(S.BUF_VAR).cpu().numpy()


def test_batched_tick_equals_plain_solves(mix):
    import torch
    d = lambda a: torch.tensor(np.float32(a), device="cuda")
    n = len(mix)
    ctls = [S.Controller(c) for c, _ in mix]
    x0, xr, fe = ([d(p[k]) for _, p in mix] for k in ("x0", "xref", "f_ext"))
    arena = sum(c.workspace_bytes() + 256 for c in ctls)
    b = S.Batch(n, 2 * arena, inflight=2)
    b.set_mode(S.BATCH_GRID)
    packed = [S.Packed(ctls, [ctls[i].problem(x0[i], xr[i], mix[i][1]["gait"], fe[i], sh) for i in range(n)])
              for sh in (0, 1)]
    res = [torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda") for _ in range(3)]
    states = []
    for t in range(3):
        b.solve_packed(packed[min(t, 1)], res[t])
        torch.cuda.synchronize()
        states.append([_state(c) for c in ctls])
    statuses = []
    for i, (cfg, prob) in enumerate(mix):
        twin = S.Controller(cfg)
        r = torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
        for t in range(3):
            twin.solve(x0[i], xr[i], prob["gait"], fe[i], min(t, 1), r)
            torch.cuda.synchronize()
            got = res[t][i * S.RESULT_BYTES:(i + 1) * S.RESULT_BYTES].cpu().numpy()
            assert bytes(got) == bytes(r.cpu().numpy()), (i, t)
            m, v = _state(twin)
            np.testing.assert_array_equal(states[t][i][0], m)
            np.testing.assert_array_equal(states[t][i][1], v)
        statuses.append(S.parse_result(r.cpu().numpy())["status"])
        twin.close()
    # most controllers of the mix stay well posed; the rest report divergence
    assert sum(s == S.OK for s in statuses) >= 0.8 * n
    b.close()


@pytest.mark.parametrize("method", ["mppi", "elite"])
def test_largest_controllers_of_the_mix_match_the_oracle(mix, method):
    # the largest controller whose samples are mostly well conditioned: the body is
    # unstable about its support (small roll errors grow about 30-fold per 0.1 s),
    # so over a 1 s open-loop horizon (H = 50) nearly every sample tumbles through
    # the pitch singularity to an infinite cost, and at H = 25 many are chaotic
    cands = sorted(((c["K"] * c["H"], i) for i, (c, _) in enumerate(mix) if c["method"] == method), reverse=True)
    for _, i in cands:
        J, _, _, _, kap = OracleRun(*mix[i]).rollout(want_theta=False)
        if np.mean(np.isfinite(J) & (J < 3e38) & (kap <= KAPPA_GATED)) >= 0.5:
            break
    cfg, prob = mix[i]
    assert cfg["K"] * cfg["H"] >= 4096 * 10
    if method == "mppi":
        rep = mppi_parity(cfg, prob, f"mix[{i}]", tile=W.BATCH_TILE)
    else:
        rep = elite_parity(cfg, prob, f"mix[{i}]", tile=W.BATCH_TILE)
    assert rep["gated"] >= 0.5 * cfg["K"], rep
