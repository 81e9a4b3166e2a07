"""Closed-loop episodes on the single-rigid-body world (paper_2403_11383_b300.episodes):
without disturbances the controllers keep the robot walking; under random
+-5 N/Nm wrenches gait adaptation (the discrete frequency set) keeps more
robots up than the fixed gait, the effect of the paper's closed-loop comparison
(Sec. V-B, Table I)."""
import pytest

from paper_2403_11383_b300 import episodes as E
from paper_2403_11383_b300 import sbs as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    S.lib()
    return torch


@pytest.mark.parametrize("variant", ["naive_fixed", "mppi_fixed", "naive_adaptive"])
def test_walks_without_disturbance(cuda, variant):
    r = E.run(variant, episodes=8, seconds=3.0, wrench=0.0, K=4096)
    assert r["success_rate"] == 1.0, r


def test_gait_adaptation_rejects_disturbances_better(cuda):
    fixed = E.run("naive_fixed", episodes=16, seconds=6.0, wrench=5.0, K=10_000, seed=1)
    adapt = E.run("naive_adaptive", episodes=16, seconds=6.0, wrench=5.0, K=10_000, seed=1)
    assert adapt["success_rate"] >= fixed["success_rate"] + 0.25, (fixed, adapt)
    assert adapt["mean_survival_s"] > fixed["mean_survival_s"]
    assert 1.3 < adapt["mean_frequency_hz"] <= 2.4
