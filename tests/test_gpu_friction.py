"""GPU parity of the friction-cone constraint on the policy output (Sec. IV-B):
stance forces projected orthogonally onto |Gamma_xy| <= mu Gamma_z before they
act, no penalty; per-step and spline policies, alone and with world-fixed feet."""
import numpy as np
import pytest

from gpu_helpers import mppi_parity
from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    S.lib()
    return torch


@pytest.mark.parametrize("name,extra", [
    ("plain_mppi_k512_h12", {}),
    ("plain_mppi_k512_h12", dict(K=3001, H=25, seed=41)),
    ("worldfeet_mppi_k4096_h25", dict(K=2048, seed=43)),
    ("spline_k262144_h100", dict(K=3000, H=25, dt_us=20000, method="mppi", compare_mppi=False, sigma_init=5.0,
                                 seed=47)),
])
def test_projected_forces_mppi_parity(cuda, name, extra):
    cfg = W.config(name)
    cfg.update(extra)
    cfg["friction_project"] = True
    rep = mppi_parity(cfg, W.problem(cfg), f"friction {name}")
    assert rep["gated"] > 0
