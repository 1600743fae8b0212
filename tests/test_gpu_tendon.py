"""Fixed tendons on the GPU against the FP64 oracle: spring-damper tendons, equality and limited
tendons on two-joint models, the Ant with three tendons, and the hand with coupled middle / distal
flexions holding a cube."""
import numpy as np
import pytest

from paper_2108_10470_gb300 import workloads as W
from test_gpu_parity import check_rollout
from test_oracle_tendon import NOGRAV, two_joints

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10470_gb300 import build
    build.build_library()
    torch.cuda.set_device(0)


TENDONS = {
    "spring": dict(coef=(1.0, -0.6), stiffness=20.0, damping=1.5, rest=0.1),
    "equality": dict(coef=(1.0, -1.0), limit=(0.0, 0.0)),
    "limit": dict(coef=(1.0, 1.0), limit=(-0.05, 0.05), stiffness=2.0),
}


@pytest.mark.parametrize("kind", sorted(TENDONS))
@pytest.mark.parametrize("steps,rtol,atol", [(1, 1e-4, 1e-5), (16, 1e-3, 1e-3)])
def test_two_joint_tendons_match_oracle(kind, steps, rtol, atol):
    w = W.homogeneous("pair", two_joints(tendon=TENDONS[kind]), 67, params=NOGRAV)
    check_rollout(w, steps, rtol, atol)


@pytest.mark.parametrize("steps,rtol,atol", [(1, 1e-4, 1e-5), (16, 1e-3, 1e-3)])
def test_coupled_hand_matches_oracle(steps, rtol, atol):
    check_rollout(W.hand_tendon_workload(37), steps, rtol, atol)


@pytest.mark.parametrize("steps,rtol,atol", [(1, 1e-4, 1e-5), (16, 1e-3, 1e-3)])
def test_tendon_ant_matches_oracle(steps, rtol, atol):
    """The Ant with a spring, a length-limited and an equality tendon (floating base, ground
    contacts and joint limits with tendon rows in the same solve)."""
    check_rollout(W.homogeneous("tendon_ant", W.ant(tendons=True), 67), steps, rtol, atol)


def test_equality_tendon_moves_joints_together_on_gpu():
    import torch
    from paper_2108_10470_gb300 import sim
    w = W.homogeneous("pair", two_joints(tendon=TENDONS["equality"]), 4, params=NOGRAV)
    s = sim.Sim(w)
    act = torch.zeros(8, device="cuda")
    act[0::2] = 0.2
    s.dof_actuation.copy_(act)
    for _ in range(120):
        s.step()
    d = s.dof_state.cpu().numpy().reshape(4, 2, 2)
    s.destroy()
    assert np.allclose(d[:, 0, 0], d[:, 1, 0], rtol=2e-3)
    assert np.allclose(d[:, 0, 0], 0.5 * 0.2 / 0.86 * (120 * w.dt) ** 2, rtol=0.02)
