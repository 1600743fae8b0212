"""GPU parity of ball joints (3 DOF: rotation vector, angular velocity in the child frame) against
the FP64 oracle: random trees mixing ball joints with hinges and sliders on fixed and floating
bases, an Ant whose hips are ball joints walking on the ground (contact rows through the ball
DOFs), and a batch mixing it with the plain Ant. Env types with ball joints run the global-rows
kernel variant. (The step derivative and the dynamics queries of ball-joint types are checked in
test_gpu_adjoint.py and test_gpu_control.py.)"""
import numpy as np
import pytest

from paper_2108_10470_gb300 import workloads as W
from test_gpu_parity import check_rollout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10470_gb300 import build
    build.build_library()
    torch.cuda.set_device(0)


def tree(seed, n_links, floating):
    rng = np.random.default_rng(seed)
    while True:
        m = W.random_tree(rng, n_links, floating, allow_fixed=False, ball_joints=True)
        if (m.jtype == W.JOINT_SPHERICAL).any() and m.n_gen <= 32:
            break
    m.armature = np.full(m.n_links, 0.05)  # keep the joint-space inertia well conditioned
    m.dof_noise = 0.3
    return m


@pytest.mark.parametrize("seed,n_links,floating", [(3, 6, False), (5, 9, True), (8, 12, False)])
@pytest.mark.parametrize("steps,rtol,atol", [(1, 1e-4, 1e-5), (16, 1e-3, 1e-3)])
def test_random_trees_with_ball_joints(seed, n_links, floating, steps, rtol, atol):
    w = W.homogeneous("balltree", tree(seed, n_links, floating), 37)
    check_rollout(w, steps, rtol, atol, min_same=1.0)


@pytest.mark.parametrize("steps,rtol,atol", [(1, 1e-4, 1e-5), (16, 1e-3, 1e-3)])
def test_ball_hip_ant_on_the_ground(steps, rtol, atol):
    w = W.homogeneous("ball_ant", W.ant(ball_hips=True), 67)
    check_rollout(w, steps, rtol, atol)


def test_ball_hip_ant_beside_the_ant():
    models = [W.ant(), W.ant(ball_hips=True)]
    eam = np.array([i % 2 for i in range(64)], np.int32)
    w = W.Workload("ants", models, eam, 1, 64, W.Params())
    check_rollout(w, 4, 1e-3, 1e-3)


def test_ball_hip_ant_persistent_launch():
    """The persistent launch (one tile body per variant) steps ball-joint envs like the per-type
    launch: against the oracle at 4 steps."""
    from paper_2108_10470_gb300 import sim
    w = W.homogeneous("ball_ant", W.ant(ball_hips=True), 64)
    check_rollout(w, 4, 1e-3, 1e-3, flags=sim.SIM_FLAG_SIGNATURE | sim.SIM_FLAG_PERSISTENT)


def test_ball_hip_ant_dof_forces_and_body_states():
    """The DOF-force view (actuation - damping qd per ball DOF) and the rigid-body states after the
    step (one more kinematics pass through the ball joints) against the oracle."""
    from paper_2108_10470_gb300 import sim
    from test_gpu_control import rollout_both, within
    w = W.homogeneous("ball_ant", W.ant(ball_hips=True), 37)
    flags = sim.SIM_FLAG_SIGNATURE | sim.SIM_FLAG_DOF_FORCE | sim.SIM_FLAG_RIGID_BODY_STATE
    g, o = rollout_both(w, 2, flags, lambda k: {})
    same = (g[0]["sig"] == o[0]["sig"]) & (g[1]["sig"] == o[1]["sig"])
    assert same.mean() >= 0.9
    m = w.models[0]
    dmask = np.repeat(same, m.n_jdof)
    bmask = np.repeat(same, m.n_body)
    ok, f = within(g[0]["dof_force"][dmask], o[0]["dof_force"][dmask], 1e-4, 1e-4)
    assert ok, f
    ok, f = within(g[0]["body"][bmask][:, :3], o[0]["body"][bmask][:, :3], 1e-4, 1e-5)
    assert ok, f
    qg, qo = g[1]["body"][bmask][:, 3:7], o[1]["body"][bmask][:, 3:7]
    assert (np.abs((qg * qo).sum(1)) > 1 - 1e-4).mean() >= 0.98


@pytest.mark.parametrize("steps,rtol,atol", [(1, 1e-4, 1e-5), (16, 1e-3, 1e-3)])
def test_ball_joint_humanoid(steps, rtol, atol):
    """The Humanoid with ball joints at the abdomen and hips (instead of hinge chains through
    virtual links; 17 links, 21 joint DOF) on the ground."""
    w = W.homogeneous("ball_humanoid", W.humanoid(ball_joints=True), 37)
    check_rollout(w, steps, rtol, atol)


def test_spinning_body_on_a_ball_joint_eight_lanes():
    """A single body on a ball joint at its centre of mass (3 generalized DOFs: the 8-lane kernel),
    spinning about all three axes of an asymmetric inertia without gravity, with random initial
    rotations: against the oracle over 16 steps."""
    prm = W.Params(gravity=(0.0, 0.0, 0.0))
    m = W.ball_pendulum(mass=1.0, com=(0, 0, 0), inertia=(0.3, 0.5, 0.8, 0, 0, 0), name="spinner")
    m.dof_noise = 1.0
    w = W.homogeneous("spinner", m, 40, params=prm)
    check_rollout(w, 16, 1e-3, 1e-3, min_same=1.0)
