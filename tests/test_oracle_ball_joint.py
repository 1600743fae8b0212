"""Pins of the FP64 oracle's ball joint (3 DOF: position = rotation vector r with R_J = exp([r]x),
velocity = the child's angular velocity relative to the parent in child coordinates, motion
subspace [I; 0], RBDA Table 4.1) against independent algorithms, a hinge, and the invariants of a
rigid body turning about a fixed point (no GPU)."""
import numpy as np
import pytest

import oracle
from paper_2108_10470_gb300 import workloads as W
from test_oracle_dynamics import one_env, random_state


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("floating", [False, True])
def test_aba_matches_crba_rnea_with_ball_joints(seed, floating):
    """ABA with 3-DOF joint blocks (RBDA Table 7.1) against CRBA + RNEA on random trees that mix
    ball joints with hinges and sliders: H qdd = tau - C to 1e-10, RNEA inverts ABA."""
    rng = np.random.default_rng(7000 + 10 * seed + floating)
    n_links = int(rng.integers(2, 9))
    m = W.random_tree(rng, n_links, floating, ball_joints=True)
    if not (m.jtype == W.JOINT_SPHERICAL).any():
        pytest.skip("tree drew no ball joint")
    O = oracle.Oracle(one_env(m))
    n = O.ngen()
    root, dof = random_state(rng, m)
    tau = rng.uniform(-5, 5, n)
    qdd = O.aba(0, root, dof, tau)
    H = O.crba(0, root, dof)
    C = O.rnea(0, root, dof, np.zeros(n))
    assert np.allclose(H, H.T, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(H) > 0)
    res = H @ qdd + C - tau
    scale = np.abs(H @ qdd).max() + np.abs(C).max() + np.abs(tau).max()
    assert np.abs(res).max() <= 1e-10 * scale
    assert np.allclose(O.rnea(0, root, dof, qdd), tau, rtol=0, atol=1e-10 * scale)


def test_planar_swing_equals_the_hinge():
    """A rod on a ball joint released from a rotation about y swings exactly like the same rod on a
    hinge about y (the other two DOFs stay at rest by symmetry): 300 production steps, positions and
    rates equal to 1e-12, the x and z components zero."""
    dt, sub = 1.0 / 120.0, 2
    ball = oracle.Oracle(one_env(W.ball_pendulum(), dt=dt, substeps=sub))
    hinge = oracle.Oracle(one_env(W.pendulum(), dt=dt, substeps=sub))
    rb = np.zeros((1, 13)); rb[0, 6] = 1.0
    rh = rb.copy()
    db = np.array([[0.0, 0.0], [0.9, 0.0], [0.0, 0.0]])
    dh = np.array([[0.9, 0.0]])
    act = np.array([0.0, 0.3, 0.0])
    for _ in range(300):
        ball.step(rb, db, act)
        hinge.step(rh, dh, act[1:2])
    assert abs(db[1, 0] - dh[0, 0]) < 1e-12 and abs(db[1, 1] - dh[0, 1]) < 1e-12
    assert np.abs(db[[0, 2]]).max() < 1e-12
    assert abs(dh[0, 0]) > 0.1  # it did swing


def test_free_rotation_about_the_centre_of_mass():
    """A body on a ball joint at its centre of mass, without gravity, spinning about all three axes
    of an asymmetric inertia: the world angular momentum R I w and the kinetic energy 1/2 w.I w stay
    constant (to the first-order integrator's error, which shrinks with the step: ratio ~2 when the
    step halves). Composing the rotation increment on the wrong side breaks both."""
    I = np.diag([0.3, 0.5, 0.8])
    m = W.ball_pendulum(mass=1.0, com=(0, 0, 0), inertia=(0.3, 0.5, 0.8, 0, 0, 0), name="spinner")

    def drift(substeps, t_end=0.25):
        prm = W.Params(gravity=(0.0, 0.0, 0.0))
        O = oracle.Oracle(one_env(m, params=prm, dt=1e-3, substeps=substeps))
        root = np.zeros((1, 13)); root[0, 6] = 1.0
        dof = np.array([[0.0, 1.0], [0.0, -2.0], [0.0, 3.0]])

        def invariants():
            R, _ = O.link_pose(0, root, dof, 1)
            w = dof[:, 1]
            return R @ I @ w, 0.5 * w @ I @ w
        L0, E0 = invariants()
        for _ in range(int(round(t_end / 1e-3))):
            O.step(root, dof, np.zeros(3))
        L1, E1 = invariants()
        return np.linalg.norm(L1 - L0) / np.linalg.norm(L0), abs(E1 - E0) / E0
    l4, e4 = drift(4)
    l8, e8 = drift(8)
    assert l4 < 2e-3 and e4 < 2e-3
    assert 1.5 < l4 / l8 < 2.6


def test_rotation_vector_round_trip_past_pi():
    """The joint position is stored as the shorter rotation: a spin that carries the joint past pi
    about one axis comes back as a rotation vector of norm <= pi with the same rotation matrix."""
    prm = W.Params(gravity=(0.0, 0.0, 0.0))
    m = W.ball_pendulum(mass=1.0, com=(0, 0, 0), inertia=(0.4, 0.4, 0.4, 0, 0, 0), name="wheel")
    O = oracle.Oracle(one_env(m, params=prm, dt=1e-2, substeps=2))
    root = np.zeros((1, 13)); root[0, 6] = 1.0
    dof = np.array([[0.0, 0.0], [0.0, 0.0], [3.1, 10.0]])  # near pi about z, spinning at 10 rad/s
    O.step(root, dof, np.zeros(3))
    r = dof[:, 0]
    assert np.linalg.norm(r) <= np.pi + 1e-12
    ang = 3.1 + 10.0 * 1e-2  # 3.2 rad about z == -(2 pi - 3.2) about z
    assert abs(r[2] - (ang - 2 * np.pi)) < 1e-9 and np.abs(r[:2]).max() < 1e-12


def test_rk4_reference_refuses_ball_joints():
    O = oracle.Oracle(one_env(W.ball_pendulum()))
    root = np.zeros((1, 13)); root[0, 6] = 1.0
    dof = np.zeros((3, 2))
    assert O.rk4(root, dof, np.zeros(3), 1e-3, 1) == -2


def test_contact_rows_match_the_link_jacobian():
    """Each contact row J_r = k . d(x_dot)/d(nu) of a ball-hip Ant on the ground (built joint by
    joint along the contact link's path) against the same direction through the link's spatial
    Jacobian (velocity propagation with the motion subspaces): k . v_O + (r x k) . w, with
    r = x - O the contact point from the link origin, to 1e-12."""
    w = W.homogeneous("ball_ant", W.ant(ball_hips=True), 1)
    O = oracle.Oracle(w)
    root, dof, acts = W.seeded_inputs(w, 0, 40)
    root = root.astype(np.float64); dof = dof.astype(np.float64)
    n_checked = 0
    for k in range(40):
        O.step(root, dof, acts[k])
        rows = O.rows(0, root, dof)
        for r in range(len(rows["d"])):
            if rows["kind"][r] == 0:
                continue
            li = int(rows["link"][r])
            Jl = O.jacobian(0, root, dof, li)
            _, p = O.link_pose(0, root, dof, li)
            kk, x = rows["k"][r], rows["x"][r]
            ref = kk @ Jl[3:] + np.cross(x - p, kk) @ Jl[:3]
            assert np.allclose(rows["J"][r], ref, rtol=0, atol=1e-12), (k, r)
            n_checked += 1
    assert n_checked > 20
