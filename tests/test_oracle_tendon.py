"""Pins of the oracle's fixed tendons: the spring-damper on a tendon's length against the closed-form
recurrence of two decoupled joints, an equality tendon (limits lo = hi) coupling an actuated joint
to an unactuated one, and a length limit holding against constant joint torques."""
import numpy as np

import oracle
from paper_2108_10470_gb300 import workloads as W

NOGRAV = W.Params(gravity=(0.0, 0.0, 0.0))


def two_joints(I=(0.3, 0.5), arm=(0.02, 0.04), tendon=None):
    """A fixed base with two sibling links on revolute joints about z (decoupled joint-space inertia
    diag(I1 + a1, I2 + a2); no gravity torque about z)."""
    b = W._Builder("pair")
    base = b.link(-1, W.JOINT_FIXED, mass=1.0, inertia=(1, 1, 1, 0, 0, 0))
    l1 = b.link(base, W.JOINT_REVOLUTE, axis=(0, 0, 1), ppos=(0.3, 0, 0), mass=1.0,
                inertia=(0.1, 0.1, I[0], 0, 0, 0), armature=arm[0])
    l2 = b.link(base, W.JOINT_REVOLUTE, axis=(0, 0, 1), ppos=(-0.3, 0, 0), mass=1.0,
                inertia=(0.1, 0.1, I[1], 0, 0, 0), armature=arm[1])
    if tendon is not None:
        b.tendon([l1, l2], **tendon)
    return b.build()


def test_tendon_spring_closed_form():
    c, k, d, rest = (1.0, -0.6), 20.0, 1.5, 0.1
    m = two_joints(tendon=dict(coef=c, stiffness=k, damping=d, rest=rest))
    w = W.homogeneous("pair", m, 1, params=NOGRAV)
    O = oracle.Oracle(w)
    root = np.zeros((1, 13)); root[0, 6] = 1.0
    dof = np.array([[0.4, 0.0], [-0.2, 0.3]])
    q, qd = dof[:, 0].copy(), dof[:, 1].copy()
    inert = np.array([0.3 + 0.02, 0.5 + 0.04])
    h = w.dt / w.substeps
    cv = np.array(c)
    for _ in range(50):
        O.step(root, dof, np.zeros(2))
        for _sub in range(w.substeps):
            F = -k * (cv @ q - rest) - d * (cv @ qd)
            qd = qd + h * cv * F / inert
            q = q + h * qd
        assert np.allclose(dof[:, 0], q, atol=1e-12) and np.allclose(dof[:, 1], qd, atol=1e-12)


def test_equality_tendon_couples_joints():
    """l = q1 - q2 held at 0 by limits lo = hi = 0: torque on joint 1 alone moves both together."""
    m = two_joints(tendon=dict(coef=(1.0, -1.0), limit=(0.0, 0.0)))
    w = W.homogeneous("pair", m, 1, params=NOGRAV)
    O = oracle.Oracle(w)
    root = np.zeros((1, 13)); root[0, 6] = 1.0
    dof = np.zeros((2, 2))
    for _ in range(120):
        out = O.step(root, dof, np.array([0.2, 0.0]))
    assert abs(dof[0, 0] - 0.5 * 0.2 / 0.86 * (120 * w.dt) ** 2) < 0.02 * dof[0, 0]  # it moved as one body
    assert abs(dof[0, 0] - dof[1, 0]) < 2e-3 * abs(dof[0, 0])
    # shared acceleration: both joints accelerate like one body of inertia I1 + a1 + I2 + a2
    assert abs(dof[0, 1] - dof[1, 1]) < 1e-3 * abs(dof[0, 1])
    t = 120 * w.dt
    assert abs(dof[0, 1] - 0.2 / (0.32 + 0.54) * t) < 0.02 * dof[0, 1]


def test_tendon_length_limit_holds():
    m = two_joints(tendon=dict(coef=(1.0, 1.0), limit=(-10.0, 0.5)))
    w = W.homogeneous("pair", m, 1, params=NOGRAV)
    O = oracle.Oracle(w)
    root = np.zeros((1, 13)); root[0, 6] = 1.0
    dof = np.zeros((2, 2))
    for _ in range(300):
        O.step(root, dof, np.array([0.3, 0.2]))
    assert abs(dof[0, 0] + dof[1, 0] - 0.5) < 1e-3
    assert abs(dof[0, 1] + dof[1, 1]) < 1e-3
