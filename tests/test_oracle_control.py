"""Pins of the oracle's control inputs and extra outputs: implicit joint drives against the
closed-form recurrence of one driven joint, convergence to the target, external body forces and
torques against Newton-Euler on a free body, body states against the root state and forward
kinematics, and link Jacobians against finite differences of forward kinematics."""
import math

import numpy as np

import oracle
from paper_2108_10470_gb300 import workloads as W

NOGRAV = W.Params(gravity=(0.0, 0.0, 0.0))


def driven_joint(kp, kd, armature=0.05, damping=0.2, inertia=0.3):
    """A fixed base with one link on a revolute joint about z (no shapes, no gravity torque)."""
    b = W._Builder("driven")
    base = b.link(-1, W.JOINT_FIXED, mass=1.0, inertia=(1, 1, 1, 0, 0, 0))
    b.link(base, W.JOINT_REVOLUTE, axis=(0, 0, 1), mass=2.0, inertia=(0.5, 0.5, inertia, 0, 0, 0),
           armature=armature, damping=damping, drive=(kp, kd))
    return b.build()


def test_implicit_drive_closed_form():
    """Per substep h: qd' = qd + h (-c qd + kp (q* - q - h qd) + kd (qd* - qd)) / (I + a + h (h kp + kd)),
    q' = q + h qd' (no constraint rows, so the solve leaves v_free unchanged and dq = h v)."""
    kp, kd, a, c, I = 40.0, 3.0, 0.05, 0.2, 0.3
    w = W.homogeneous("driven", driven_joint(kp, kd, a, c, I), 1, params=NOGRAV)
    O = oracle.Oracle(w)
    root = np.zeros((1, 13)); root[0, 6] = 1.0
    dof = np.array([[0.1, -0.4]])
    qt, vt = 0.7, 0.25
    q, qd = 0.1, -0.4
    h = w.dt / w.substeps
    for step in range(50):
        out = O.step(root, dof, np.zeros(1), pos_target=[qt], vel_target=[vt])
        for sub in range(w.substeps):
            f = -c * qd + kp * (qt - q - h * qd) + kd * (vt - qd)
            if sub == w.substeps - 1:
                f_last = f
            qd = qd + h * f / (I + a + h * (h * kp + kd))
            q = q + h * qd
        assert abs(dof[0, 0] - q) < 1e-12 and abs(dof[0, 1] - qd) < 1e-12
        assert abs(out["dof_force"][0] - f_last) < 1e-10


def test_stiff_drive_settles_at_target():
    """kp = 1e4 with critical-ish damping: stable (implicit) and settles at q* (no other forces)."""
    w = W.homogeneous("driven", driven_joint(1e4, 150.0), 1, params=NOGRAV)
    O = oracle.Oracle(w)
    root = np.zeros((1, 13)); root[0, 6] = 1.0
    dof = np.array([[0.0, 0.0]])
    for _ in range(600):
        O.step(root, dof, np.zeros(1), pos_target=[0.5], vel_target=[0.0])
    assert abs(dof[0, 0] - 0.5) < 1e-6 and abs(dof[0, 1]) < 1e-6


def free_body(com=(0.05, -0.02, 0.03)):
    b = W._Builder("body")
    b.link(-1, W.JOINT_FREE, mass=2.0, com=com, inertia=(0.4, 0.4, 0.4, 0, 0, 0))
    return b.build()


def test_external_force_and_torque_on_a_free_body():
    """Zero gravity, isotropic inertia (no gyroscopic term): a force at the COM accelerates the COM
    by F/m and turns nothing (even with the COM away from the link origin); a torque changes the
    angular velocity by I^-1 tau dt."""
    w = W.homogeneous("body", free_body(), 1, params=NOGRAV)
    O = oracle.Oracle(w)
    root = np.zeros((1, 13)); root[0, 6] = 1.0; root[0, :3] = (0.3, 0.1, 2.0)
    F = np.array([1.5, -0.5, 2.0])
    O.step(root, np.zeros((0, 2)), np.zeros(0), body_force=np.concatenate([F, np.zeros(3)])[None])
    assert np.abs(root[0, 10:13]).max() < 1e-13
    assert np.allclose(root[0, 7:10], F / 2.0 * w.dt, atol=1e-13)  # origin moves with the COM when w = 0
    root2 = np.zeros((1, 13)); root2[0, 6] = 1.0
    tau = np.array([0.2, 0.0, -0.1])
    O2 = oracle.Oracle(w)
    O2.step(root2, np.zeros((0, 2)), np.zeros(0), body_force=np.concatenate([np.zeros(3), tau])[None])
    # I_com = 0.4 (isotropic) -> omega = tau dt / 0.4
    assert np.allclose(root2[0, 10:13], tau * w.dt / 0.4, rtol=1e-12, atol=1e-14)


def test_body_states_match_root_and_kinematics():
    w = W.ant_workload(3)
    O = oracle.Oracle(w)
    root, dof, acts = W.seeded_inputs(w, 0, 2)
    r, d = root.astype(np.float64), dof.astype(np.float64)
    O.step(r, d, acts[0])
    out = O.step(r, d, acts[1])
    bs = out["body_state"]
    m = w.models[0]
    nb = m.n_body
    for e in range(w.n_envs):
        b0 = bs[e * nb]
        assert np.allclose(b0[:3], r[e, :3], atol=1e-12)
        q = r[e, 3:7] * (1 if r[e, 6] >= 0 else -1)
        assert np.allclose(b0[3:7], q, atol=1e-12)
        assert np.allclose(b0[7:10], r[e, 7:10], atol=1e-12) and np.allclose(b0[10:13], r[e, 10:13], atol=1e-12)
        # every body: pose from forward kinematics, velocity by central differences of it
        de = d[e * 8:(e + 1) * 8]
        bodies = [l for l in range(m.n_links) if not m.is_virtual[l]]
        for k, l in enumerate(bodies):
            R, p = O.link_pose(e, r[e:e + 1], de, l)
            s = bs[e * nb + k]
            assert np.allclose(s[:3], p, atol=1e-12)
            x, y, z, ww = s[3:7]
            Rq = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * ww), 2 * (x * z + y * ww)],
                           [2 * (x * y + z * ww), 1 - 2 * (x * x + z * z), 2 * (y * z - x * ww)],
                           [2 * (x * z - y * ww), 2 * (y * z + x * ww), 1 - 2 * (x * x + y * y)]])
            assert np.allclose(Rq, R, atol=1e-12) and s[6] >= 0
            eps = 1e-6

            def pose(sgn):
                rr = r[e:e + 1].copy()
                om = rr[0, 10:13] * eps * sgn
                a = np.linalg.norm(om)
                dq = np.array([*(om / a * math.sin(a / 2)), math.cos(a / 2)]) if a > 0 else np.array([0, 0, 0, 1.0])
                qx, qy, qz, qw = rr[0, 3:7]
                ex, ey, ez, ew = dq
                rr[0, 3:7] = [ew * qx + ex * qw + ey * qz - ez * qy, ew * qy - ex * qz + ey * qw + ez * qx,
                              ew * qz + ex * qy - ey * qx + ez * qw, ew * qw - ex * qx - ey * qy - ez * qz]
                rr[0, :3] += rr[0, 7:10] * eps * sgn
                dd = de.copy()
                dd[:, 0] += dd[:, 1] * eps * sgn
                return O.link_pose(e, rr, dd, l)

            (Rp, pp), (Rm, pm) = pose(1), pose(-1)
            assert np.allclose((pp - pm) / (2 * eps), s[7:10], atol=1e-6)
            Om = (Rp - Rm) / (2 * eps) @ R.T
            assert np.allclose([Om[2, 1], Om[0, 2], Om[1, 0]], s[10:13], atol=1e-6)


def test_jacobian_columns_and_velocity():
    """Joint columns by central differences of forward kinematics; J nu equals the body velocities."""
    w = W.ant_workload(2)
    O = oracle.Oracle(w)
    root, dof, acts = W.seeded_inputs(w, 3, 1)
    r, d = root.astype(np.float64), dof.astype(np.float64)
    d[:, 1] = np.random.default_rng(0).uniform(-1, 1, d.shape[0])
    r[:, 7:13] = np.random.default_rng(1).uniform(-1, 1, (2, 6))
    m = w.models[0]
    e = 1
    de = d[8:16]
    nu = np.concatenate([r[e, 10:13], r[e, 7:10], de[:, 1]])  # [omega; p_dot; joint rates]
    for l in range(m.n_links):
        J = O.jacobian(e, r[e:e + 1], de, l)
        assert J.shape == (6, 14)
        R, p = O.link_pose(e, r[e:e + 1], de, l)
        for j in range(8):
            eps = 1e-6
            dp, dm = de.copy(), de.copy()
            dp[j, 0] += eps
            dm[j, 0] -= eps
            (Rp, pp), (Rm, pm) = O.link_pose(e, r[e:e + 1], dp, l), O.link_pose(e, r[e:e + 1], dm, l)
            col = J[:, 6 + j]
            assert np.allclose((pp - pm) / (2 * eps), col[3:], atol=1e-7)
            Om = (Rp - Rm) / (2 * eps) @ R.T
            assert np.allclose([Om[2, 1], Om[0, 2], Om[1, 0]], col[:3], atol=1e-7)
        # J nu: the link's velocity along the state's generalized velocity (central differences of
        # the pose with the root advanced by exp(eps omega), p + eps p_dot, q + eps q_dot)
        eps = 1e-6

        def pose(sgn):
            rr = r[e:e + 1].copy()
            om = rr[0, 10:13] * eps * sgn
            a = np.linalg.norm(om)
            ex, ey, ez, ew = (*(om / a * math.sin(a / 2)), math.cos(a / 2))
            qx, qy, qz, qw = rr[0, 3:7]
            rr[0, 3:7] = [ew * qx + ex * qw + ey * qz - ez * qy, ew * qy - ex * qz + ey * qw + ez * qx,
                          ew * qz + ex * qy - ey * qx + ez * qw, ew * qw - ex * qx - ey * qy - ez * qz]
            rr[0, :3] += rr[0, 7:10] * eps * sgn
            dd = de.copy()
            dd[:, 0] += dd[:, 1] * eps * sgn
            return O.link_pose(e, rr, dd, l)

        (Rp, pp), (Rm, pm) = pose(1), pose(-1)
        Jn = J @ nu
        assert np.allclose((pp - pm) / (2 * eps), Jn[3:], atol=1e-6)
        Om = (Rp - Rm) / (2 * eps) @ R.T
        assert np.allclose([Om[2, 1], Om[0, 2], Om[1, 0]], Jn[:3], atol=1e-6)
        # root columns: unit world angular velocity turns the link about the root origin
        for k in range(3):
            ek = np.eye(3)[k]
            assert np.allclose(J[:3, k], ek, atol=1e-12)
            assert np.allclose(J[3:, k], np.cross(ek, p - r[e, :3]), atol=1e-12)
            assert np.allclose(J[:3, 3 + k], 0, atol=1e-12) and np.allclose(J[3:, 3 + k], ek, atol=1e-12)
