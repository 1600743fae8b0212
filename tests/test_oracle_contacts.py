"""Pins of the FP64 oracle's contact generation, constraint rows and TGS-style solve (no GPU):
hand-derived iterates, closed-form motions (free fall, sliding, rolling), resting contact,
joint limits, brute-force geometry and finite-difference Jacobians."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2108_10470_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def one_env(model, params=None, dt=1.0 / 60.0, substeps=2):
    return W.homogeneous(model.name, model, 1, params=params or W.Params(), dt=dt, substeps=substeps)


def root_row(p=(0, 0, 0), q=(0, 0, 0, 1), v=(0, 0, 0), w=(0, 0, 0)):
    r = np.zeros((1, 13))
    r[0, 0:3], r[0, 3:7], r[0, 7:10], r[0, 10:13] = p, q, v, w
    return r


def run(O, root, dof, act, steps):
    out = None
    for _ in range(steps):
        out = O.step(root, dof, act)
    return out


def fnv1a32(data: bytes) -> int:
    h = 2166136261
    for b in data:
        h ^= b
        h = (h * 16777619) & 0xFFFFFFFF
    return h


def test_fnv1a_reference_vectors():
    """The signature hash is FNV-1a 32-bit; pin the reference implementation used below to the
    published test vectors (offset basis for the empty string, 'a', 'foobar')."""
    assert fnv1a32(b"") == 0x811C9DC5
    assert fnv1a32(b"a") == 0xE40C292C
    assert fnv1a32(b"foobar") == 0xBF9CF968


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "tgs_single_contact.json")))["cases"],
                         ids=lambda c: c["name"])
def test_tgs_single_contact_golden(case):
    """Hand-derived TGS iterates for one sphere-ground contact (tests/golden/tgs_single_contact.json)."""
    m = W.free_sphere(r=0.1, mass=1.0)
    O = oracle.Oracle(one_env(m, W.Params(gravity=(0, 0, 0)), dt=1.0 / 120.0, substeps=1))
    root = root_row(p=(0, 0, case["z0"]), v=(0, 0, case["vz0"]))
    dof = np.zeros((0, 2))
    out = O.step(root, dof, np.zeros(0))
    assert abs(root[0, 2] - case["z1"]) < 1e-12
    assert abs(root[0, 9] - case["vz1"]) < 1e-9
    assert np.allclose(root[0, 7:9], 0.0, atol=1e-12) and np.allclose(root[0, 10:13], 0.0, atol=1e-12)
    assert abs(out["net_force"][0, 2] * (1.0 / 120.0) - case["impulse"]) < 1e-9
    # the constraint-set signature covers: 0 limit rows, 1 contact (shape 0, ground, slot 0)
    seq = [0, 1, 0, -1, 0]
    assert int(out["signature"][0]) == fnv1a32(b"".join(int(v).to_bytes(4, "little", signed=True) for v in seq))


def test_free_fall_discrete_closed_form():
    """Contact-free substeps are symplectic Euler: z_n = z0 + v0 n h - g h^2 n (n+1) / 2 exactly."""
    m = W.free_sphere(r=0.1)
    w = one_env(m)
    O = oracle.Oracle(w)
    z0, vx, vz = 3.0, 0.3, 0.5
    root = root_row(p=(0, 0, z0), v=(vx, 0, vz), w=(0.2, -0.1, 0.4))
    h = w.dt / w.substeps
    for k in range(1, 21):
        O.step(root, np.zeros((0, 2)), np.zeros(0))
        n = k * w.substeps
        assert abs(root[0, 2] - (z0 + vz * n * h - 9.81 * h * h * n * (n + 1) / 2)) < 1e-12
        assert abs(root[0, 0] - vx * n * h) < 1e-12
        assert abs(root[0, 9] - (vz - 9.81 * n * h)) < 1e-12


def test_box_at_rest_1000_steps():
    """A box resting on the ground stays at rest for 1000 steps (|v| <= 1e-3 m/s, drift <= 1e-3 m)
    and the net contact force balances its weight (within 1 %)."""
    m = W.free_box(0.2, 0.1, 0.1, mass=2.0)
    O = oracle.Oracle(one_env(m))
    root = root_row(p=(0, 0, 0.1))
    out = run(O, root, np.zeros((0, 2)), np.zeros(0), 1000)
    assert np.abs(root[0, 7:13]).max() <= 1e-3
    assert np.abs(root[0, 0:3] - [0, 0, 0.1]).max() <= 1e-3
    assert abs(out["net_force"][0, 2] - 2.0 * 9.81) <= 0.01 * 2.0 * 9.81
    assert out["n_contacts"][0] == 4
    assert out["contacts"][0, :4].tolist() == [[0, -1, 0], [0, -1, 2], [0, -1, 4], [0, -1, 6]]


def test_sphere_drop_settles():
    """A sphere dropped from 0.5 m settles with its centre at z = r (within 1e-3)."""
    m = W.free_sphere(r=0.1)
    O = oracle.Oracle(one_env(m))
    root = root_row(p=(0, 0, 0.5))
    run(O, root, np.zeros((0, 2)), np.zeros(0), 300)
    assert abs(root[0, 2] - 0.1) <= 1e-3
    assert np.abs(root[0, 7:13]).max() <= 1e-3


def test_sliding_box_decelerates_at_mu_g():
    """A flat box (half extents 0.2, 0.2, 0.05: it would tip only for mu > 4) sliding at v0 on
    mu = 1 ground decelerates at mu g and stops after v0^2 / (2 mu g) (within O(h))."""
    m = W.free_box(0.2, 0.2, 0.05, mass=1.0)
    w = one_env(m)
    O = oracle.Oracle(w)
    v0 = 2.0
    root = root_row(p=(0, 0, 0.05), v=(v0, 0, 0))
    vs = []
    for _ in range(30):
        O.step(root, np.zeros((0, 2)), np.zeros(0))
        vs.append(root[0, 7])
    vs = np.array(vs)
    t = w.dt * np.arange(1, 31)
    sliding = vs > 0.2
    assert np.allclose(vs[sliding], v0 - 9.81 * t[sliding], atol=0.02)
    assert abs(root[0, 7]) < 1e-3
    assert abs(root[0, 0] - v0 * v0 / (2 * 9.81)) <= 3 * v0 * w.dt / w.substeps


def test_sphere_rolls_at_five_sevenths():
    """A uniform solid sphere launched with tangential velocity v0 and no spin ends up rolling
    without slipping at 5 v0 / 7."""
    m = W.free_sphere(r=0.1, mass=1.0)
    O = oracle.Oracle(one_env(m))
    v0 = 1.0
    root = root_row(p=(0, 0, 0.1), v=(v0, 0, 0))
    run(O, root, np.zeros((0, 2)), np.zeros(0), 120)
    assert abs(root[0, 7] - 5.0 * v0 / 7.0) <= 2e-3
    assert abs(root[0, 11] * 0.1 - root[0, 7]) <= 2e-3  # omega_y r = v_x


def test_joint_limit_holds_constant_torque():
    """A hinge about the vertical axis (no gravity torque) pushed by a constant torque into its
    upper limit stays within hi + 1e-3 and comes to rest there."""
    b = W._Builder("limited")
    b.link(-1, W.JOINT_FIXED, mass=1.0, inertia=(1, 1, 1, 0, 0, 0))
    b.link(0, W.JOINT_REVOLUTE, axis=(0, 0, 1), mass=1.0, com=(0.3, 0, 0), inertia=(0.01, 0.01, 0.01, 0, 0, 0),
           limit=(-0.5, 0.5))
    m = b.build()
    O = oracle.Oracle(one_env(m))
    root = root_row()
    dof = np.zeros((1, 2))
    qmax = -1.0
    for _ in range(300):
        O.step(root, dof, np.array([2.0]))
        qmax = max(qmax, dof[0, 0])
    assert qmax <= 0.5 + 1e-3
    assert abs(dof[0, 0] - 0.5) <= 1e-3 and abs(dof[0, 1]) <= 1e-3


def test_box_contact_points_by_hand():
    """Axis-aligned box (half extents 0.2, 0.1, 0.1) resting at z = 0.1: the four bottom vertices
    (slots k = 4[sx>0] + 2[sy>0] + [sz>0] with sz < 0) are the contacts, at the hand-listed points."""
    m = W.free_box(0.2, 0.1, 0.1)
    O = oracle.Oracle(one_env(m))
    r = O.rows(0, root_row(p=(0.5, -0.3, 0.1)), np.zeros((0, 2)))
    normals = r["kind"] == 1
    assert normals.sum() == 4 and (r["kind"] == 2).sum() == 8 and (r["kind"] == 0).sum() == 0
    expect = np.array([[-0.2, -0.1, 0.0], [-0.2, 0.1, 0.0], [0.2, -0.1, 0.0], [0.2, 0.1, 0.0]]) + [0.5, -0.3, 0.0]
    assert np.allclose(r["x"][normals], expect, atol=1e-15)
    assert np.allclose(r["d"][normals], 0.0, atol=1e-15)
    # row order: all normal rows, then per contact the x and y friction rows
    assert r["kind"].tolist() == [1] * 4 + [2] * 8
    assert np.allclose(r["k"][4:], np.tile([[1, 0, 0], [0, 1, 0]], (4, 1)))


def test_capsule_and_sphere_points_by_hand():
    """Capsule (axis = local x) rotated 30 degrees about y: endpoint 0 = centre - h axis, endpoint 1 =
    centre + h axis; each contact point sits one radius below its endpoint; only d < 0.02 is kept."""
    b = W._Builder("cap")
    rl = b.link(-1, W.JOINT_FREE, mass=1.0, inertia=(0.1, 0.1, 0.1, 0, 0, 0))
    b.shape(rl, W.SHAPE_CAPSULE, (0.05, 0.2))
    ang = math.radians(30)
    zb = -0.08 / math.cos(ang)  # body-frame sphere offset that puts its centre 0.08 below the root
    b.shape(rl, W.SHAPE_SPHERE, (0.07,), pos=(0.0, 0.3, zb))
    m = b.build()
    O = oracle.Oracle(one_env(m))
    q = (0.0, math.sin(ang / 2), 0.0, math.cos(ang / 2))
    c = np.array([0.0, 0.0, 0.2 * math.sin(ang) + 0.05 + 0.01])  # low capsule end 0.01 above ground
    r = O.rows(0, root_row(p=tuple(c), q=q), np.zeros((0, 2)))
    normals = r["kind"] == 1
    # rotation about +y by ang maps (x, z) -> (x cos + z sin, -x sin + z cos)
    axis = np.array([math.cos(ang), 0.0, -math.sin(ang)])
    e1 = c + 0.2 * axis  # the low endpoint is centre + h axis (slot 1); slot 0 is 0.21 m higher
    sc = c + np.array([zb * math.sin(ang), 0.3, zb * math.cos(ang)])  # sphere centre, z = 0.08
    assert normals.sum() == 2  # capsule slot 1 (d = 0.01) then the sphere (d = 0.08 - 0.07 = 0.01)
    assert np.allclose(r["x"][normals][0], e1 - [0, 0, 0.05], atol=1e-14)
    assert np.allclose(r["d"][normals], [0.01, 0.01], atol=1e-14)
    assert np.allclose(r["x"][normals][1], sc - [0, 0, 0.07], atol=1e-14)


def test_capsule_distance_brute_force():
    """Lowest point of a randomly posed capsule found by brute-force sampling of its surface (1e5
    samples) agrees with the oracle's endpoint rule: min separation = min endpoint z - r."""
    rng = np.random.default_rng(5)
    b = W._Builder("cap")
    rl = b.link(-1, W.JOINT_FREE, mass=1.0, inertia=(0.1, 0.1, 0.1, 0, 0, 0))
    b.shape(rl, W.SHAPE_CAPSULE, (0.05, 0.2))
    m = b.build()
    O = oracle.Oracle(one_env(m, W.Params(contact_offset=10.0)))
    for _ in range(5):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        p = np.array([0.0, 0.0, 0.3])
        r = O.rows(0, root_row(p=tuple(p), q=tuple(q)), np.zeros((0, 2)))
        dmin = r["d"][r["kind"] == 1].min()
        Rm, _ = O.link_pose(0, root_row(p=tuple(p), q=tuple(q)), np.zeros((0, 2)), 0)
        ax = Rm[:, 0]
        t = rng.uniform(-0.2, 0.2, 100000)
        dirs = rng.normal(size=(100000, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        pts = p + t[:, None] * ax + 0.05 * dirs
        assert dmin <= pts[:, 2].min() + 1e-12
        assert pts[:, 2].min() - dmin < 2e-3


def test_contact_jacobian_finite_difference():
    """Each contact row J satisfies J nu = k . d/dt x(t) for the body-fixed contact point, checked
    by central differences of forward kinematics along the generalized velocity (root: p + eps v,
    quat <- exp(eps omega) quat; joints: q + eps qd)."""
    rng = np.random.default_rng(9)
    m = W.ant()
    O = oracle.Oracle(one_env(m, W.Params(contact_offset=5.0)))
    root = root_row(p=(0.1, -0.2, 0.3), q=tuple(np.array([0.1, -0.05, 0.2, 0.97]) / np.linalg.norm([0.1, -0.05, 0.2, 0.97])),
                    v=tuple(rng.uniform(-1, 1, 3)), w=tuple(rng.uniform(-1, 1, 3)))
    dof = np.zeros((8, 2))
    dof[:, 0] = rng.uniform(-0.4, 0.4, 8)
    dof[:, 1] = rng.uniform(-1, 1, 8)
    r = O.rows(0, root, dof)
    nu = np.concatenate([root[0, 10:13], root[0, 7:10], dof[:, 1]])

    def quat_exp(th):
        a = np.linalg.norm(th)
        if a < 1e-30:
            return np.array([*(th / 2), 1.0])
        return np.array([*(th / a * math.sin(a / 2)), math.cos(a / 2)])

    def qmul(a, b):
        ax, ay, az, aw = a
        bx, by, bz, bw = b
        return np.array([aw * bx + ax * bw + ay * bz - az * by, aw * by - ax * bz + ay * bw + az * bx,
                         aw * bz + ax * by - ay * bx + az * bw, aw * bw - ax * bx - ay * by - az * bz])

    def moved(eps):
        rr = root.copy()
        rr[0, 0:3] += eps * root[0, 7:10]
        rr[0, 3:7] = qmul(quat_exp(eps * root[0, 10:13]), root[0, 3:7])
        dd = dof.copy()
        dd[:, 0] += eps * dof[:, 1]
        return rr, dd

    checked = 0
    for i in range(len(r["kind"])):
        if r["kind"][i] == 0:
            continue
        link = int(r["link"][i])
        R0, p0 = O.link_pose(0, root, dof, link)
        xl = R0.T @ (r["x"][i] - p0)
        eps = 1e-6
        xs = []
        for e in (eps, -eps):
            rr, dd = moved(e)
            R, p = O.link_pose(0, rr, dd, link)
            xs.append(p + R @ xl)
        fd = r["k"][i] @ (xs[0] - xs[1]) / (2 * eps)
        assert abs(r["J"][i] @ nu - fd) < 1e-8
        checked += 1
    assert checked >= 9 * 3


def test_limit_rows_by_hand():
    """Limit rows appear when q - lo < margin (J = +e_j, d = q - lo) or hi - q < margin
    (J = -e_j, d = hi - q), DOF ascending, before the contact rows."""
    m = W.ant()
    O = oracle.Oracle(one_env(m, W.Params(contact_offset=-1.0)))
    dof = np.zeros((8, 2))
    dof[1, 0] = math.radians(70) - 0.05   # near hi of DOF 1 (knee)
    dof[4, 0] = -math.radians(30) + 0.02  # near lo of DOF 4 (hip)
    r = O.rows(0, root_row(p=(0, 0, 1.0)), dof)
    assert r["kind"].tolist() == [0, 0]
    assert np.allclose(r["d"], [0.05, 0.02], atol=1e-12)
    assert r["J"][0, 6 + 1] == -1.0 and r["J"][1, 6 + 4] == 1.0
    assert np.count_nonzero(r["J"]) == 2


def test_contact_signature_is_fnv1a_of_constraint_set():
    """The per-env signature of a step equals FNV-1a over, per substep: limit-row count, (DOF,
    side) pairs, contact count, (shape_a, shape_b, slot) triples."""
    m = W.free_box(0.1, 0.1, 0.1)
    w = one_env(m)
    O = oracle.Oracle(w)
    out = O.step(root_row(p=(0, 0, 0.1)), np.zeros((0, 2)), np.zeros(0))
    seq = []
    for _ in range(w.substeps):
        seq += [0, 4] + [0, -1, 0, 0, -1, 2, 0, -1, 4, 0, -1, 6]
    assert int(out["signature"][0]) == fnv1a32(b"".join(int(v).to_bytes(4, "little", signed=True) for v in seq))


def test_contact_free_step_is_symplectic_euler():
    """With no active rows the TGS solve returns Delta q = h v_free and qd = v_free: one substep of
    the Ant in the air equals q + h (qd + h qdd_ABA), qd + h qdd_ABA."""
    m = W.ant(damping=0.0)
    w = one_env(m, W.Params(contact_offset=-10.0, limit_margin=-10.0), substeps=1)
    O = oracle.Oracle(w)
    rng = np.random.default_rng(2)
    root = root_row(p=(0, 0, 2.0), v=(0.1, 0.2, 0.0), w=(0.0, 0.0, 0.0))
    dof = np.zeros((8, 2))
    dof[:, 0] = rng.uniform(-0.3, 0.3, 8)
    dof[:, 1] = rng.uniform(-1, 1, 8)
    act = rng.uniform(-5, 5, 8)
    tau = np.concatenate([np.zeros(6), act])
    qdd = O.aba(0, root, dof, tau)
    q0, qd0 = dof[:, 0].copy(), dof[:, 1].copy()
    O.step(root, dof, act)
    h = w.dt
    vnew = qd0 + h * qdd[6:]
    assert np.allclose(dof[:, 1], vnew, atol=1e-13)
    assert np.allclose(dof[:, 0], q0 + h * vnew, atol=1e-13)
