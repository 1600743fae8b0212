"""Pins of the oracle's capsule-box contact geometry (the hand-and-cube workload) and of two-body
constraint rows: hand-derived cases, brute force over the segment and the box, finite-difference
Jacobians of both bodies, and a box resting on two fixed capsules."""
import math

import numpy as np
import pytest

import oracle
from paper_2108_10470_gb300 import workloads as W
from scenes import two_actor_env

E = np.array([0.1, 0.1, 0.1])


def test_parallel_capsule_above_face():
    """Capsule parallel to the top face, 1 cm above it: the endpoints are the contacts (normal +z,
    d = 0.03 - r), the closest point is not interior (the distance is constant, ties go to t = 0)."""
    ts, s = oracle.capsule_box([-0.05, 0, 0.13], [0.05, 0, 0.13], 0.02, E)
    assert ts == 0.0
    for k, xe in ((0, -0.05), (1, 0.05)):
        assert np.allclose(s[k]["n"], [0, 0, 1]) and abs(s[k]["d"] - 0.01) < 1e-15
        assert np.allclose(s[k]["x"], [xe, 0, 0.13 - 0.02 - 0.005], atol=1e-15)


def test_face_clip_by_hand():
    """A capsule along y over the top face (box half extents 0.1), from y = -0.2 to 0.2: the closest
    point's normal is +z, so the segment is clipped to |x| <= 0.1 and |y| <= 0.1, i.e. t in
    [0.25, 0.75]; both ends are supporting samples. Over an edge (normal along x) the clip is in y
    and z instead."""
    ts, s = oracle.capsule_box([0.03, -0.2, 0.13], [0.03, 0.2, 0.13], 0.02, E)
    assert s[3]["clip"] and abs(s[3]["ta"] - 0.25) < 1e-15 and abs(s[3]["tb"] - 0.75) < 1e-15
    assert abs(ts - 0.25) < 1e-15  # constant distance over the clip: the smallest t
    ts, s = oracle.capsule_box([0.05, 0, 0.2], [0.25, 0, 0.0], 0.01, E)  # normal (1, 0, 1)/sqrt 2: axis x
    assert s[3]["clip"] and abs(s[3]["ta"] - 0.5) < 1e-15 and s[3]["tb"] == 1.0
    _, s = oracle.capsule_box([0.3, 0.3, 0.3], [0.5, 0.3, 0.3], 0.01, E)  # off every slab
    assert not s[3]["clip"]


def test_capsule_over_an_edge():
    """Segment from (0.05, 0, 0.2) to (0.25, 0, 0) passes the box edge x = z = 0.1: by hand the
    closest point is t* = 0.375, p = (0.125, 0, 0.125), at distance 0.025 sqrt(2) along (1, 0, 1)/sqrt(2)."""
    ts, s = oracle.capsule_box([0.05, 0, 0.2], [0.25, 0, 0.0], 0.01, E)
    assert abs(ts - 0.375) < 1e-12
    assert np.allclose(s[2]["n"], np.array([1, 0, 1]) / math.sqrt(2), atol=1e-12)
    assert abs(s[2]["d"] - (0.025 * math.sqrt(2) - 0.01)) < 1e-12


def test_endpoint_inside_box():
    """An endpoint inside the box pushes out through the nearest face (z here: 0.01 away)."""
    _, s = oracle.capsule_box([0.02, 0.03, 0.09], [0.02, 0.03, 0.3], 0.02, E)
    assert np.allclose(s[0]["n"], [0, 0, 1])
    assert abs(s[0]["d"] - (-0.01 - 0.02)) < 1e-15


@pytest.mark.parametrize("seed", range(10))
def test_closest_point_brute_force(seed):
    """t* minimises the segment-box distance: no point of a 20001-sample grid of the segment is
    closer (to 1e-12), and each slot's separation equals the brute-force point-box distance - r."""
    rng = np.random.default_rng(seed)
    ext = rng.uniform(0.02, 0.2, 3)
    p0 = rng.uniform(-0.4, 0.4, 3)
    p1 = rng.uniform(-0.4, 0.4, 3)
    r = 0.03
    ts, s = oracle.capsule_box(p0, p1, r, ext)
    t = np.linspace(0, 1, 20001)
    pts = p0[None] + t[:, None] * (p1 - p0)[None]
    d2 = (np.maximum(np.abs(pts) - ext, 0.0) ** 2).sum(1)
    pt = p0 + ts * (p1 - p0)
    f = (np.maximum(np.abs(pt) - ext, 0.0) ** 2).sum()
    assert f <= d2.min() + 1e-12
    for k, tk in ((0, 0.0), (1, 1.0), (2, ts)):
        p = p0 + tk * (p1 - p0)
        out = np.maximum(np.abs(p) - ext, 0.0)
        if out.any():
            assert abs(s[k]["d"] - (np.linalg.norm(out) - r)) < 1e-12
        else:
            assert abs(s[k]["d"] - (-(ext - np.abs(p)).min() - r)) < 1e-12


def test_box_rests_on_two_capsules():
    """A box laid across two parallel horizontal capsules stays at rest; the pair contacts carry
    its weight (the capsules are 0.5 m up, so there is no ground contact)."""
    qy = W.Q_X_TO_Y
    w, root = two_actor_env([(-0.03, 0, 0.5), (0.03, 0, 0.5)], [qy, qy], (0, 0, 0.5 + 0.02 + 0.05))
    O = oracle.Oracle(w)
    out = None
    for _ in range(600):
        out = O.step(root, np.zeros((0, 2)), np.zeros(0))
    assert np.abs(root[1, 7:13]).max() < 1e-3
    assert abs(root[1, 2] - 0.57) < 1e-3
    assert out["n_contacts"][0] >= 2
    assert all(int(c[1]) == 2 for c in out["contacts"][0, :out["n_contacts"][0]])  # (capsule, box) pairs
    # net contact force on the box (body 1) balances gravity; the holder gets the opposite
    assert abs(out["net_force"][1, 2] - 0.2 * 9.81) < 0.01 * 0.2 * 9.81
    assert np.allclose(out["net_force"][0], -out["net_force"][1], atol=1e-9)


def test_two_body_jacobian_finite_difference():
    """Each pair row's J equals k . (x_dot_a - x_dot_b) of body-fixed points at the contact point,
    by central differences, with both bodies moving (hand finger and free cube)."""
    rng = np.random.default_rng(4)
    w = W.hand_workload(1)
    w.params = W.Params(contact_offset=0.5)
    O = oracle.Oracle(w)
    root, dof, _ = W.seeded_inputs(w, 0, 1)
    root = root.astype(np.float64)
    dof = dof.astype(np.float64)
    dof[:, 1] = rng.uniform(-1, 1, dof.shape[0])
    root[1, 7:13] = rng.uniform(-0.5, 0.5, 6)
    r = O.rows(0, root, dof, cap=400)
    nu = np.concatenate([dof[:, 1], root[1, 10:13], root[1, 7:10]])  # hand joints, then cube [w; v]

    def quat_exp(th):
        a = np.linalg.norm(th)
        return np.array([*(th / a * math.sin(a / 2)), math.cos(a / 2)]) if a > 1e-30 else np.array([*(th / 2), 1.0])

    def qmul(a, b):
        ax, ay, az, aw = a
        bx, by, bz, bw = b
        return np.array([aw * bx + ax * bw + ay * bz - az * by, aw * by - ax * bz + ay * bw + az * bx,
                         aw * bz + ax * by - ay * bx + az * bw, aw * bw - ax * bx - ay * by - az * bz])

    def moved(eps):
        rr, dd = root.copy(), dof.copy()
        rr[1, 0:3] += eps * root[1, 7:10]
        rr[1, 3:7] = qmul(quat_exp(eps * root[1, 10:13]), root[1, 3:7])
        dd[:, 0] += eps * dof[:, 1]
        return rr, dd

    hand_links = w.models[0].n_links
    checked = 0
    for i in range(len(r["kind"])):
        if r["kind"][i] == 0 or r["info"][i, 1] < 0:
            continue
        la, lb = int(r["link"][i]), hand_links  # body a on the hand, body b = the cube
        x = r["x"][i]
        locs = []
        for link in (la, lb):
            R0, p0 = O.link_pose(0, root, dof, link)
            locs.append(R0.T @ (x - p0))
        vel = []
        for eps in (1e-6, -1e-6):
            rr, dd = moved(eps)
            pts = []
            for link, xl in zip((la, lb), locs):
                R, p = O.link_pose(0, rr, dd, link)
                pts.append(p + R @ xl)
            vel.append(pts[0] - pts[1])
        fd = r["k"][i] @ (vel[0] - vel[1]) / 2e-6
        assert abs(r["J"][i] @ nu - fd) < 1e-7
        checked += 1
    assert checked >= 9
