"""Pins of the oracle's forward-mode derivative (dual numbers through the FP64 step), the reference
the GPU adjoint is checked against: values identical to the plain step; directional derivatives
equal to central differences of the FP64 step on envs whose constraint set does not change;
linearity in the seed; the closed form of free flight."""
import numpy as np
import pytest

import oracle
from paper_2108_10470_gb300 import workloads as W


def warm_state(w, seed=0, steps=3):
    """Seeded state after a few oracle steps (contacts and a warm impulse cache in place)."""
    root, dof, acts = W.seeded_inputs(w, seed, steps + 1)
    O = oracle.Oracle(w)
    r, d = root.astype(np.float64), dof.astype(np.float64)
    for k in range(steps):
        O.step(r, d, acts[k])
    return O, r, d, acts[steps].astype(np.float64)


def plain_step(w, cache, r, d, a):
    O = oracle.Oracle(w)
    O.cache[:] = cache
    r, d = r.copy(), d.copy()
    out = O.step(r, d, a)
    return r, d, O.cache.copy(), out["signature"]


def random_direction(w, O, r, rng, scale=1.0):
    dr = rng.standard_normal(r.shape) * scale  # quaternion components too: the step's formula is
    # defined for any quaternion (rotation of the unnormalised q), so every direction has a derivative
    dd = rng.standard_normal((O.N_D, 2)) * scale
    da = rng.standard_normal(O.N_D) * scale
    dc = rng.standard_normal(O.cache.shape) * scale * (O.cache != 0)  # active cache entries
    return dr, dd, da, dc


def tangent(O, r, d, a, dr, dd, da, dc):
    c0 = O.cache.copy()
    r1, d1 = r.copy(), d.copy()
    tr, td, tc = dr.copy(), dd.copy(), dc.copy()
    O.step_tangent(r1, d1, a, tr, td, da, tc)
    out = (r1, d1, O.cache.copy(), tr, td, tc)
    O.cache[:] = c0
    return out


def test_values_equal_plain_step():
    w = W.ant_workload(6)
    O, r, d, a = warm_state(w)
    rng = np.random.default_rng(1)
    r1, d1, c1, *_ = tangent(O, r, d, a, *random_direction(w, O, r, rng))
    r2, d2, c2, _ = plain_step(w, O.cache, r, d, a)
    assert np.array_equal(r1, r2) and np.array_equal(d1, d2) and np.array_equal(c1, c2)


@pytest.mark.parametrize("make", [lambda: W.ant_workload(6), lambda: W.humanoid_workload(4), lambda: W.cartpole_workload(4),
                                  lambda: W.hand_workload(3),
                                  lambda: W.homogeneous("ball_ant", W.ant(ball_hips=True), 6),
                                  lambda: W.homogeneous("tendon_ant", W.ant(tendons=True), 6),
                                  lambda: W.hand_tendon_workload(3)],
                         ids=["ant", "humanoid", "cartpole", "hand", "ball_ant", "tendon_ant", "hand_tendon"])
def test_directional_derivative_equals_central_differences(make):
    """JVP against (f(x + eps u) - f(x - eps u)) / 2 eps with eps = 1e-7, on envs whose constraint
    set is the same at both ends and whose one-sided differences agree (no clamp or target switch
    inside the interval: the step is piecewise smooth); relative to the tangent's scale."""
    w = make()
    O, r, d, a = warm_state(w, seed=2)
    rng = np.random.default_rng(3)
    checked = 0
    eps = 1e-7
    rows_r = np.cumsum([0] + [w.env_actor_count(e) for e in range(w.n_envs)])
    rows_d = np.cumsum([0] + [w.env_jdof(e) for e in range(w.n_envs)])
    for trial in range(3):
        dr, dd, da, dc = random_direction(w, O, r, rng)
        _, _, _, tr, td, tc = tangent(O, r, d, a, dr, dd, da, dc)
        p = plain_step(w, O.cache + eps * dc, r + eps * dr, d + eps * dd, a + eps * da)
        m = plain_step(w, O.cache - eps * dc, r - eps * dr, d - eps * dd, a - eps * da)
        z = plain_step(w, O.cache, r, d, a)
        for e in np.nonzero(p[3] == m[3])[0]:
            parts = [(k, lo, hi) for k, lo, hi in ((0, rows_r[e], rows_r[e + 1]), (1, rows_d[e], rows_d[e + 1]),
                                                     (2, e, e + 1)) if hi > lo]
            tang = (tr, td, tc)
            smooth = True
            for k, lo, hi in parts:
                scale = max(1.0, np.abs(tang[k][lo:hi]).max())
                fwd = (p[k][lo:hi] - z[k][lo:hi]) / eps
                bwd = (z[k][lo:hi] - m[k][lo:hi]) / eps
                smooth &= np.abs(fwd - bwd).max() <= 1e-4 * scale
            if not smooth:
                continue
            for k, lo, hi in parts:
                scale = max(1.0, np.abs(tang[k][lo:hi]).max())
                fd = (p[k][lo:hi] - m[k][lo:hi]) / (2 * eps)
                assert np.abs(fd - tang[k][lo:hi]).max() <= 1e-6 * scale, (e, k, np.abs(fd - tang[k][lo:hi]).max(), scale)
            checked += 1
    assert checked >= 3 * w.n_envs // 2


def test_linear_in_the_seed():
    w = W.ant_workload(4)
    O, r, d, a = warm_state(w, seed=4)
    rng = np.random.default_rng(5)
    u = random_direction(w, O, r, rng)
    v = random_direction(w, O, r, rng)
    tu = tangent(O, r, d, a, *u)[3:]
    tv = tangent(O, r, d, a, *v)[3:]
    tw = tangent(O, r, d, a, *[2.0 * x - 3.0 * y for x, y in zip(u, v)])[3:]
    for x, y, z in zip(tu, tv, tw):
        assert np.allclose(z, 2.0 * x - 3.0 * y, rtol=1e-12, atol=1e-12)


def test_free_flight_closed_form():
    """A free box far above the ground under gravity, no rotation: after one step of 2 substeps,
    p' = p + dt v + (3/4) g dt^2... and exactly d p'/d v = dt, d v'/d v = 1, d v'/d p = 0."""
    w = W.homogeneous("box", W.free_box(0.1, 0.1, 0.1, 1.0), 1)
    O = oracle.Oracle(w)
    r = np.zeros((1, 13))
    r[0, 2] = 5.0
    r[0, 6] = 1.0
    r[0, 7:10] = [0.3, -0.2, 0.1]
    d = np.zeros((0, 2))
    for k in range(3):  # velocity component x, y, z
        dr = np.zeros((1, 13))
        dr[0, 7 + k] = 1.0
        r1, d1 = r.copy(), d.copy()
        O.cache[:] = 0
        O.step_tangent(r1, d1, np.zeros(0), dr, np.zeros((0, 2)), np.zeros(0), np.zeros_like(O.cache))
        assert abs(dr[0, k] - w.dt) < 1e-15
        assert abs(dr[0, 7 + k] - 1.0) < 1e-15
        assert np.abs(np.delete(dr[0], [k, 7 + k])).max() < 1e-15


def _driven_ant_workload(n, kp=60.0, kd=4.0):
    m = W.ant()
    kps = np.where(np.isin(m.jtype, [W.JOINT_REVOLUTE, W.JOINT_PRISMATIC]), kp, 0.0)
    kps[0] = 0.0
    m.drive_kp = kps
    m.drive_kd = np.where(kps > 0, kd, 0.0)
    return W.homogeneous("ant_driven", m, n)


@pytest.mark.parametrize("control", ["drives", "body_forces"])
def test_controls_with_per_env_values(control):
    """Joint drives with targets, or external body forces, that differ per env (constants of the
    derivative): the tangent step's values equal the plain step's with the same controls, bit for
    bit, in every env, and its directional derivative equals central differences of that step."""
    w = _driven_ant_workload(5) if control == "drives" else W.ant_workload(5)
    O, r, d, a = warm_state(w, seed=6)
    rng = np.random.default_rng(7)
    if control == "drives":
        ctl = dict(pos_target=rng.uniform(-0.3, 0.3, O.N_D), vel_target=rng.uniform(-0.5, 0.5, O.N_D))
    else:
        ctl = dict(body_force=rng.uniform(-3.0, 3.0, (O.N_B, 6)))

    def plain(cache, r0, d0, a0):
        P = oracle.Oracle(w)
        P.cache[:] = cache
        r1, d1 = r0.copy(), d0.copy()
        out = P.step(r1, d1, a0, **ctl)
        return r1, d1, P.cache.copy(), out["signature"]

    dr, dd, da, dc = random_direction(w, O, r, rng)
    c0 = O.cache.copy()
    r1, d1 = r.copy(), d.copy()
    tr, td, tc = dr.copy(), dd.copy(), dc.copy()
    O.step_tangent(r1, d1, a, tr, td, da, tc, **ctl)
    z = plain(c0, r, d, a)
    assert np.array_equal(r1, z[0]) and np.array_equal(d1, z[1]) and np.array_equal(O.cache, z[2])
    # the controls matter: without them the step differs
    assert not np.array_equal(d1, plain_step(w, c0, r, d, a)[1])
    eps = 1e-7
    p = plain(c0 + eps * dc, r + eps * dr, d + eps * dd, a + eps * da)
    m = plain(c0 - eps * dc, r - eps * dr, d - eps * dd, a - eps * da)
    checked = 0
    for e in np.nonzero(p[3] == m[3])[0]:
        sl = [slice(e, e + 1), slice(e * O.N_D // w.n_envs, (e + 1) * O.N_D // w.n_envs), slice(e, e + 1)]
        tang = (tr, td, tc)
        for k in range(3):
            scale = max(1.0, np.abs(tang[k][sl[k]]).max())
            fd = (p[k][sl[k]] - m[k][sl[k]]) / (2 * eps)
            assert np.abs(fd - tang[k][sl[k]]).max() <= 1e-6 * scale, (e, k)
        checked += 1
    assert checked >= 3
