"""Pins of the FP64 oracle's rigid-body dynamics against closed forms, invariants and independent
algorithms (no GPU). Each test names what it pins and the textbook fact that fixes it."""
import math

import numpy as np
import pytest

import oracle
from paper_2108_10470_gb300 import workloads as W


def one_env(model, params=None, dt=1.0 / 60.0, substeps=2):
    return W.homogeneous(model.name, model, 1, params=params or W.Params(), dt=dt, substeps=substeps)


def rand_quat(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def random_state(rng, m):
    root = np.zeros((1, 13))
    root[0, 0:3] = rng.uniform(-1, 1, 3)
    root[0, 3:7] = rand_quat(rng) if m.free_root else (0, 0, 0, 1)
    if m.free_root:
        root[0, 7:10] = rng.uniform(-1, 1, 3)
        root[0, 10:13] = rng.uniform(-2, 2, 3)
    dof = np.zeros((m.n_jdof, 2))
    dof[:, 0] = rng.uniform(-1.5, 1.5, m.n_jdof)
    dof[:, 1] = rng.uniform(-2.0, 2.0, m.n_jdof)
    return root, dof


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("floating", [False, True])
def test_aba_matches_crba_rnea_random_trees(seed, floating):
    """ABA (RBDA Table 7.1) against CRBA (Table 6.2) + RNEA (Table 5.1) on random trees of up to 8
    links with mixed revolute / prismatic / fixed joints: H(q) qdd = tau - C(q, qd) to 1e-10."""
    rng = np.random.default_rng(1000 * seed + floating)
    n_links = int(rng.integers(1 if floating else 2, 9))
    m = W.random_tree(rng, n_links, floating)
    O = oracle.Oracle(one_env(m))
    n = O.ngen()
    if n == 0:
        pytest.skip("tree without DOFs")
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
    # RNEA inverts ABA
    assert np.allclose(O.rnea(0, root, dof, qdd), tau, rtol=0, atol=1e-10 * scale)


def test_free_body_euler_equations():
    """A single torque-free body with COM at its origin: omega_dot_body = I^-1 (-w x I w) (Euler's
    equations) and the root-origin spatial acceleration's linear part is -omega x v."""
    rng = np.random.default_rng(7)
    b = W._Builder("rigid")
    b.link(-1, W.JOINT_FREE, mass=2.0, inertia=(1.0, 2.0, 3.0, 0, 0, 0))
    m = b.build()
    O = oracle.Oracle(one_env(m, W.Params(gravity=(0, 0, 0))))
    for _ in range(5):
        q = rand_quat(rng)
        w = rng.uniform(-3, 3, 3)
        v = rng.uniform(-1, 1, 3)
        root = np.zeros((1, 13))
        root[0, 3:7] = q
        root[0, 7:10] = v
        root[0, 10:13] = w
        qdd = O.aba(0, root, np.zeros((0, 2)), np.zeros(6))
        x, y, z, s = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * s), 2 * (x * z + y * s)],
                      [2 * (x * y + z * s), 1 - 2 * (x * x + z * z), 2 * (y * z - x * s)],
                      [2 * (x * z - y * s), 2 * (y * z + x * s), 1 - 2 * (x * x + y * y)]])
        Ib = np.diag([1.0, 2.0, 3.0])
        wb = R.T @ w
        wdot = R @ np.linalg.solve(Ib, -np.cross(wb, Ib @ wb))
        assert np.allclose(qdd[:3], wdot, atol=1e-12)
        assert np.allclose(qdd[3:], -np.cross(w, v), atol=1e-12)


def test_gravity_free_fall_acceleration():
    """Uniform gravity accelerates every free body's COM by g: a single body with COM offset c
    from its origin has a root-origin spatial acceleration [0; g - w x v] only when w = 0; with
    w = 0 the linear part is exactly g."""
    b = W._Builder("rigid")
    b.link(-1, W.JOINT_FREE, mass=1.5, com=(0.1, -0.2, 0.05), inertia=(0.3, 0.2, 0.25, 0.01, 0.0, 0.02))
    O = oracle.Oracle(one_env(b.build()))
    root = np.zeros((1, 13))
    root[0, 3:7] = (0.2, 0.1, -0.3, 0.9)
    root[0, 3:7] /= np.linalg.norm(root[0, 3:7])
    root[0, 7:10] = (0.4, -0.2, 1.0)
    qdd = O.aba(0, root, np.zeros((0, 2)), np.zeros(6))
    assert np.allclose(qdd, [0, 0, 0, 0, 0, -9.81], atol=1e-12)


def test_free_flight_momentum_conserved():
    """Free flight (g = 0) of the floating Ant under random internal joint torques: the total
    spatial momentum's rate from the ABA accelerations is zero (internal forces cancel)."""
    rng = np.random.default_rng(3)
    m = W.ant()
    O = oracle.Oracle(one_env(m, W.Params(gravity=(0, 0, 0))))
    for _ in range(5):
        root, dof = random_state(rng, m)
        tau = np.zeros(O.ngen())
        tau[6:] = rng.uniform(-15, 15, m.n_jdof)
        qdd = O.aba(0, root, dof, tau)
        h, hdot = O.momentum(0, root, dof, qdd)
        scale = np.abs(tau).max()
        assert np.abs(hdot).max() <= 1e-10 * scale


def test_free_flight_momentum_rk4_drift():
    """1000 RK4 steps of the free-flying Ant with constant internal torques conserve the total
    spatial momentum to 1e-8 relative."""
    rng = np.random.default_rng(4)
    m = W.ant(damping=0.0)
    w = one_env(m, W.Params(gravity=(0, 0, 0)))
    O = oracle.Oracle(w)
    root, dof = random_state(rng, m)
    dof[:, 0] = rng.uniform(-0.3, 0.3, m.n_jdof)
    act = rng.uniform(-0.5, 0.5, m.n_jdof)
    h0, _ = O.momentum(0, root, dof, np.zeros(O.ngen()))
    O.rk4(root, dof, act, 1.0 / 1200.0, 1000)
    h1, _ = O.momentum(0, root, dof, np.zeros(O.ngen()))
    assert np.abs(h1 - h0).max() <= 1e-8 * np.abs(h0).max()


@pytest.mark.parametrize("model_name", ["pendulum", "cartpole_hanging", "random_tree"])
def test_energy_rk4_1000_steps(model_name):
    """Undamped, contact-free, unactuated motion conserves T + V: 1000 RK4 steps at h = 1/1200
    drift by at most 1e-6 relative."""
    rng = np.random.default_rng(11)
    if model_name == "pendulum":
        m = W.pendulum()
    elif model_name == "cartpole_hanging":
        m = W.cartpole(hanging=True)
    else:
        m = W.random_tree(rng, 6, False, allow_fixed=True)
        m.damping[:] = 0.0
    O = oracle.Oracle(one_env(m))
    root = np.zeros((1, 13))
    root[0, 6] = 1.0
    dof = np.zeros((m.n_jdof, 2))
    dof[:, 0] = rng.uniform(-1.0, 1.0, m.n_jdof)
    dof[:, 1] = rng.uniform(-1.0, 1.0, m.n_jdof)
    e0 = O.energy(0, root, dof).sum()
    ke0 = O.energy(0, root, dof)[0]
    O.rk4(root, dof, np.zeros(m.n_jdof), 1.0 / 1200.0, 1000)
    e1 = O.energy(0, root, dof).sum()
    scale = max(abs(e0), ke0, 1e-3)
    assert abs(e1 - e0) <= 1e-6 * scale


def _period_from_crossings(t, x):
    s = np.sign(x)
    idx = np.where((s[:-1] < 0) & (s[1:] >= 0))[0]
    tc = [t[i] - x[i] * (t[i + 1] - t[i]) / (x[i + 1] - x[i]) for i in idx]
    return np.diff(tc).mean()


def _simulate(model, q0, n_steps, dof_index, params=None):
    w = one_env(model, params)
    O = oracle.Oracle(w)
    root = np.zeros((1, 13))
    root[0, 6] = 1.0
    dof = np.zeros((model.n_jdof, 2))
    dof[dof_index, 0] = q0
    act = np.zeros(model.n_jdof)
    ts, xs = [0.0], [q0]
    for k in range(n_steps):
        O.step(root, dof, act)
        ts.append((k + 1) * w.dt)
        xs.append(dof[dof_index, 0])
    return np.array(ts), np.array(xs)


def test_pendulum_small_angle_period():
    """Production step (TGS, no contacts = symplectic Euler at h = 1/120): a 0.5 kg uniform 1 m rod
    pivoted at its end has T = 2 pi sqrt(2 L / 3 g) = 1.63795 s for small amplitude (0.01 rad)."""
    t, x = _simulate(W.pendulum(), 0.01, 600, 0)
    T = _period_from_crossings(t, x)
    assert abs(T - 2 * math.pi * math.sqrt(2.0 / (3 * 9.81))) <= 1e-3 * 1.63795


def test_free_cartpole_period():
    """Free hanging cartpole (cart 1 kg, pole 0.5 kg, l = 0.5 m, I_c = m L^2 / 12): small
    oscillations have omega^2 = m l g (M+m) / ((M+m)(I_c + m l^2) - m^2 l^2) -> T = 1.41850 s."""
    M, m, l, g = 1.0, 0.5, 0.5, 9.81
    Ic = m * 1.0 / 12.0
    w2 = m * l * g * (M + m) / ((M + m) * (Ic + m * l * l) - m * m * l * l)
    t, x = _simulate(W.cartpole(hanging=True), 0.01, 600, 1)
    T = _period_from_crossings(t, x)
    assert abs(T - 2 * math.pi / math.sqrt(w2)) <= 1e-3 * T


def test_production_energy_band_scales_with_h():
    """The first-order production step keeps the pendulum's energy in a bounded band (no secular
    drift) whose width shrinks in proportion to h."""
    def band(substeps):
        w = one_env(W.pendulum(), substeps=substeps)
        O = oracle.Oracle(w)
        root = np.zeros((1, 13)); root[0, 6] = 1.0
        dof = np.array([[0.5, 0.0]])
        es = []
        for _ in range(600):
            O.step(root, dof, np.zeros(1))
            es.append(O.energy(0, root, dof).sum())
        es = np.array(es)
        return es.max() - es.min(), abs(es[-100:].mean() - es[:100].mean())
    b2, d2 = band(2)
    b4, d4 = band(4)
    assert 1.6 < b2 / b4 < 2.4
    assert d2 < 0.1 * b2 and d4 < 0.1 * b4


def test_op_count_positive_and_deterministic():
    w = W.ant_workload(4)
    O = oracle.Oracle(w)
    root, dof, act = W.seeded_inputs(w, 0, 1)
    r1, d1 = root.astype(np.float64), dof.astype(np.float64)
    r2, d2 = r1.copy(), d1.copy()
    f1 = O.step_flops(r1, d1, act[0])
    O.cache[:] = 0.0  # same cold impulse cache for every run
    f2 = O.step_flops(r2, d2, act[0])
    assert f1 == f2 and f1 > 1e4
    # the counting scalar computes the same values as the double path
    r3, d3 = root.astype(np.float64), dof.astype(np.float64)
    O.cache[:] = 0.0
    O.step(r3, d3, act[0])
    assert np.array_equal(r1, r3) and np.array_equal(d1, d3)
