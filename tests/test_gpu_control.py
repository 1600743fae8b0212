"""Control inputs and extra outputs on the GPU against the FP64 oracle: joint drives with position
and velocity targets, external body forces and torques, the joint-force and rigid-body-state
views, and the mass-matrix and Jacobian queries."""
import numpy as np
import pytest

import oracle
from paper_2108_10470_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10470_gb300 import build
    build.build_library()
    torch.cuda.set_device(0)


def driven_ant(kp=60.0, kd=4.0):
    m = W.ant()
    kps = np.where(np.isin(m.jtype, [W.JOINT_REVOLUTE, W.JOINT_PRISMATIC]), kp, 0.0)
    kps[0] = 0.0
    m.drive_kp = kps
    m.drive_kd = np.where(kps > 0, kd, 0.0)
    return m


def rollout_both(w, steps, flags, extra, seed=0):
    """GPU and oracle over `steps` steps with the same seeded inputs and per-step extras."""
    import torch
    from paper_2108_10470_gb300 import sim
    root, dof, acts = W.seeded_inputs(w, seed, steps)
    s = sim.Sim(w, flags=flags)
    s.root_state.copy_(torch.from_numpy(root))
    s.dof_state.copy_(torch.from_numpy(dof))
    O = oracle.Oracle(w)
    r, d = root.astype(np.float64), dof.astype(np.float64)
    g_out, o_out = [], []
    for k in range(steps):
        ex = extra(k)
        s.dof_actuation.copy_(torch.from_numpy(acts[k]))
        if "pos_target" in ex:
            s.dof_position_target.copy_(torch.from_numpy(ex["pos_target"].astype(np.float32)))
            s.dof_velocity_target.copy_(torch.from_numpy(ex["vel_target"].astype(np.float32)))
        if "body_force" in ex:
            s.rigid_body_force.copy_(torch.from_numpy(ex["body_force"].astype(np.float32)))
        s.step()
        torch.cuda.synchronize()
        g_out.append(dict(root=s.root_state.cpu().numpy().astype(np.float64), dof=s.dof_state.cpu().numpy().astype(np.float64),
                          dof_force=s.dof_force.cpu().numpy().astype(np.float64),
                          body=s.rigid_body_state.cpu().numpy().astype(np.float64),
                          sig=s.signature.cpu().numpy().astype(np.uint32)))
        out = O.step(r, d, acts[k], **ex)
        o_out.append(dict(root=r.copy(), dof=d.copy(), dof_force=out["dof_force"], body=out["body_state"],
                          sig=out["signature"]))
    s.destroy()
    return g_out, o_out


def within(a, b, rtol, atol, frac=0.98):
    ok = np.abs(a - b) <= atol + rtol * np.abs(b)
    return ok.mean() >= frac, ok.mean()


def test_drives_track_targets_and_match_oracle():
    from paper_2108_10470_gb300 import sim
    w = W.homogeneous("ant_driven", driven_ant(), 37)
    rng = np.random.default_rng(5)
    targets = [dict(pos_target=rng.uniform(-0.3, 0.3, w.n_dof), vel_target=rng.uniform(-0.5, 0.5, w.n_dof))
               for _ in range(4)]
    flags = sim.SIM_FLAG_SIGNATURE | sim.SIM_FLAG_DOF_FORCE | sim.SIM_FLAG_RIGID_BODY_STATE
    g, o = rollout_both(w, 4, flags, lambda k: targets[k])
    same = np.ones(w.n_envs, bool)
    for k in range(4):
        same &= g[k]["sig"] == o[k]["sig"]
    assert same.mean() >= 0.9
    m = w.models[0]
    dmask = np.repeat(same, m.n_jdof)
    bmask = np.repeat(same, m.n_body)
    ok, f = within(g[0]["dof"][dmask], o[0]["dof"][dmask], 1e-4, 1e-5)
    assert ok, f
    ok, f = within(g[0]["dof_force"][dmask], o[0]["dof_force"][dmask], 1e-4, 1e-4)
    assert ok, f
    for k in (1, 3):
        ok, f = within(g[k]["dof"][dmask], o[k]["dof"][dmask], 1e-3, 1e-3)
        assert ok, (k, f)
        ok, f = within(g[k]["body"][bmask][:, :3], o[k]["body"][bmask][:, :3], 1e-3, 1e-3)
        assert ok, (k, f)
    # quaternions: equal up to sign
    qg, qo = g[3]["body"][bmask][:, 3:7], o[3]["body"][bmask][:, 3:7]
    dots = np.abs((qg * qo).sum(1))
    assert (dots > 1 - 1e-4).mean() >= 0.98


def test_body_forces_match_oracle():
    from paper_2108_10470_gb300 import sim
    w = W.ant_workload(37)
    rng = np.random.default_rng(6)
    forces = [dict(body_force=rng.uniform(-2, 2, (w.n_body, 6))) for _ in range(3)]
    flags = sim.SIM_FLAG_SIGNATURE | sim.SIM_FLAG_BODY_FORCES
    g, o = rollout_both(w, 3, flags, lambda k: forces[k])
    same = (g[0]["sig"] == o[0]["sig"])
    assert same.mean() >= 0.9
    rows = np.repeat(same, 1)
    ok, f = within(g[0]["root"][rows], o[0]["root"][rows], 1e-4, 1e-5)
    assert ok, f
    # and the force matters: without it the state differs
    g2, _ = rollout_both(w, 1, sim.SIM_FLAG_SIGNATURE, lambda k: {})
    assert np.abs(g2[0]["root"] - g[0]["root"]).max() > 1e-4


def test_free_body_pushed_in_zero_gravity():
    """Newton on the GPU: a 2 kg body with a 3 N force at its COM gains 1.5 m/s^2 x dt per step."""
    import torch
    from paper_2108_10470_gb300 import sim
    b = W._Builder("body")
    b.link(-1, W.JOINT_FREE, mass=2.0, com=(0.05, -0.02, 0.03), inertia=(0.4, 0.4, 0.4, 0, 0, 0))
    w = W.homogeneous("body", b.build(), 3, params=W.Params(gravity=(0.0, 0.0, 0.0)))
    s = sim.Sim(w, flags=sim.SIM_FLAG_BODY_FORCES | sim.SIM_FLAG_RIGID_BODY_STATE)
    root = torch.zeros((3, 13))
    root[:, 6] = 1
    root[:, 2] = 3.0
    s.root_state.copy_(root)
    f = torch.zeros((3, 6))
    f[:, 0] = 3.0
    s.rigid_body_force.copy_(f)
    for _ in range(10):
        s.step()
    r = s.root_state.cpu().numpy()
    assert np.allclose(r[:, 7], 1.5 * 10 * w.dt, rtol=1e-5) and np.abs(r[:, 10:13]).max() < 1e-6
    bs = s.rigid_body_state.cpu().numpy()
    assert np.allclose(bs[:, :3], r[:, :3], atol=1e-6) and np.allclose(bs[:, 7:10], r[:, 7:10], atol=1e-6)
    s.destroy()


@pytest.mark.parametrize("name", ["ant", "humanoid", "ball_ant"])
def test_mass_matrix_and_jacobian_match_oracle(name):
    import torch
    from paper_2108_10470_gb300 import sim
    w = {"ant": W.ant_workload, "humanoid": W.humanoid_workload,
         "ball_ant": lambda n: W.homogeneous("ball_ant", W.ant(ball_hips=True), n)}[name](5)
    root, dof, _ = W.seeded_inputs(w, 2, 1)
    rng = np.random.default_rng(7)
    root[:, 7:13] = rng.uniform(-1, 1, (w.n_envs, 6))
    dof[:, 1] = rng.uniform(-1, 1, dof.shape[0])
    s = sim.Sim(w)
    s.root_state.copy_(torch.from_numpy(root))
    s.dof_state.copy_(torch.from_numpy(dof))
    M = s.compute_mass_matrix().cpu().numpy()
    J = s.compute_jacobian().cpu().numpy()
    s.destroy()
    O = oracle.Oracle(w)
    m = w.models[0]
    nj = m.n_jdof
    for e in range(w.n_envs):
        re, de = root[e:e + 1].astype(np.float64), dof[e * nj:(e + 1) * nj].astype(np.float64)
        H = O.crba(e, re, de)
        n = H.shape[0]
        assert np.allclose(M[e, :n, :n], H, rtol=1e-4, atol=1e-5 * np.abs(H).max())
        assert np.all(M[e, n:, :] == 0) and np.all(M[e, :, n:] == 0)
        for l in range(m.n_links):
            Jo = O.jacobian(e, re, de, l)
            assert np.allclose(J[e, l, :, :n], Jo, rtol=1e-4, atol=1e-4), (e, l)
