"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerance. The strict bound per component is |gpu - oracle| <= atol + rtol |oracle| with
1e-4 / 1e-5 after one env-step and 1e-3 / 1e-3 after 16. The method is ill-conditioned in
places (the TGS position bias divides separations by h/n_pos, and light links amplify contact
impulses), so a faithful FP32 evaluation cannot meet the strict bound on every component: the
oracle's own algorithm run in single precision misses it on a small fraction of components. With
f32 = the lowest fraction of components within the strict bound over four single-precision
evaluations of the oracle (inputs as given and nudged by one float32 ulp), every sample, however
small, must have
  (a) a fraction within the strict bound of at least max(0.98, f32 - 0.005), or f32 - 0.005 where
      the FP32 evaluations themselves stay below 98 % (the Humanoid over 16 steps);
  (b) every component within the strict bound plus K = 16 times its env's FP32 conditioning scale
      (the largest deviation from FP64 of those four evaluations over the env's components);
  (c) on samples of fewer than 1000 components, where the fraction is coarse, every component
      within the strict bound or within 4 times that component's own FP32 deviation.

Integer work (contact pairs, counts, the constraint-set signature) must match bit-exactly; an
environment whose constraint set differs at some step (a contact or limit decision within
rounding of its threshold) is counted as a contact-set change, reported, and excluded from the
state comparison from then on. At most 5 % of the envs of a small one-step batch may change
(1 % at full size), and 10 % over 16 steps.
"""
import numpy as np
import pytest

from paper_2108_10470_gb300 import workloads as W
from parity_util import compare, env_rows, fp32_scales, gpu_rollout, oracle_rollout

pytestmark = pytest.mark.gpu
K_COND = 16.0


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10470_gb300 import build
    build.build_library()
    torch.cuda.set_device(0)


def workload(name, n_envs):
    return {"cartpole": W.cartpole_workload, "ant": W.ant_workload, "humanoid": W.humanoid_workload,
            "hand": W.hand_workload, "mixed": W.mixed_workload}[name](n_envs)


PER = {"root": lambda w: w.env_actor_count, "dof": lambda w: w.env_jdof, "net_force": lambda w: w.env_body}


K_COMPONENT = 4.0
SMALL_SAMPLE = 1000


def strict_fraction_bar(f32_frac):
    """Lowest admissible fraction of components within the strict bound: 98 %, or half a
    percentage point under the FP32 evaluations of the oracle where those do better or worse."""
    return max(0.98, f32_frac - 0.005) if f32_frac >= 0.98 else f32_frac - 0.005


def check_rollout(w, steps, rtol, atol, seed=0, min_same=None, flags=1, setup=None):
    if min_same is None:
        min_same = (0.99 if w.n_envs >= 1024 else 0.95) if steps == 1 else 0.9
    root, dof, acts = W.seeded_inputs(w, seed, steps)
    g = gpu_rollout(w, root, dof, acts, steps, flags=flags, setup=setup)
    o, scales = fp32_scales(w, root, dof, acts, steps, rtol, atol)
    same = np.ones(w.n_envs, bool)
    for k in range(steps):
        assert o[k]["failed"] == 0 and not g[k]["status"].any()
        same &= g[k]["sig"] == o[k]["sig"]
        # integer contact lists: identical wherever the constraint sets agree
        for e in np.nonzero(same)[0]:
            assert g[k]["n_pairs"][e] == o[k]["n_pairs"][e]
            c = int(o[k]["n_pairs"][e])
            assert np.array_equal(g[k]["pairs"][e, :c], o[k]["pairs"][e, :c])
    changed = int((~same).sum())
    assert same.mean() >= min_same, \
        f"{changed} of {w.n_envs} envs changed constraint sets (at most {(1 - min_same) * 100:.0f} % may)"
    report = [f"{w.name} x{w.n_envs}, {steps} steps: contact-set changes in {changed} envs"]
    for key in ("root", "dof", "net_force"):
        a, b = g[-1][key], o[-1][key]
        strict = atol + rtol * np.abs(b)
        within = np.abs(a - b) <= strict
        rows = env_rows(w, PER[key](w))
        comp_mask = np.zeros(a.shape[0], bool)
        for e in np.nonzero(same)[0]:
            comp_mask[rows[e]] = True
        count = int(comp_mask.sum()) * (a.shape[1] if a.ndim > 1 else 1)
        frac = float(within[comp_mask].mean()) if comp_mask.any() else 1.0
        f32_frac = scales[-1]["strict_frac"][key]
        bar = strict_fraction_bar(f32_frac)
        report.append(f"  {key}: {100 * frac:.3f} % of {count} components within the strict bound "
                      f"(CPU FP32 evaluation: {100 * f32_frac:.3f} %, bar {100 * bar:.3f} %)")
        assert frac >= bar, f"{key}: only {frac:.4f} of {count} components within the strict bound (bar {bar:.4f})"
        if count < SMALL_SAMPLE and comp_mask.any():
            own = scales[-1]["component"][key]
            ok = within | (np.abs(a - b) <= K_COMPONENT * own)
            bad = int((~ok[comp_mask]).sum())
            assert bad == 0, f"{key}: {bad} of {count} components outside both the strict bound and " \
                             f"{K_COMPONENT:g} x their own FP32 deviation"
        for e in np.nonzero(same)[0]:
            sl = rows[e]
            if sl.stop == sl.start:
                continue
            excess = (np.abs(a[sl] - b[sl]) - strict[sl]).max()
            bound = K_COND * scales[-1][key][e]
            assert excess <= bound, f"{key} env {e}: exceeds strict bound by {excess:.3e} > {bound:.3e}"
    print("\n".join(report))
    return g, o, same


@pytest.mark.parametrize("name,n_envs", [("cartpole", 64), ("cartpole", 67), ("ant", 67), ("humanoid", 37),
                                         ("hand", 37), ("mixed", 67)])
def test_one_step(name, n_envs):
    """One env-step (2 substeps) at 1e-4 relative / 1e-5 absolute; sizes span several CTAs and a
    ragged last block."""
    check_rollout(workload(name, n_envs), 1, 1e-4, 1e-5)


@pytest.mark.parametrize("name,n_envs", [("cartpole", 64), ("ant", 67), ("humanoid", 37), ("hand", 37),
                                         ("mixed", 67)])
def test_sixteen_steps(name, n_envs):
    """16 env-steps at 1e-3 relative / absolute on envs whose constraint sets never changed."""
    check_rollout(workload(name, n_envs), 16, 1e-3, 1e-3)


@pytest.mark.parametrize("name,n_envs", [("ant", 67), ("humanoid", 37), ("hand", 37), ("mixed", 67)])
@pytest.mark.parametrize("steps,rtol,atol", [(1, 1e-4, 1e-5), (16, 1e-3, 1e-3)])
def test_row_solver_form(name, n_envs, steps, rtol, atol):
    """The row form of the Gauss-Seidel solve (SIM_FLAG_ROW_SOLVER: each row's J v and separation
    as group reductions over Y), the form a substep falls back to when its Delassus block does not
    fit beside Y, against the oracle at the same bars as the default form."""
    check_rollout(workload(name, n_envs), steps, rtol, atol, flags=1 | 64)


def tray_arm_workload(n_envs):
    """A fixed pivot and a hinged arm (one generalized DOF) carrying a flat box at ground height:
    up to eight box-corner contacts, 24 rows, against one DOF, so the Gauss-Seidel solve works on a
    rank-one Delassus matrix (every row's response lies along the same generalized direction)."""
    b = W._Builder("tray_arm")
    b.link(-1, W.JOINT_FIXED, mass=1.0, inertia=(1, 1, 1, 0, 0, 0))
    m, inn = W.box_mass(0.2, 0.15, 0.05, 1.0)
    arm = b.link(0, W.JOINT_REVOLUTE, axis=(0, 1, 0), mass=m, com=(0.3, 0.0, -0.25), inertia=inn, damping=0.1)
    b.shape(arm, W.SHAPE_BOX, (0.2, 0.15, 0.05), pos=(0.3, 0.0, -0.25))
    return W.homogeneous("tray_arm", b.build(root_pos=(0.0, 0.0, 0.3), dof_noise=0.05), n_envs)


@pytest.mark.parametrize("steps,rtol,atol", [(1, 1e-4, 1e-5), (16, 1e-3, 1e-3)])
def test_overconstrained_tray(steps, rtol, atol):
    """Many contact rows on one generalized DOF (two to four box corners down): the impulses that
    satisfy the contacts are not unique, and the Gauss-Seidel sweep picks one by its row order, as
    the oracle's does; against the oracle at the usual bars."""
    check_rollout(tray_arm_workload(48), steps, rtol, atol)


@pytest.mark.parametrize("name,n_envs", [("ant", 4096), ("humanoid", 4096), ("hand", 4096), ("mixed", 16384)])
def test_full_size_one_step(name, n_envs):
    """Full-size configurations (one launch per env type and step) against the oracle on all envs."""
    check_rollout(workload(name, n_envs), 1, 1e-4, 1e-5)


def test_impulse_cache_and_forces_match():
    w = W.ant_workload(40)
    g, o, same = check_rollout(w, 4, 1e-3, 1e-3)
    for e in np.nonzero(same)[0]:
        assert np.allclose(g[-1]["cache"][e, :w.models[0].contact_cap * 3 + 16],
                           o[-1]["cache"][e, :w.models[0].contact_cap * 3 + 16], rtol=1e-3, atol=1e-4)


def test_box_rest_on_gpu():
    """The resting box stays at rest on the GPU too (1000 steps) and matches the oracle."""
    m = W.free_box(0.2, 0.1, 0.1, mass=2.0)
    w = W.homogeneous("box", m, 3)
    root = np.zeros((3, 13), np.float32)
    root[:, 2] = 0.1
    root[:, 6] = 1.0
    acts = np.zeros((1000, 0), np.float32)
    g = gpu_rollout(w, root, np.zeros((0, 2), np.float32), acts, 1000, flags=0)
    r = g[-1]["root"]
    assert np.abs(r[:, 7:13]).max() <= 1e-3
    assert np.abs(r[:, 0:3] - [0, 0, 0.1]).max() <= 1e-3
    assert np.allclose(g[-1]["net_force"][:, 2], 2.0 * 9.81, rtol=0.01)


def test_pendulum_period_on_gpu():
    """Small-angle period of the 1 m, 0.5 kg rod measured on the GPU: 1.63795 s within 1e-3."""
    import math
    w = W.homogeneous("pendulum", W.pendulum(), 1)
    root = np.zeros((1, 13), np.float32)
    root[0, 6] = 1
    dof = np.array([[0.01, 0.0]], np.float32)
    steps = 600
    g = gpu_rollout(w, root, dof, np.zeros((steps, 1), np.float32), steps, flags=0)
    x = np.array([0.01] + [s["dof"][0, 0] for s in g])
    t = w.dt * np.arange(steps + 1)
    sgn = np.sign(x)
    idx = np.where((sgn[:-1] < 0) & (sgn[1:] >= 0))[0]
    tc = [t[i] - x[i] * (t[i + 1] - t[i]) / (x[i + 1] - x[i]) for i in idx]
    T = np.diff(tc).mean()
    assert abs(T - 2 * math.pi * math.sqrt(2.0 / (3 * 9.81))) <= 1e-3 * 1.63795


def test_heterogeneous_batch_two_types():
    """Ant and Humanoid envs interleaved in one simulation (two env types, two launches)."""
    ant, hum = W.ant(), W.humanoid()
    n = 24
    eam = np.array([i % 2 for i in range(n)], np.int32)
    w = W.Workload("mixed", [ant, hum], eam, 1, n, W.Params())
    check_rollout(w, 4, 1e-3, 1e-3)


def test_box_rests_on_two_capsules_gpu():
    """Capsule-box pair contacts on the GPU: a box laid across two fixed capsules comes to rest
    0.57 m up with the pair contacts carrying its weight; the first step's contact list (shape a,
    shape b, slot) equals the oracle's."""
    import torch
    from paper_2108_10470_gb300 import sim
    from scenes import two_actor_env

    qy = W.Q_X_TO_Y
    w, root = two_actor_env([(-0.03, 0, 0.5), (0.03, 0, 0.5)], [qy, qy], (0, 0, 0.5 + 0.02 + 0.05))
    o = oracle_rollout(w, root, np.zeros((0, 2)), np.zeros((1, 0)), 1)
    s = sim.Sim(w)
    s.root_state.copy_(torch.from_numpy(root))
    for k in range(600):
        s.step()
        if k == 0:
            n = int(s.contact_count.cpu()[0])
            assert n == int(o[0]["n_pairs"][0]) and n >= 2
            assert np.array_equal(s.contact_pairs.cpu().numpy()[0, :n], o[0]["pairs"][0, :n])
    r = s.root_state.cpu().numpy()
    f = s.net_contact_force.cpu().numpy()
    assert not s.status.cpu().numpy().any()
    assert np.abs(r[1, 7:13]).max() < 1e-3 and abs(r[1, 2] - 0.57) < 1e-3
    assert abs(f[1, 2] - 0.2 * 9.81) < 0.01 * 0.2 * 9.81
    assert np.allclose(f[0], -f[1], atol=1e-4)
    s.destroy()


def test_padded_actor_lists_map_rows():
    """Envs with fewer actors than the widest (-1 padding): the root-state rows run on without gaps
    and a row reset through the indexed setter lands on the right env."""
    import torch
    from paper_2108_10470_gb300 import sim

    w = W.mixed_workload(40)
    root, dof, acts = W.seeded_inputs(w, 1, 2)
    counts = [w.env_actor_count(e) for e in range(w.n_envs)]
    assert root.shape[0] == sum(counts) < 2 * w.n_envs
    check_rollout(w, 2, 1e-3, 1e-3)
    # reset the second actor (the cube) of the first two-actor env: only that env's cache clears
    e = counts.index(2)
    a = sum(counts[:e]) + 1
    s = sim.Sim(w)
    s.root_state.copy_(torch.from_numpy(root))
    s.dof_state.copy_(torch.from_numpy(dof))
    s.dof_actuation.copy_(torch.from_numpy(acts[0]))
    s.step()
    before = s.impulse_cache.clone()
    assert before[e].abs().sum() > 0
    new_root = s.root_state[a:a + 1].clone()
    new_root[0, 2] += 0.1
    s.set_root_state_indexed(new_root, torch.tensor([a], dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(s.root_state[a], new_root[0])
    assert torch.all(s.impulse_cache[e] == 0)
    keep = [i for i in range(w.n_envs) if i != e]
    assert torch.equal(s.impulse_cache[keep], before[keep])
    s.destroy()


def test_single_env_and_no_contacts():
    w = W.ant_workload(1)
    check_rollout(w, 2, 1e-4, 1e-5, min_same=1.0)
    w = W.homogeneous("ant_air", W.ant(), 5, params=W.Params(gravity=(0, 0, 0)))
    root, dof, acts = W.seeded_inputs(w, 3, 3)
    root[:, 2] = 3.0  # far above the ground: no contacts
    g = gpu_rollout(w, root, dof, acts, 3)
    o = oracle_rollout(w, root, dof, acts, 3)
    assert (g[-1]["n_pairs"] == 0).all()
    rep = compare(w, g[-1], o[-1], 1e-4, 1e-5, np.ones(5, bool))
    for key, (ok, worst) in rep.items():
        assert ok.all(), (key, worst)


def test_deterministic():
    w = W.ant_workload(64)
    root, dof, acts = W.seeded_inputs(w, 1, 5)
    a = gpu_rollout(w, root, dof, acts, 5)
    b = gpu_rollout(w, root, dof, acts, 5)
    for k in ("root", "dof", "net_force", "cache"):
        assert np.array_equal(a[-1][k], b[-1][k])


def test_set_state_indexed_and_views():
    import torch
    from paper_2108_10470_gb300 import sim

    w = W.ant_workload(10)
    s = sim.Sim(w)
    assert tuple(s.root_state.shape) == (10, 13) and tuple(s.dof_state.shape) == (80, 2)
    assert tuple(s.net_contact_force.shape) == (90, 3) and tuple(s.dof_actuation.shape) == (80,)
    root, dof, acts = W.seeded_inputs(w, 0, 3)
    s.root_state.copy_(torch.from_numpy(root))
    s.dof_state.copy_(torch.from_numpy(dof))
    for k in range(3):
        s.dof_actuation.copy_(torch.from_numpy(acts[k]))
        s.step()
    before_root = s.root_state.clone()
    before_dof = s.dof_state.clone()
    idx = torch.tensor([2, 7], dtype=torch.int32, device="cuda")
    new_root = torch.zeros((2, 13), device="cuda")
    new_root[:, 2] = 1.0
    new_root[:, 6] = 1.0
    s.set_root_state_indexed(new_root, idx)
    new_dof = torch.full((2, 16), 0.05, device="cuda")
    s.set_dof_state_indexed(new_dof, idx)
    torch.cuda.synchronize()
    assert torch.equal(s.root_state[idx.long()], new_root)
    keep = [i for i in range(10) if i not in (2, 7)]
    assert torch.equal(s.root_state[keep], before_root[keep])
    d = s.dof_state.view(10, 8, 2)
    assert torch.all(d[idx.long()] == 0.05)
    assert torch.equal(d[keep], before_dof.view(10, 8, 2)[keep])
    assert torch.all(s.impulse_cache[idx.long()] == 0)
    s.destroy()


def test_status_reports_nonfinite_input():
    """A NaN written into one env's input state (from the host) is reported for that env only."""
    import torch
    from paper_2108_10470_gb300 import sim

    w = W.ant_workload(8)
    s = sim.Sim(w)
    root, dof, _ = W.seeded_inputs(w, 0, 1)
    dof[3 * 8 + 2, 1] = np.nan
    s.root_state.copy_(torch.from_numpy(root))
    s.dof_state.copy_(torch.from_numpy(dof))
    s.step()
    assert s.sync_status() == 1
    st = s.status.cpu().numpy()
    assert st[3] != 0 and (np.delete(st, 3) == 0).all()
    s.destroy()


@pytest.mark.parametrize("pinned,plan", [(False, "per_type"), (True, "per_type"), (True, "persistent"),
                                         (True, "graph")])
def test_step_host_matches_device_path(pinned, plan):
    """sim_step_host from pageable host buffers (copied) and from pinned ones (read and written by
    the per-type step kernels themselves; copied for persistent and graph handles): the same outputs
    as the device path of the same plan, bit for bit, and the views (root, DOF state, actuation) as
    after sim_step."""
    import torch
    from paper_2108_10470_gb300 import sim

    flags = {"per_type": 0, "persistent": sim.SIM_FLAG_PERSISTENT, "graph": sim.SIM_FLAG_GRAPH}[plan]
    w = W.ant_workload(32)
    root, dof, acts = W.seeded_inputs(w, 5, 2)
    host = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()) if pinned else np.ascontiguousarray
    outs, views = [], []
    for use_host in (False, True):
        s = sim.Sim(w, flags=flags)
        s.root_state.copy_(torch.from_numpy(root))
        s.dof_state.copy_(torch.from_numpy(dof))
        r = host(np.zeros_like(root))
        d = host(np.zeros_like(dof))
        for k in range(2):
            if use_host:
                s.step_host(host(acts[k]), r, d)
            else:
                s.dof_actuation.copy_(torch.from_numpy(acts[k]))
                s.step()
                r, d = s.root_state.cpu().numpy(), s.dof_state.cpu().numpy()
        outs.append((r.copy(), d.copy()))
        views.append([getattr(s, v).cpu().numpy() for v in ("root_state", "dof_state", "dof_actuation")])
        s.destroy()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    for a, b in zip(*views):
        assert np.array_equal(a, b)
    assert np.array_equal(views[1][2], acts[1])


@pytest.mark.parametrize("source,plan", [("device", "per_type"), ("pinned", "per_type"), ("pageable", "per_type"),
                                         ("device", "mixed"), ("device", "persistent"), ("device", "graph")])
def test_step_actuated_equals_writing_the_view(source, plan):
    """sim_step_actuated with this step's forces in a caller buffer (read in place by the step
    kernel of a one-type handle from device or pinned host memory; copied into the view from
    pageable memory and for mixed, persistent and graph handles): every view bit for bit as after
    writing DOF_ACTUATION and calling sim_step, over three steps, the actuation view holding the
    last step's forces."""
    import torch
    from paper_2108_10470_gb300 import sim

    flags = sim.SIM_FLAG_SIGNATURE | {"per_type": 0, "mixed": 0, "persistent": sim.SIM_FLAG_PERSISTENT,
                                      "graph": sim.SIM_FLAG_GRAPH}[plan]
    w = W.mixed_workload(48) if plan == "mixed" else W.ant_workload(40)
    root, dof, acts = W.seeded_inputs(w, 7, 3)
    a, b = sim.Sim(w, flags=flags), sim.Sim(w, flags=flags)
    for s in (a, b):
        s.root_state.copy_(torch.from_numpy(root))
        s.dof_state.copy_(torch.from_numpy(dof))
    for k in range(3):
        a.dof_actuation.copy_(torch.from_numpy(acts[k]))
        a.step()
        f = torch.from_numpy(np.ascontiguousarray(acts[k]))
        f = {"device": lambda t: t.cuda(), "pinned": lambda t: t.pin_memory(), "pageable": lambda t: t}[source](f)
        if source == "pageable":  # the binding passes only device or pinned tensors: call the C ABI directly
            sim.check(sim.load().sim_step_actuated(b.h, f.data_ptr(), float(w.dt), int(w.substeps)), "step")
        else:
            b.step_actuated(f)
        torch.cuda.synchronize()
        for name in b.STATE_NAMES:
            x, y = getattr(a, name).cpu().numpy(), getattr(b, name).cpu().numpy()
            assert np.array_equal(x.view(np.uint32), y.view(np.uint32)), (name, k)
    assert np.array_equal(b.dof_actuation.cpu().numpy(), acts[2])
    a.destroy()
    b.destroy()


def test_step_actuated_without_dofs():
    """A batch with no joint DOFs (free boxes dropped on the ground): sim_step_actuated takes an
    empty tensor (a null buffer at the C ABI) and steps exactly as sim_step."""
    import torch
    from paper_2108_10470_gb300 import sim

    w = W.homogeneous("boxes", W.free_box(0.2, 0.1, 0.1, mass=2.0, z=0.12), 24)
    root, dof, _ = W.seeded_inputs(w, 3, 1)
    root[:, 2] += 0.01 * np.arange(24)
    a, b = sim.Sim(w, flags=sim.SIM_FLAG_SIGNATURE), sim.Sim(w, flags=sim.SIM_FLAG_SIGNATURE)
    assert a.N_D == 0
    for s in (a, b):
        s.root_state.copy_(torch.from_numpy(root))
    for k in range(4):
        a.step()
        b.step_actuated(torch.empty(0, device="cuda"))
    torch.cuda.synchronize()
    for name in ("root_state", "net_contact_force", "impulse_cache", "contact_count"):
        assert np.array_equal(getattr(a, name).cpu().numpy(), getattr(b, name).cpu().numpy()), name
    assert int(a.contact_count.cpu().numpy().sum()) > 0
    a.destroy()
    b.destroy()


def test_fp32_probe_reports_plausible_peak():
    from paper_2108_10470_gb300 import sim
    f = sim.probe_fp32_peak(2000)
    assert 1e12 < f < 2e14
