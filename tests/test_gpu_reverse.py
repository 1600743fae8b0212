"""The reverse pass of the env-step on the GPU (sim_step_taped + sim_step_adjoint, and sim_step_vjp,
which uses them where they cover the handle) against the FP64 oracle's forward-mode derivative.

* The taped step is the step: the same states, contacts and impulses bit for bit as sim_step.
* The vector-Jacobian product of one step: for every input direction of every env (root position,
  root rotation along the unit sphere, root velocities of floating roots, joint positions and
  velocities, actuation, every impulse-cache slot) the GPU's J^T g against the oracle's J u . g,
  per env in the max norm relative to the env's gradient scale: within 1e-3 of the scale plus
  16 times the env's FP32 conditioning spread (the largest deviation from FP64 of the oracle's own
  derivative evaluated in single precision, at the input and at inputs nudged by one float32 ulp).
  An env whose FP32 evaluation takes a different branch (a clamp or target within rounding of its
  threshold) may deviate: at most one env per test.
* The reverse and the forward-mode GPU evaluations agree (the second, independent kernel).
* Capsule-box shape pairs (the hand holding its cube; a batch mixing Ant, Humanoid and hand envs)
  and ball joints (the Ant with ball hips, the Humanoid with ball abdomen and hips) go through the
  same checks; every handle has a tape.
"""
import numpy as np
import pytest

import oracle
from paper_2108_10470_gb300 import workloads as W
from test_gpu_adjoint import K_COND, WORKLOADS, make_sim, warm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10470_gb300 import build
    build.build_library()
    torch.cuda.set_device(0)


STATE = ("root_state", "dof_state", "impulse_cache", "net_contact_force", "contact_pairs", "contact_count", "signature")


@pytest.mark.parametrize("name,n,plan", [("ant", 67, "per_type"), ("humanoid", 37, "per_type"), ("cartpole", 64, "per_type"),
                                         ("driven_ant", 40, "per_type"), ("ant", 67, "persistent"),
                                         ("humanoid", 37, "row_solver"), ("mixed_no_hand", 48, "per_type"),
                                         ("hand", 37, "per_type"), ("mixed", 48, "per_type"), ("mixed", 48, "persistent"),
                                         ("ball_ant", 40, "per_type"), ("ball_humanoid", 16, "per_type")])
def test_taped_step_is_the_step(name, n, plan):
    """Six steps of sim_step and of sim_step_taped from the same seeded state: every view equal bit
    for bit (the same kernels, given a tape pointer: the tape stores are their only difference).
    A persistent handle's taped step runs the per-type kernels, while its step runs the persistent
    kernel, whose tile bodies are compiled without the tape stores (another register allocation):
    there the float views agree to rounding and the integer views exactly."""
    import torch
    from paper_2108_10470_gb300 import sim
    if name == "mixed_no_hand":
        ant, hum = W.ant(), W.humanoid()
        w = W.Workload("two_types", [ant, hum], np.array([i % 2 for i in range(n)], np.int32), 1, n, W.Params())
    elif name == "mixed":
        w = W.mixed_workload(n)
    else:
        w = WORKLOADS[name](n)
    flags = sim.SIM_FLAG_SIGNATURE | {"per_type": 0, "persistent": sim.SIM_FLAG_PERSISTENT,
                                      "row_solver": sim.SIM_FLAG_ROW_SOLVER}[plan]
    root, dof, acts = W.seeded_inputs(w, 4, 6)
    handles = []
    for _ in range(2):
        if name == "driven_ant":
            s, _ = make_sim(name, w)
            s.destroy()
            s, _ = make_sim(name, w)
        else:
            s = sim.Sim(w, flags=flags)
        s.root_state.copy_(torch.from_numpy(root))
        s.dof_state.copy_(torch.from_numpy(dof))
        handles.append(s)
    ref, tap = handles
    tape = torch.empty(tap.tape_floats(), device="cuda")
    for k in range(6):
        for s in handles:
            s.dof_actuation.copy_(torch.from_numpy(acts[k]))
        ref.step()
        tap.step_taped(tape)
        torch.cuda.synchronize()
        for v in STATE:
            x, y = getattr(ref, v), getattr(tap, v)
            if plan == "persistent" and x.dtype == torch.float32:
                assert torch.allclose(x, y, rtol=1e-4, atol=1e-5), (v, k, (x - y).abs().max().item())
            else:
                assert torch.equal(x, y), (v, k)
    for s in handles:
        s.destroy()


def gpu_vjp(s, r, d, c, a, gout):
    import torch
    f = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    bufs = {"root_state": f(r), "dof_state": f(d), "dof_actuation": f(a), "impulse_cache": f(c),
            "grad_root_state": f(gout[0]), "grad_dof_state": f(gout[1]), "grad_impulse_cache": f(gout[2]),
            "grad_root_state_in": torch.full_like(f(r), 5.0), "grad_dof_state_in": torch.full_like(f(d), 5.0),
            "grad_dof_actuation": torch.full_like(f(a), 5.0), "grad_impulse_cache_in": torch.full_like(f(c), 7.0),
            "status": torch.full((s.w.n_envs,), 9, dtype=torch.int32, device="cuda")}
    s.step_vjp(bufs)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in bufs.items()}


def qtangent(q, k):
    """(1/2) [e_k; 0] (x) q: the quaternion's tangent of a world-axis rotation about axis k."""
    om = np.zeros((q.shape[0], 3))
    om[:, k] = 1.0
    t = np.zeros_like(q)
    t[:, 0] = 0.5 * (om[:, 0] * q[:, 3] + om[:, 1] * q[:, 2] - om[:, 2] * q[:, 1])
    t[:, 1] = 0.5 * (-om[:, 0] * q[:, 2] + om[:, 1] * q[:, 3] + om[:, 2] * q[:, 0])
    t[:, 2] = 0.5 * (om[:, 0] * q[:, 1] - om[:, 1] * q[:, 0] + om[:, 2] * q[:, 3])
    t[:, 3] = 0.5 * (-om[:, 0] * q[:, 0] - om[:, 1] * q[:, 1] - om[:, 2] * q[:, 2])
    return t


def free_rows(w):
    """Per root-state row (actor): whether its root is floating (its velocities are state)."""
    return np.array([m.free_root for e in range(w.n_envs) for m in w.actor_models(e)])


def directions(w, r, c):
    """Input directions seeded in every env at once: (label, root, dof, act, cache) tangents; the
    root velocity directions on the floating roots only."""
    nj = w.n_dof // w.n_envs
    free = free_rows(w)
    out = []
    for k in range(3):
        t = np.zeros_like(r); t[:, k] = 1.0
        out.append((f"p{k}", t, None, None, None))
        t = np.zeros_like(r); t[:, 3:7] = qtangent(r[:, 3:7], k)
        out.append((f"th{k}", t, None, None, None))
        if free.any():
            for base, nm in ((7, "v"), (10, "w")):
                t = np.zeros_like(r); t[free, base + k] = 1.0
                out.append((f"{nm}{k}", t, None, None, None))
    for j in range(nj):
        for comp, nm in ((0, "q"), (1, "qd")):
            t = np.zeros((w.n_dof, 2)); t[j::nj, comp] = 1.0
            out.append((f"{nm}{j}", None, t, None, None))
        t = np.zeros(w.n_dof); t[j::nj] = 1.0
        out.append((f"a{j}", None, None, t, None))
    for k in range(c.shape[1]):
        t = np.zeros_like(c); t[:, k] = 1.0
        out.append((f"c{k}", None, None, None, t))
    return out


def oracle_grad(w, r, d, c, a, gout, dirs, ctl, single=False, nudge=None):
    """Per env and direction: the oracle's directional derivative of <gout, step output>."""
    from test_gpu_adjoint import oracle_tangent
    ra = np.cumsum([0] + [w.env_actor_count(e) for e in range(w.n_envs)])
    rd = np.cumsum([0] + [w.env_jdof(e) for e in range(w.n_envs)])
    G = np.zeros((w.n_envs, len(dirs)))
    for i, (_, tr, td, ta, tc) in enumerate(dirs):
        t = (np.zeros_like(r) if tr is None else tr, np.zeros((w.n_dof, 2)) if td is None else td,
             np.zeros(w.n_dof) if ta is None else ta, np.zeros_like(c) if tc is None else tc)
        _, _, _, orr, odd, occ = oracle_tangent(w, r, d, c, a, t, single=single, nudge=nudge, ctl=ctl)
        for e in range(w.n_envs):
            G[e, i] = ((gout[0][ra[e]:ra[e + 1]] * orr[ra[e]:ra[e + 1]]).sum()
                       + (gout[1][rd[e]:rd[e + 1]] * odd[rd[e]:rd[e + 1]]).sum() + (gout[2][e] * occ[e]).sum())
    return G


def gpu_grad(w, g, r, dirs):
    ra = np.cumsum([0] + [w.env_actor_count(e) for e in range(w.n_envs)])
    rd = np.cumsum([0] + [w.env_jdof(e) for e in range(w.n_envs)])
    G = np.zeros((w.n_envs, len(dirs)))
    for i, (_, tr, td, ta, tc) in enumerate(dirs):
        for e in range(w.n_envs):
            v = 0.0
            if tr is not None:
                v += (g["grad_root_state_in"][ra[e]:ra[e + 1]] * tr[ra[e]:ra[e + 1]]).sum()
            if td is not None:
                v += (g["grad_dof_state_in"][rd[e]:rd[e + 1]] * td[rd[e]:rd[e + 1]]).sum()
            if ta is not None:
                v += (g["grad_dof_actuation"][rd[e]:rd[e + 1]] * ta[rd[e]:rd[e + 1]]).sum()
            if tc is not None:
                v += (g["grad_impulse_cache_in"][e] * tc[e]).sum()
            G[e, i] = v
    return G


def output_gradient(w, r, d, c, rng):
    gout = (rng.standard_normal(r.shape), rng.standard_normal(d.shape), rng.standard_normal(c.shape))
    gout[0][~free_rows(w), 7:] = 0.0  # a fixed root's velocity is not state
    return gout


@pytest.mark.parametrize("name,n", [("ant", 40), ("humanoid", 16), ("cartpole", 32), ("driven_ant", 24),
                                    ("tendon_ant", 24), ("pushed_ant", 24), ("hand", 12), ("hand_tendon", 8),
                                    ("ball_ant", 24), ("ball_humanoid", 12)])
def test_reverse_vjp_matches_oracle_derivative(name, n):
    w = WORKLOADS[name](n)
    r, d, c, a = warm(w, seed=5)
    rng = np.random.default_rng(6)
    gout = output_gradient(w, r, d, c, rng)
    s, ctl = make_sim(name, w)
    check_vjp_against_oracle(name, w, s, ctl, r, d, c, a, gout)


def box_on_capsules(n, rng):
    """n envs of a free 0.2 kg box (half extents 0.05) lying across two fixed capsules 0.06 m apart
    (a holder of one link: 8 lanes per env), each box nudged, tilted and moving a little."""
    from scenes import two_actor_env
    qy = W.Q_X_TO_Y
    w1, root1 = two_actor_env([(-0.03, 0, 0.5), (0.03, 0, 0.5)], [qy, qy], (0, 0, 0.572))
    w = W.Workload("box_on_capsules", w1.models, np.tile(np.array([0, 1], np.int32), n), 2, n, w1.params)
    root = np.tile(root1, (n, 1))
    box = root[1::2]
    box[:, 0] += rng.uniform(-0.01, 0.01, n)
    box[:, 2] += rng.uniform(-0.001, 0.003, n)
    ang = rng.uniform(-0.05, 0.05, (n, 3))
    half = 0.5 * np.linalg.norm(ang, axis=1)
    box[:, 3:6] = ang / np.maximum(2 * half, 1e-12)[:, None] * np.sin(half)[:, None]
    box[:, 6] = np.cos(half)
    box[:, 7:13] = rng.uniform(-0.05, 0.05, (n, 6))
    return w, root


def test_reverse_vjp_of_pairs_at_eight_lanes():
    """Capsule-box pairs in the 8-lane instantiation of the pair kernels (every arena in shared
    memory): boxes lying across two capsules, against the oracle's derivative in every direction."""
    rng = np.random.default_rng(21)
    w, root = box_on_capsules(24, rng)
    O = oracle.Oracle(w)
    r, d = root.copy(), np.zeros((0, 2))
    a0 = np.zeros((1, 0))
    for _ in range(3):  # warm impulses
        O.step(r, d, a0[0])
    f = lambda x: x.astype(np.float32).astype(np.float64)
    r, c = f(r), f(O.cache)
    from paper_2108_10470_gb300 import sim
    s = sim.Sim(w)
    assert s.type_config(0)["lanes_per_env"] == 8
    gout = output_gradient(w, r, d, c, rng)
    got = check_vjp_against_oracle("box_on_capsules", w, s, None, r, d, c, np.zeros(0), gout)
    # and against the forward-mode kernel: two FP32 evaluations of the same derivative
    s = sim.Sim(w, flags=sim.SIM_FLAG_TANGENT_VJP)
    g_fwd = gpu_vjp(s, r, d, c, np.zeros(0), gout)
    s.destroy()
    fwd = gpu_grad(w, g_fwd, r, directions(w, r, c))
    rel = np.abs(got - fwd).max(1) / np.maximum(1.0, np.abs(fwd).max(1))
    print(f"box_on_capsules x{w.n_envs}: reverse vs forward mode, relative deviation median {np.median(rel):.2e}, "
          f"max {rel.max():.2e}")
    assert (rel > 1e-2).sum() <= 1 and np.median(rel) <= 1e-3


def check_vjp_against_oracle(name, w, s, ctl, r, d, c, a, gout):
    """The handle's VJP (the reverse pass) of one step against the oracle's derivative in every
    input direction of every env, per env within 1e-3 of its gradient scale plus 16 times its FP32
    conditioning spread; at most one env outside. Destroys the handle."""
    assert s.tape_floats() is not None
    g = gpu_vjp(s, r, d, c, a, gout)
    n = w.n_envs
    s.destroy()
    assert not g["status"].any()
    g32 = tuple(x.astype(np.float32).astype(np.float64) for x in gout)
    dirs = directions(w, r, c)
    ref = oracle_grad(w, r, d, c, a, g32, dirs, ctl)
    probes = [oracle_grad(w, r, d, c, a, g32, dirs, ctl, single=True, nudge=x) for x in (None, 1)]
    got = gpu_grad(w, g, r, dirs)
    bad = []
    worst = 0.0
    for e in range(w.n_envs):
        scale = max(1.0, np.abs(ref[e]).max())
        spread = max(np.abs(p[e] - ref[e]).max() for p in probes)
        dev = np.abs(got[e] - ref[e]).max()
        worst = max(worst, dev / scale)
        if dev > 1e-3 * scale + K_COND * spread:
            bad.append((e, dev / scale, dirs[int(np.argmax(np.abs(got[e] - ref[e])))][0]))
    spreads = np.array([max(np.abs(p[e] - ref[e]).max() for p in probes) / max(1.0, np.abs(ref[e]).max())
                        for e in range(w.n_envs)])
    print(f"{name} x{n}: {len(dirs)} directions per env, largest relative deviation {worst:.2e}, "
          f"{len(bad)} envs outside the bound {bad}; FP32 conditioning spread median {np.median(spreads):.1e}, "
          f"max {spreads.max():.1e}")
    assert len(bad) <= 1, bad
    return got


@pytest.mark.parametrize("name,n", [("ant", 40), ("humanoid", 16), ("driven_ant", 24), ("tendon_ant", 24),
                                    ("pushed_ant", 24), ("hand", 12), ("ball_ant", 24), ("ball_humanoid", 12)])
def test_reverse_and_forward_mode_agree(name, n):
    """The reverse pass against the forward-mode kernel (SIM_FLAG_TANGENT_VJP) on the same inputs:
    two FP32 evaluations of the same derivative; the quaternion gradient compared along the sphere."""
    import torch
    from paper_2108_10470_gb300 import sim
    w = WORKLOADS[name](n)
    r, d, c, a = warm(w, seed=7)
    rng = np.random.default_rng(8)
    gout = output_gradient(w, r, d, c, rng)
    s, ctl = make_sim(name, w)
    assert s.tape_floats() is not None
    g_rev = gpu_vjp(s, r, d, c, a, gout)
    s.destroy()
    flags = sim.SIM_FLAG_TANGENT_VJP | (sim.SIM_FLAG_BODY_FORCES if name == "pushed_ant" else 0)
    s = sim.Sim(WORKLOADS[name](n), flags=flags)
    t32 = lambda x: torch.from_numpy(x.astype(np.float32))
    if ctl and "pos_target" in ctl:
        s.dof_position_target.copy_(t32(ctl["pos_target"]))
        s.dof_velocity_target.copy_(t32(ctl["vel_target"]))
    if ctl and "body_force" in ctl:
        s.rigid_body_force.copy_(t32(ctl["body_force"]))
    g_fwd = gpu_vjp(s, r, d, c, a, gout)
    s.destroy()
    dirs = directions(w, r, c)
    A, B = gpu_grad(w, g_rev, r, dirs), gpu_grad(w, g_fwd, r, dirs)
    rel = np.abs(A - B).max(1) / np.maximum(1.0, np.abs(B).max(1))
    far = [(e, dirs[int(np.argmax(np.abs(A[e] - B[e])))][0]) for e in np.nonzero(rel > 1e-2)[0]]
    print(f"{name} x{n}: reverse vs forward mode, relative deviation median {np.median(rel):.2e}, max {rel.max():.2e}, "
          f"envs past 1e-2 (env, direction) {far}")
    # two FP32 evaluations of the forward values too: an env whose contact or clamp decision lies
    # within rounding of its threshold may take different branches in the two kernels
    assert len(far) <= max(1, n // 20) and np.median(rel) <= 1e-3


def test_every_handle_has_a_tape():
    """Shape pairs, tendons and ball joints: the reverse pass covers them all."""
    for name in ("ball_ant", "ball_humanoid", "hand", "hand_tendon"):
        w = WORKLOADS[name](4)
        s, _ = make_sim(name, w)
        assert s.tape_floats() is not None, name
        s.destroy()


def env_cache_len(w, e):
    """Impulse-cache entries of env e: 3 per contact candidate (ground candidates of every shape,
    five per capsule-box pair across actors), 2 per joint DOF, 2 per tendon."""
    models = w.actor_models(e)
    per = {W.SHAPE_SPHERE: 1, W.SHAPE_CAPSULE: 2, W.SHAPE_BOX: 8}
    cand = sum(per[int(t)] for m in models for t in m.shape_type)
    caps = [sum(int(t == W.SHAPE_CAPSULE) for t in m.shape_type) for m in models]
    boxes = [sum(int(t == W.SHAPE_BOX) for t in m.shape_type) for m in models]
    cand += 5 * sum(caps[i] * boxes[j] + boxes[i] * caps[j] for i in range(len(models)) for j in range(i + 1, len(models)))
    return 3 * cand + 2 * w.env_jdof(e) + 2 * sum(len(m.tendons or []) for m in models)


def test_reverse_and_forward_mode_agree_on_a_mixed_batch():
    """Ant, Humanoid and hand envs in one handle (three env types, each with its own adjoint
    launch; the hand's with the pair phase, Y read from the tape and its adjoint in global memory):
    the reverse pass against the forward-mode kernel, per env over all of its input gradients."""
    import torch
    from paper_2108_10470_gb300 import sim
    w = W.mixed_workload(24)
    r, d, c, a = warm(w, seed=14)
    rng = np.random.default_rng(15)
    gout = output_gradient(w, r, d, c, rng)
    s = sim.Sim(w)
    assert s.tape_floats() is not None
    g_rev = gpu_vjp(s, r, d, c, a, gout)
    s.destroy()
    s = sim.Sim(w, flags=sim.SIM_FLAG_TANGENT_VJP)
    g_fwd = gpu_vjp(s, r, d, c, a, gout)
    s.destroy()
    assert not g_rev["status"].any() and not g_fwd["status"].any()
    ra = np.cumsum([0] + [w.env_actor_count(e) for e in range(w.n_envs)])
    rd = np.cumsum([0] + [w.env_jdof(e) for e in range(w.n_envs)])
    free = free_rows(w)
    rel = []
    for e in range(w.n_envs):
        parts = []
        for k in ("grad_root_state_in", "grad_dof_state_in", "grad_dof_actuation", "grad_impulse_cache_in"):
            A, B = g_rev[k], g_fwd[k]
            if k == "grad_root_state_in":  # the quaternion gradient along the sphere, velocities of free roots
                rows = slice(ra[e], ra[e + 1])
                qa, qb, q = A[rows, 3:7], B[rows, 3:7], r[rows, 3:7]
                ta = np.stack([(qa * qtangent(q, k2)).sum(1) for k2 in range(3)], 1)
                tb = np.stack([(qb * qtangent(q, k2)).sum(1) for k2 in range(3)], 1)
                vel = free[rows][:, None]
                parts.append((np.concatenate([A[rows, :3], ta, A[rows, 7:] * vel], 1).ravel(),
                              np.concatenate([B[rows, :3], tb, B[rows, 7:] * vel], 1).ravel()))
            elif k == "grad_impulse_cache_in":
                parts.append((A[e, :env_cache_len(w, e)], B[e, :env_cache_len(w, e)]))
            else:
                parts.append((A[rd[e]:rd[e + 1]].ravel(), B[rd[e]:rd[e + 1]].ravel()))
        x = np.concatenate([p[0] for p in parts])
        y = np.concatenate([p[1] for p in parts])
        rel.append(np.abs(x - y).max() / max(1.0, np.abs(y).max()))
    rel = np.array(rel)
    print(f"mixed x{w.n_envs}: reverse vs forward mode, relative deviation median {np.median(rel):.2e}, max {rel.max():.2e}")
    assert (rel <= 1e-2).mean() >= 0.9 and np.median(rel) <= 1e-3


def test_reverse_vjp_full_size_sampled_envs():
    """The differentiation workload's size and launch (1024 Ant-like envs, the reverse pass's
    per-type launch): one step's VJP over all envs, 16 of them (strided) checked against the oracle's
    derivative in every input direction."""
    w = W.ant_workload(1024)
    r, d, c, a = warm(w, seed=12)
    rng = np.random.default_rng(13)
    gout = output_gradient(w, r, d, c, rng)
    s, ctl = make_sim("ant", w)
    g = gpu_vjp(s, r, d, c, a, gout)
    s.destroy()
    assert not g["status"].any()
    idx = list(range(0, 1024, 64))
    ws = w.subset(idx)
    nj = 8
    rows = lambda x, per: np.concatenate([x[e * per:(e + 1) * per] for e in idx])
    rs, ds, cs, as_ = r[idx], rows(d, nj), c[idx], rows(a, nj)
    gs = (gout[0][idx], rows(gout[1], nj), gout[2][idx])
    g32 = tuple(x.astype(np.float32).astype(np.float64) for x in gs)
    dirs = directions(ws, rs, cs)
    ref = oracle_grad(ws, rs, ds, cs, as_, g32, dirs, None)
    probes = [oracle_grad(ws, rs, ds, cs, as_, g32, dirs, None, single=True, nudge=x) for x in (None, 1)]
    gsub = {"grad_root_state_in": g["grad_root_state_in"][idx], "grad_dof_state_in": rows(g["grad_dof_state_in"], nj),
            "grad_dof_actuation": rows(g["grad_dof_actuation"], nj), "grad_impulse_cache_in": g["grad_impulse_cache_in"][idx]}
    got = gpu_grad(ws, gsub, rs, dirs)
    bad = []
    for e in range(ws.n_envs):
        scale = max(1.0, np.abs(ref[e]).max())
        spread = max(np.abs(p[e] - ref[e]).max() for p in probes)
        if np.abs(got[e] - ref[e]).max() > 1e-3 * scale + K_COND * spread:
            bad.append(idx[e])
    print(f"ant x1024 (16 sampled envs, {len(dirs)} directions each): {len(bad)} outside the bound {bad}")
    assert len(bad) <= 1, bad
