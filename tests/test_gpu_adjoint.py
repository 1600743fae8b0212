"""The step's derivative on the GPU (sim_step_jvp / sim_step_vjp and the autograd wrappers) against
the FP64 oracle's forward-mode derivative.

Bounds. The serial step's value is checked like the forward kernel (strict bound plus 16 times the
env's FP32 conditioning scale). A derivative is compared per env in the max norm relative to the
env's derivative scale, with the bound 1e-3 + 16 times its FP32 conditioning scale: the largest
deviation from the FP64 derivative of the oracle's own derivative evaluated in single precision at
inputs nudged by one float32 ulp. Where FP32 and FP64 take different branches (a clamp or target
switch within rounding of its threshold, which the constraint-set signature does not capture) the
derivative jumps: such envs are counted and reported, and at most 5 % of the checked envs may be
outside the bound.
"""
import numpy as np
import pytest

import oracle
from paper_2108_10470_gb300 import workloads as W
from parity_util import _ulp

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


def warm(w, seed=0, steps=3):
    """Seeded state after a few oracle steps, with its warm impulse cache (FP64, float32-rounded)."""
    root, dof, acts = W.seeded_inputs(w, seed, steps + 1)
    O = oracle.Oracle(w)
    r, d = root.astype(np.float64), dof.astype(np.float64)
    for k in range(steps):
        O.step(r, d, acts[k])
    f = lambda x: x.astype(np.float32).astype(np.float64)
    return f(r), f(d), f(O.cache), acts[steps].astype(np.float64)


def direction(w, r, cache, rng):
    """Random input tangent. Orientations move along the unit sphere (dq = [w; 0] q / 2): off it the
    step's dependence on the quaternion's norm is an artefact of the formulation (the GPU works in
    world axes, the oracle in body coordinates; they agree for unit quaternions only)."""
    dr = rng.standard_normal(r.shape)
    om = rng.standard_normal((r.shape[0], 3))
    q = r[:, 3:7]
    # [om; 0] (x) q, Hamilton product with (x, y, z, w) storage
    dr[:, 3] = 0.5 * (om[:, 0] * q[:, 3] + om[:, 1] * q[:, 2] - om[:, 2] * q[:, 1])
    dr[:, 4] = 0.5 * (-om[:, 0] * q[:, 2] + om[:, 1] * q[:, 3] + om[:, 2] * q[:, 0])
    dr[:, 5] = 0.5 * (om[:, 0] * q[:, 1] - om[:, 1] * q[:, 0] + om[:, 2] * q[:, 3])
    dr[:, 6] = 0.5 * (-om[:, 0] * q[:, 0] - om[:, 1] * q[:, 1] - om[:, 2] * q[:, 2])
    dd = rng.standard_normal((w.n_dof, 2))
    da = rng.standard_normal(w.n_dof)
    dc = rng.standard_normal(cache.shape) * (cache != 0)
    return dr, dd, da, dc


def oracle_tangent(w, r, d, c, a, t, single=False, nudge=None, ctl=None):
    O = oracle.Oracle(w)
    r, d = r.copy(), d.copy()
    if nudge is not None:
        r[:, :3] = _ulp(r[:, :3], nudge)
        d[:, 0] = _ulp(d[:, 0], -nudge)
    O.cache[:] = c
    tr, td, tc = t[0].copy(), t[1].copy(), t[3].copy()
    O.step_tangent(r, d, a, tr, td, t[2], tc, single=single, **(ctl or {}))
    return r, d, O.cache.copy(), tr, td, tc


def gpu_jvp(s, r, d, c, a, t):
    import torch
    f = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    bufs = {"root_state": f(r), "dof_state": f(d), "dof_actuation": f(a), "impulse_cache": f(c),
            "tan_root_state": f(t[0]), "tan_dof_state": f(t[1]), "tan_dof_actuation": f(t[2]),
            "tan_impulse_cache": f(t[3]), "status": torch.zeros(s.w.n_envs, dtype=torch.int32, device="cuda")}
    for k, v in (("root_state_out", r), ("dof_state_out", d), ("impulse_cache_out", c), ("tan_root_state_out", r),
                 ("tan_dof_state_out", d), ("tan_impulse_cache_out", c)):
        bufs[k] = torch.zeros(v.shape, dtype=torch.float32, device="cuda")
    s.step_jvp(bufs)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in bufs.items()}
    return g


def env_slices(w):
    ra = np.cumsum([0] + [w.env_actor_count(e) for e in range(w.n_envs)])
    rd = np.cumsum([0] + [w.env_jdof(e) for e in range(w.n_envs)])
    return [(slice(ra[e], ra[e + 1]), slice(rd[e], rd[e + 1]), slice(e, e + 1)) for e in range(w.n_envs)]


def env_max(arrs, sl):
    return max(float(np.abs(x[s]).max()) if x[s].size else 0.0 for x, s in zip(arrs, sl))


def _driven_ant(n):
    from test_gpu_control import driven_ant
    return W.homogeneous("ant_driven", driven_ant(), n)


WORKLOADS = {"ant": W.ant_workload, "humanoid": W.humanoid_workload, "cartpole": W.cartpole_workload,
             "ball_ant": lambda n: W.homogeneous("ball_ant", W.ant(ball_hips=True), n), "driven_ant": _driven_ant,
             "pushed_ant": W.ant_workload,
             "tendon_ant": lambda n: W.homogeneous("tendon_ant", W.ant(tendons=True), n),
             "hand": W.hand_workload, "hand_tendon": W.hand_tendon_workload,
             "ball_humanoid": lambda n: W.homogeneous("ball_humanoid", W.humanoid(ball_joints=True), n)}


def make_sim(name, w, seed=9):
    """The handle for a workload and the controls it carries (random per-env drive targets for
    driven_ant, random external body forces for pushed_ant: constants of the derivative), as the
    oracle's keyword arguments (values rounded to FP32 like the views)."""
    import torch
    from paper_2108_10470_gb300 import sim
    rng = np.random.default_rng(seed)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)
    t32 = lambda x: torch.from_numpy(x.astype(np.float32))
    if name == "driven_ant":
        s = sim.Sim(w)
        ctl = dict(pos_target=r32(rng.uniform(-0.3, 0.3, w.n_dof)), vel_target=r32(rng.uniform(-0.5, 0.5, w.n_dof)))
        s.dof_position_target.copy_(t32(ctl["pos_target"]))
        s.dof_velocity_target.copy_(t32(ctl["vel_target"]))
        return s, ctl
    if name == "pushed_ant":
        s = sim.Sim(w, flags=sim.SIM_FLAG_BODY_FORCES)
        ctl = dict(body_force=r32(rng.uniform(-3.0, 3.0, (w.n_body, 6))))
        s.rigid_body_force.copy_(t32(ctl["body_force"]))
        return s, ctl
    return sim.Sim(w), None


@pytest.mark.parametrize("name,n", [("ant", 67), ("humanoid", 37), ("cartpole", 67), ("ball_ant", 40),
                                    ("driven_ant", 40), ("pushed_ant", 40), ("tendon_ant", 40), ("hand", 24),
                                    ("hand_tendon", 16)])
def test_jvp_value_and_tangent_match_oracle(name, n):
    """(driven_ant / pushed_ant: drive targets / body forces from the handle's views, constants of
    the derivative)"""
    w = WORKLOADS[name](n)
    r, d, c, a = warm(w, seed=1)
    t = direction(w, r, c, np.random.default_rng(2))
    s, ctl = make_sim(name, w)
    g = gpu_jvp(s, r, d, c, a, t)
    s.destroy()
    assert not g["status"].any()
    ref = oracle_tangent(w, r, d, c, a, t, ctl=ctl)
    probes = [oracle_tangent(w, r, d, c, a, t, single=True, nudge=x, ctl=ctl) for x in (None, 1, -1)]
    val_keys = ("root_state_out", "dof_state_out", "impulse_cache_out")
    tan_keys = ("tan_root_state_out", "tan_dof_state_out", "tan_impulse_cache_out")
    bad_val, bad_tan, checked = [], [], 0
    for e, sl in enumerate(env_slices(w)):
        checked += 1
        # value: strict bound 1e-4 relative / 1e-5 absolute plus the FP32 scale
        vscale = max(env_max([p[i] - ref[i] for i in range(3)], sl) for p in probes)
        vdev = max(float(np.max(np.abs(g[k][s_] - ref[i][s_]) - (1e-5 + 1e-4 * np.abs(ref[i][s_])), initial=-1))
                   for i, (k, s_) in enumerate(zip(val_keys, sl)))
        if vdev > K_COND * vscale:
            bad_val.append(e)
        tscale = max(1.0, env_max(ref[3:], sl))
        tcond = max(env_max([p[3 + i] - ref[3 + i] for i in range(3)], sl) for p in probes)
        tdev = max(float(np.abs(g[k][s_] - ref[3 + i][s_]).max(initial=0.0)) for i, (k, s_) in enumerate(zip(tan_keys, sl)))
        if tdev > 1e-3 * tscale + K_COND * tcond:
            bad_tan.append(e)
    print(f"{name} x{n}: value outside bound in {len(bad_val)} envs, tangent outside bound in {len(bad_tan)} envs")
    assert len(bad_val) <= 0.05 * checked, bad_val
    assert len(bad_tan) <= 0.05 * checked, bad_tan


@pytest.mark.parametrize("name,n", [("ant", 40), ("humanoid", 20), ("ball_ant", 20), ("driven_ant", 20),
                                    ("pushed_ant", 20), ("tendon_ant", 20), ("hand", 12)])
def test_vjp_is_the_transpose_of_the_jvp(name, n):
    """<g, J u> (tangent mode) equals <J^T g, u> (adjoint mode) per env, for random g and u."""
    import torch
    from paper_2108_10470_gb300 import sim
    w = WORKLOADS[name](n)
    r, d, c, a = warm(w, seed=3)
    rng = np.random.default_rng(4)
    u = direction(w, r, c, rng)
    gout = (rng.standard_normal(r.shape), rng.standard_normal(d.shape), rng.standard_normal(c.shape) * (c != 0))
    s, _ = make_sim(name, w)
    jv = gpu_jvp(s, r, d, c, a, u)
    f = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    bufs = {"root_state": f(r), "dof_state": f(d), "dof_actuation": f(a), "impulse_cache": f(c),
            "grad_root_state": f(gout[0]), "grad_dof_state": f(gout[1]), "grad_impulse_cache": f(gout[2]),
            "grad_root_state_in": torch.zeros_like(f(r)), "grad_dof_state_in": torch.zeros_like(f(d)),
            "grad_dof_actuation": torch.zeros_like(f(a)), "grad_impulse_cache_in": torch.full_like(f(c), 7.0)}
    s.step_vjp(bufs)
    torch.cuda.synchronize()
    s.destroy()
    gi = [bufs[k].cpu().numpy().astype(np.float64) for k in ("grad_root_state_in", "grad_dof_state_in",
                                                             "grad_dof_actuation", "grad_impulse_cache_in")]
    u32 = [x.astype(np.float32).astype(np.float64) for x in u]
    g32 = [x.astype(np.float32).astype(np.float64) for x in gout]
    for e, (ra, rd, rc) in enumerate(env_slices(w)):
        lhs = float((g32[0][ra] * jv["tan_root_state_out"][ra]).sum() + (g32[1][rd] * jv["tan_dof_state_out"][rd]).sum()
                    + (g32[2][rc] * jv["tan_impulse_cache_out"][rc]).sum())
        rhs = float((gi[0][ra] * u32[0][ra]).sum() + (gi[1][rd] * u32[1][rd]).sum() + (gi[2][rd] * u32[2][rd]).sum()
                    + (gi[3][rc] * u32[3][rc]).sum())
        scale = float(np.abs(gi[0][ra]).sum() + np.abs(gi[1][rd]).sum() + np.abs(gi[2][rd]).sum() + np.abs(gi[3][rc]).sum())
        assert abs(lhs - rhs) <= 1e-4 * max(1.0, scale), (e, lhs, rhs, scale)


def loss_grad_gpu(w, root, dof, acts, checkpoint, keep_tapes=None):
    import torch
    from paper_2108_10470_gb300 import autograd as AG, sim
    s = sim.Sim(w)
    r0 = torch.from_numpy(root.astype(np.float32)).cuda()
    d0 = torch.from_numpy(dof.astype(np.float32)).cuda().requires_grad_(True)
    c0 = torch.zeros((w.n_envs, s.cache_len), device="cuda")
    A = torch.from_numpy(acts.astype(np.float32)).cuda().requires_grad_(True)
    rf, df, cf = AG.rollout(s, r0, d0, c0, A, checkpoint=checkpoint, keep_tapes=keep_tapes)
    loss = rf[:, 7].mean()  # mean final root x-velocity
    loss.backward()
    # whether the backward pass re-ran the segments on the handle or used the tapes the forward
    # pass kept, its views are at the final state
    assert torch.equal(s.root_state, rf.detach()) and torch.equal(s.dof_state, df.detach())
    assert torch.equal(s.impulse_cache, cf.detach())
    out = (float(loss), d0.grad.cpu().numpy().astype(np.float64), A.grad.cpu().numpy().astype(np.float64),
           rf.detach().cpu().numpy())
    s.destroy()
    return out


def loss_grad_oracle(w, root, dof, acts):
    """d(mean final root v_x over all actors)/d(actions) and /d(initial DOF state) by forward mode:
    one dual rollout per input direction, seeded in every env at once (envs are independent)."""
    steps = acts.shape[0]
    nj = w.n_dof // w.n_envs
    g_act = np.zeros((steps, w.n_dof))
    g_dof = np.zeros((w.n_dof, 2))

    def run(seed_step, seed_j, seed_dof_comp):
        O = oracle.Oracle(w)
        r, d = root.astype(np.float64), dof.astype(np.float64)
        tr, td, tc = np.zeros_like(r), np.zeros_like(d), np.zeros_like(O.cache)
        if seed_dof_comp is not None:
            td[seed_j::nj, seed_dof_comp] = 1.0
        for k in range(steps):
            da = np.zeros(w.n_dof)
            if seed_step == k:
                da[seed_j::nj] = 1.0
            O.step_tangent(r, d, acts[k].astype(np.float64), tr, td, da, tc)
        return (tr[:, 7] / tr.shape[0]).reshape(w.n_envs, -1).sum(1)  # mean over actors, per env

    for k in range(steps):
        for j in range(nj):
            g_act[k, j::nj] = run(k, j, None)
    for j in range(nj):
        for comp in range(2):
            g_dof[j::nj, comp] = run(None, j, comp)
    return g_dof, g_act


@pytest.mark.parametrize("name,steps,max_bad", [("ant", 12, 1), ("hand", 6, 2)])
def test_rollout_gradient_matches_oracle_and_checkpointing_is_exact(name, steps, max_bad):
    """8 envs (Ant over 12 steps; the hand holding its cube over 6), loss = mean final root
    x-velocity: gradients w.r.t. every action and the initial DOF state through the autograd rollout
    (checkpoints of 4 steps) against the oracle's forward-mode rollout; checkpoint lengths 1, 4 and
    the whole rollout, with the tapes kept from the forward pass or recomputed, give bitwise equal
    gradients (both through the reverse pass, the hand's with its capsule-box pair contacts).
    max_bad envs may deviate by more than 1e-2: the hand's contact-rich rollouts include an env
    whose derivative evaluated in single precision by the oracle itself lands 8e-2 from its FP64
    value (a clamp within rounding of its threshold)."""
    w = W.ant_workload(8) if name == "ant" else W.hand_workload(8)
    root, dof, acts = W.seeded_inputs(w, 11, steps)
    l4, gd4, ga4, _ = loss_grad_gpu(w, root, dof, acts, 4, keep_tapes=False)
    for ck, keep in ((1, False), (steps, False), (4, True), (steps, True), (4, None)):
        l, gd, ga, _ = loss_grad_gpu(w, root, dof, acts, ck, keep_tapes=keep)
        assert l == l4 and np.array_equal(gd, gd4) and np.array_equal(ga, ga4), (ck, keep)
    od, oa = loss_grad_oracle(w, root, dof, acts)
    nj = w.n_dof // w.n_envs
    bad = []
    for e in range(w.n_envs):
        gpu = np.concatenate([gd4[e * nj:(e + 1) * nj].ravel(), ga4[:, e * nj:(e + 1) * nj].ravel()])
        ref = np.concatenate([od[e * nj:(e + 1) * nj].ravel(), oa[:, e * nj:(e + 1) * nj].ravel()])
        rel = np.abs(gpu - ref).max() / max(np.abs(ref).max(), 1e-12)
        print(f"env {e}: max |grad| {np.abs(ref).max():.3e}, relative deviation {rel:.2e}")
        if rel > 1e-2:
            bad.append(e)
    assert len(bad) <= max_bad, bad


def test_rollout_gradient_matches_central_differences():
    """The differentiable-rollout workload's check: the GPU gradient of loss = mean final root
    x-velocity of a 12-step, 8-env Ant rollout (through the autograd rollout and the reverse pass)
    against central finite differences with h = 1e-4 of the FP64 oracle's rollout, w.r.t. the
    actions of steps 0, 5 and 11 and the initial DOF positions and velocities. A difference counts
    where the rollout is smooth over +-h: every step's constraint set is that of the unperturbed
    rollout under both perturbations, and the difference agrees with the one at h / 4 to 1e-3 of
    the env's gradient scale (the derivative holds the solver's clamps at the forward pass's
    choices, which the constraint set does not record: within 1e-4 of some initial joint positions
    a friction or impulse clamp switches over the 12 steps). Envs are independent, so each
    direction perturbs the same component in every env at once."""
    w = W.ant_workload(8)
    steps, h = 12, 1e-4
    root, dof, acts = W.seeded_inputs(w, 11, steps)
    _, gd, ga, _ = loss_grad_gpu(w, root, dof, acts, 4)
    nj = w.n_dof // w.n_envs

    def rollout(d_act=None, d_dof=None):
        O = oracle.Oracle(w)
        r, d = root.astype(np.float64), dof.astype(np.float64)
        if d_dof is not None:
            d += d_dof
        sigs = []
        for k in range(steps):
            a = acts[k].astype(np.float64) + (d_act[k] if d_act is not None else 0.0)
            sigs.append(O.step(r, d, a)["signature"].copy())
        return r[:, 7].copy(), np.array(sigs)  # per env (one actor each): final v_x; signatures

    _, base_sig = rollout()

    def central(make):  # d loss / d(component), per env, at h and h / 4; constraint sets kept at +-h
        (vp, sp), (vm, sm) = rollout(**make(h)), rollout(**make(-h))
        (vq, _), (vn, _) = rollout(**make(h / 4)), rollout(**make(-h / 4))
        same = (sp == base_sig).all(0) & (sm == base_sig).all(0)
        return (vp - vm) / (2 * h * w.n_envs), (vq - vn) / (h / 2 * w.n_envs), same

    fd, fd4, same, gpu = [], [], [], []
    for k in (0, 5, 11):
        for j in range(nj):
            def act(x, k=k, j=j):
                da = np.zeros((steps, w.n_dof))
                da[k, j::nj] = x
                return {"d_act": da}
            a, b, c = central(act)
            fd.append(a), fd4.append(b), same.append(c), gpu.append(ga[k, j::nj])
    for j in range(nj):
        for comp in range(2):
            def ini(x, j=j, comp=comp):
                dd = np.zeros((w.n_dof, 2))
                dd[j::nj, comp] = x
                return {"d_dof": dd}
            a, b, c = central(ini)
            fd.append(a), fd4.append(b), same.append(c), gpu.append(gd[j::nj, comp])
    fd, fd4, same, gpu = (np.array(x) for x in (fd, fd4, same, gpu))  # (directions, envs)
    bad, checked = [], 0
    for e in range(w.n_envs):
        scale = max(np.abs(fd4[:, e]).max(), 1e-12)
        m = same[:, e] & (np.abs(fd[:, e] - fd4[:, e]) <= 1e-3 * scale)
        if m.any():  # the scale of the smooth directions alone, and the mask again with it
            scale = max(np.abs(fd4[m, e]).max(), 1e-12)
            m = same[:, e] & (np.abs(fd[:, e] - fd4[:, e]) <= 1e-3 * scale)
        if m.sum() < len(m) // 2:
            continue  # no smooth neighbourhood in most directions
        checked += 1
        rel = np.abs(gpu[m, e] - fd[m, e]).max() / scale
        print(f"env {e}: {int(m.sum())} of {len(m)} directions smooth over +-h, gradient scale {scale:.3e}, "
              f"relative deviation from central differences {rel:.2e}")
        if rel > 1e-2:
            bad.append(e)
    assert checked >= w.n_envs // 2 and len(bad) <= 1, (checked, bad)


def many_boxes(n_boxes=19):
    """A free body carrying n_boxes box shapes (8 ground candidates each) and a hinged child: 19
    boxes give an impulse cache of 3 * 152 + 2 = 458 entries, past the derivative's 448."""
    b = W._Builder("boxes")
    root = b.link(-1, W.JOINT_FREE, mass=1.0, inertia=(0.1, 0.1, 0.1, 0, 0, 0))
    b.link(root, W.JOINT_REVOLUTE, axis=(0, 0, 1), ppos=(0.0, 0.2, 0.0), mass=0.1, inertia=(0.01, 0.01, 0.01, 0, 0, 0))
    for i in range(n_boxes):
        b.shape(root, W.SHAPE_BOX, (0.05, 0.05, 0.05), pos=(0.1 * i, 0.0, 0.0))
    return b.build(root_pos=(0.0, 0.0, 1.0))


def test_forward_mode_refuses_large_caches_the_reverse_pass_does_not():
    """An impulse cache past 448 entries: the forward-mode kernel (SIM_FLAG_TANGENT_VJP) refuses the
    handle with CAPACITY; the reverse pass, which keeps no per-lane copy of the cache, differentiates it."""
    import torch
    from paper_2108_10470_gb300 import sim
    w = W.homogeneous("boxes", many_boxes(), 4)
    for flags in (sim.SIM_FLAG_TANGENT_VJP, 0):
        s = sim.Sim(w, flags=flags)
        assert s.cache_len > 448
        z = lambda v: torch.zeros_like(v)
        bufs = {"root_state": s.root_state, "dof_state": s.dof_state, "dof_actuation": s.dof_actuation,
                "impulse_cache": s.impulse_cache, "grad_root_state": torch.ones_like(s.root_state),
                "grad_root_state_in": z(s.root_state), "grad_dof_state_in": z(s.dof_state),
                "grad_dof_actuation": z(s.dof_actuation), "grad_impulse_cache_in": z(s.impulse_cache),
                "status": torch.full((w.n_envs,), 9, dtype=torch.int32, device="cuda")}
        if flags:
            with pytest.raises(sim.SimError) as err:
                s.step_vjp(bufs)
            assert err.value.code == -4
        else:
            s.step_vjp(bufs)
            torch.cuda.synchronize()
            assert not bufs["status"].any() and torch.isfinite(bufs["grad_root_state_in"]).all()
            assert bufs["grad_root_state_in"][:, 2].abs().sum() > 0  # the height reaches the output
        s.destroy()
