"""GPU parity at the kernel's capacity limits and across lane widths: random articulated trees (mixed
revolute / prismatic joints, random frames, axes and inertias) with 32 links and 31 joint DOFs on
a fixed base, 27 links and 32 generalized DOFs on a floating base, a batch mixing tree sizes
that map to 8, 16 and 32 lanes per env, and substeps with more constraint rows than the shared Y
region of a 32-lane env holds (Y in the group's global slot: bit for bit the same steps as with the
whole row capacity in shared memory)."""
import numpy as np
import pytest

from paper_2108_10470_gb300 import workloads as W
from scenes import capsule_chain
from test_gpu_parity import check_rollout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10470_gb300 import build
    build.build_library()
    torch.cuda.set_device(0)


def tree(seed, n_links, floating):
    m = W.random_tree(np.random.default_rng(seed), n_links, floating, allow_fixed=False)
    m.armature = np.full(m.n_links, 0.05)  # keep the joint-space inertia well conditioned
    return m


@pytest.mark.parametrize("n_links,floating", [(32, False), (27, True)])
@pytest.mark.parametrize("steps,rtol,atol", [(1, 1e-4, 1e-5), (16, 1e-3, 1e-3)])
def test_largest_trees(n_links, floating, steps, rtol, atol):
    m = tree(11, n_links, floating)
    assert m.n_links <= 32 and m.n_gen <= 32 and (m.n_gen == 32 or m.n_links == 32)
    w = W.homogeneous("tree", m, 37)
    check_rollout(w, steps, rtol, atol, min_same=1.0)


def test_mixed_lane_widths():
    models = [tree(1, 5, False), tree(2, 12, False), tree(3, 24, True)]  # 8, 16 and 32 lanes
    eam = np.array([i % 3 for i in range(60)], np.int32)
    w = W.Workload("trees", models, eam, 1, 60, W.Params())
    check_rollout(w, 4, 1e-3, 1e-3, min_same=1.0)


def staggered(w):
    """Lift env e's chain by 4 mm x (e mod 10): one launch then steps envs without contacts, with a
    few and with up to 34 (102 rows and more)."""
    def start(root, dof):
        root[:, 2] += 0.004 * (np.arange(w.n_envs) % 10)
    return start


def shared_rows(s):
    s.set_type_config(0, 32, 0, 4)
    assert s.type_config(0)["rows_global"] == 0


def test_persistent_global_y_slots_match_per_type_launch():
    """The persistent launch gives every resident warp its own global Y slot (the per-type launch
    one per env): 4 steps of the capsule chain, whose substeps put Y past 33 rows in those slots,
    agree with the per-type launch's to rounding (1e-4 relative, 1e-5 absolute) and in every
    integer output."""
    import torch
    from paper_2108_10470_gb300 import sim

    w = W.homogeneous("capsule_chain", capsule_chain(), 37)
    root, dof, acts = W.seeded_inputs(w, 2, 4)
    staggered(w)(root, dof)
    a = sim.Sim(w, flags=sim.SIM_FLAG_SIGNATURE)
    b = sim.Sim(w, flags=sim.SIM_FLAG_SIGNATURE | sim.SIM_FLAG_PERSISTENT)
    most = 0
    for s in (a, b):
        shared_rows(s)
        s.root_state.copy_(torch.from_numpy(root))
        s.dof_state.copy_(torch.from_numpy(dof))
    for k in range(4):
        for s in (a, b):
            s.dof_actuation.copy_(torch.from_numpy(acts[k]))
            s.step()
        for name in a.STATE_NAMES:
            x, y = getattr(a, name), getattr(b, name)
            if x.dtype == torch.float32:
                assert torch.allclose(x, y, rtol=1e-4, atol=1e-5), (name, k, (x - y).abs().max().item())
            else:
                assert np.array_equal(x.cpu().numpy(), y.cpu().numpy()), (name, k)
        most = max(most, int(a.contact_count.max()))
    assert most >= 12 and not a.status.any() and not b.status.any()
    a.destroy()
    b.destroy()


def test_global_y_slot_is_bitwise_the_shared_region():
    """Where Y lives does not change the arithmetic: with the row form of the solve forced (so
    that the Delassus form's fit, which depends on the region's size, plays no part), 16 steps of
    the capsule chain with Y past 33 rows in global slots equal, bit for bit, the same steps with
    the whole row capacity in shared memory (sim_step_static_scratch lays such a type out that
    way)."""
    import torch
    from paper_2108_10470_gb300 import sim

    w = W.homogeneous("capsule_chain", capsule_chain(), 37)
    root, dof, acts = W.seeded_inputs(w, 1, 16)
    staggered(w)(root, dof)
    flags = sim.SIM_FLAG_SIGNATURE | sim.SIM_FLAG_ROW_SOLVER
    a, b = sim.Sim(w, flags=flags), sim.Sim(w, flags=flags)
    shared_rows(a)
    shared_rows(b)
    a.root_state.copy_(torch.from_numpy(root))
    a.dof_state.copy_(torch.from_numpy(dof))
    def raw(t):  # the bits of a float32 / int32 / uint32 tensor
        return t.cpu().numpy().view(np.uint32)

    bufs = {}
    for name in b.STATE_NAMES:
        v = getattr(b, name)
        dtype = v.dtype if v.dtype in (torch.float32, torch.int32) else torch.int32  # u32 as raw bits
        bufs[name] = torch.zeros(tuple(v.shape), dtype=dtype, device=v.device)
    bufs["root_state"].copy_(torch.from_numpy(root))
    bufs["dof_state"].copy_(torch.from_numpy(dof))
    most = 0
    for k in range(16):
        a.dof_actuation.copy_(torch.from_numpy(acts[k]))
        a.step()
        bufs["dof_actuation"].copy_(torch.from_numpy(acts[k]))
        b.step_static_scratch(bufs)
        for name in b.STATE_NAMES:
            assert np.array_equal(raw(getattr(a, name)), raw(bufs[name])), f"{name} after step {k + 1}"
        most = max(most, int(a.contact_count.max()))
    assert most >= 12 and not a.status.any()
    a.destroy()
    b.destroy()


def test_reverse_pass_with_global_y_slots():
    """The reverse pass of steps whose Y lies in the global slots (the taped step records Y from
    wherever the step keeps it): four taped steps of the staggered capsule chain equal the plain
    steps bit for bit, and one step's vector-Jacobian product through the tape and the adjoint
    kernel agrees with the forward-mode kernel (which keeps no Y) as in the reverse-pass tests."""
    import torch
    from paper_2108_10470_gb300 import sim
    from test_gpu_adjoint import warm
    from test_gpu_reverse import STATE, directions, gpu_grad, gpu_vjp, output_gradient

    w = W.homogeneous("capsule_chain", capsule_chain(), 16)
    root, dof, acts = W.seeded_inputs(w, 5, 4)
    staggered(w)(root, dof)
    ref, tap = sim.Sim(w, flags=sim.SIM_FLAG_SIGNATURE), sim.Sim(w, flags=sim.SIM_FLAG_SIGNATURE)
    for s in (ref, tap):
        shared_rows(s)
        s.root_state.copy_(torch.from_numpy(root))
        s.dof_state.copy_(torch.from_numpy(dof))
    tape = torch.empty(tap.tape_floats(), device="cuda")
    for k in range(4):
        for s in (ref, tap):
            s.dof_actuation.copy_(torch.from_numpy(acts[k]))
        ref.step()
        tap.step_taped(tape)
        torch.cuda.synchronize()
        for v in STATE:
            assert torch.equal(getattr(ref, v), getattr(tap, v)), (v, k)
    assert int(ref.contact_count.max()) >= 12
    ref.destroy()
    tap.destroy()

    r, d, c, a = warm(w, seed=7)  # 7 to 34 contacts per env: Y in the shared region or the global slot
    gout = output_gradient(w, r, d, c, np.random.default_rng(8))
    s = sim.Sim(w)
    shared_rows(s)
    assert s.tape_floats() is not None  # the reverse pass covers the type
    g_rev = gpu_vjp(s, r, d, c, a, gout)
    s.destroy()
    s = sim.Sim(w, flags=sim.SIM_FLAG_TANGENT_VJP)
    g_fwd = gpu_vjp(s, r, d, c, a, gout)
    s.destroy()
    dirs = directions(w, r, c)
    A, B = gpu_grad(w, g_rev, r, dirs), gpu_grad(w, g_fwd, r, dirs)
    rel = np.abs(A - B).max(1) / np.maximum(1.0, np.abs(B).max(1))
    print(f"capsule chain x16: reverse vs forward mode, relative deviation median {np.median(rel):.2e}, "
          f"max {rel.max():.2e}")
    assert (rel > 1e-2).sum() <= 1 and np.median(rel) <= 1e-3
