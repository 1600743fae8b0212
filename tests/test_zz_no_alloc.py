"""sim_step_static_scratch, the step on caller-owned buffers with the library's built-in scratch
array (no device allocation in the call), against sim_step: the same seeded inputs, two calls in
a row, floating-point state within the parity tests' one-step bound (1e-4 relative, 1e-5
absolute), integer outputs identical, over the launch plans a handle can have; steps that would
use the handle's own views are refused. The file is collected last, so in a full run the entry
point is exercised after every other GPU test in the same process; alone it starts cold."""
import numpy as np
import pytest

from paper_2108_10470_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL, ATOL = 1e-4, 1e-5
FLOATS = ("root_state", "dof_state", "net_contact_force", "impulse_cache")
INTS = ("contact_pairs", "contact_count", "signature", "status")


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10470_gb300 import build
    build.build_library()
    torch.cuda.set_device(0)


def caller_buffers(s):
    """Zeroed device tensors shaped like the handle's views, owned by the caller (torch here)."""
    import torch
    out = {}
    for name in s.STATE_NAMES:
        v = getattr(s, name)
        dtype = torch.int32 if v.dtype not in (torch.float32, torch.int32) else v.dtype  # u32 as raw bits
        out[name] = torch.zeros(tuple(v.shape), dtype=dtype, device=v.device)
    return out


def as_np(t):
    a = t.cpu().numpy()
    return a.view(np.uint32) if a.dtype in (np.int32, np.uint32) else a.astype(np.float64)


def retune_ant_rows(s):
    """Move the Ant type's rows (type 0 of the mixed batch) to global scratch with 32 lanes per
    env: a retuned launch plan whose Ant envs then use the static array too."""
    s.set_type_config(0, 32, 1, 2)


@pytest.mark.parametrize("plan", ["per_type", "persistent", "graph", "retuned"])
def test_static_scratch_matches_sim_step(plan):
    """The same step on caller-owned buffers as sim_step on a handle of the same launch plan: the
    default per-type launches, a persistent handle, a CUDA-graph handle (both step here with one
    launch per type on the handle's stream) and a type whose knobs were changed."""
    import torch
    from paper_2108_10470_gb300 import sim

    flags = sim.SIM_FLAG_SIGNATURE | {"per_type": 0, "persistent": sim.SIM_FLAG_PERSISTENT,
                                      "graph": sim.SIM_FLAG_GRAPH, "retuned": 0}[plan]
    # Ant and Humanoid envs keep their rows in shared memory; hand-with-cube envs use the scratch
    w = W.mixed_workload(96)
    root, dof, acts = W.seeded_inputs(w, 5, 2)
    ref = sim.Sim(w, flags=flags)
    new = sim.Sim(w, flags=flags)
    if plan == "retuned":
        retune_ant_rows(ref)
        retune_ant_rows(new)
        assert new.type_config(0)["rows_global"] == 1
    ref.root_state.copy_(torch.from_numpy(root))
    ref.dof_state.copy_(torch.from_numpy(dof))
    bufs = caller_buffers(new)
    bufs["root_state"].copy_(torch.from_numpy(root))
    bufs["dof_state"].copy_(torch.from_numpy(dof))
    untouched = {name: as_np(getattr(new, name)) for name in FLOATS + INTS}
    for k in range(2):
        ref.dof_actuation.copy_(torch.from_numpy(acts[k]))
        ref.step()
        bufs["dof_actuation"].copy_(torch.from_numpy(acts[k]))
        new.step_static_scratch(bufs)
        torch.cuda.synchronize()
        for name in FLOATS:
            np.testing.assert_allclose(as_np(bufs[name]), as_np(getattr(ref, name)), rtol=RTOL, atol=ATOL,
                                       err_msg=f"{name} after call {k + 1}")
        for name in INTS:
            assert np.array_equal(as_np(bufs[name]), as_np(getattr(ref, name))), f"{name} after call {k + 1}"
        assert not as_np(bufs["status"]).any()
        hand_envs = [e for e in range(w.n_envs) if w.env_actor_count(e) == 2]
        assert (as_np(bufs["contact_count"])[hand_envs] > 0).all()
    # the handle's own views were neither read nor written
    for name in FLOATS + INTS:
        assert np.array_equal(as_np(getattr(new, name)), untouched[name]), name
    ref.destroy()
    new.destroy()


@pytest.mark.parametrize("case", ["dof_force", "rigid_body_state", "body_forces", "drives"])
def test_static_scratch_refuses_steps_that_use_handle_views(case):
    """Steps that would read the handle's control views or write its output views are refused with
    INVALID_ARG before any launch, leaving the caller's buffers as they were."""
    import torch
    from paper_2108_10470_gb300 import sim
    from test_gpu_control import driven_ant

    flags = {"dof_force": sim.SIM_FLAG_DOF_FORCE, "rigid_body_state": sim.SIM_FLAG_RIGID_BODY_STATE,
             "body_forces": sim.SIM_FLAG_BODY_FORCES, "drives": 0}[case]
    w = W.homogeneous("driven", driven_ant(), 8) if case == "drives" else W.ant_workload(8)
    root, dof, acts = W.seeded_inputs(w, 0, 1)
    s = sim.Sim(w, flags=sim.SIM_FLAG_SIGNATURE | flags)
    bufs = caller_buffers(s)
    bufs["root_state"].copy_(torch.from_numpy(root))
    bufs["dof_state"].copy_(torch.from_numpy(dof))
    bufs["dof_actuation"].copy_(torch.from_numpy(acts[0]))
    with pytest.raises(sim.SimError) as err:
        s.step_static_scratch(bufs)
    assert err.value.code == -1
    torch.cuda.synchronize()
    assert np.array_equal(bufs["root_state"].cpu().numpy(), root)
    s.destroy()


def test_static_scratch_rejects_a_type_beyond_its_size():
    """2048 hand-with-cube envs need about 124 MiB of scratch: refused before any launch, with the
    sizes in the message; a batch that fits then still steps."""
    import torch
    from paper_2108_10470_gb300 import sim

    s = sim.Sim(W.hand_workload(2048))
    bufs = caller_buffers(s)
    with pytest.raises(sim.SimError) as err:
        s.step_static_scratch(bufs)
    assert err.value.code == -4 and "static array" in str(err.value) and "envs of this type fit" in str(err.value)
    s.destroy()
    w = W.hand_workload(256)
    root, dof, acts = W.seeded_inputs(w, 0, 1)
    s = sim.Sim(w)
    bufs = caller_buffers(s)
    bufs["root_state"].copy_(torch.from_numpy(root))
    bufs["dof_state"].copy_(torch.from_numpy(dof))
    bufs["dof_actuation"].copy_(torch.from_numpy(acts[0]))
    s.step_static_scratch(bufs)
    torch.cuda.synchronize()
    assert not as_np(bufs["status"]).any()
    s.destroy()
