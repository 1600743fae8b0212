"""Host-only checks of the binding's argument marshalling: caller-owned device tensors handed to
the C ABI (the VJP / JVP buffers, the static-scratch state, the indexed setters) are checked for
dtype, contiguity, device and size before any library call, so a wrong tensor raises instead of
being read or written out of bounds by a kernel. Runs without a GPU: a handle-less Sim stands in,
its views replaced by CPU tensors of the right shapes."""
import numpy as np
import pytest
import torch

from paper_2108_10470_gb300 import sim, workloads as W


def fake_sim(n_envs=4):
    """A Sim whose views are CPU tensors shaped like a real handle's (no library, no device)."""
    w = W.ant_workload(n_envs)
    s = object.__new__(sim.Sim)
    s.w = w
    s._torch = torch
    s.h = None
    N_A, N_D, N_B, K, C = n_envs, 8 * n_envs, 9 * n_envs, 64, 17
    s.root_state = torch.zeros((N_A, 13))
    s.dof_state = torch.zeros((N_D, 2))
    s.dof_actuation = torch.zeros((N_D,))
    s.net_contact_force = torch.zeros((N_B, 3))
    s.impulse_cache = torch.zeros((n_envs, K))
    s.contact_pairs = torch.zeros((n_envs, C, 3), dtype=torch.int32)
    s.contact_count = torch.zeros((n_envs,), dtype=torch.int32)
    s.signature = torch.zeros((n_envs,), dtype=torch.int32)
    s.status = torch.zeros((n_envs,), dtype=torch.int32)
    return s


def good_state(s):
    return {k: torch.zeros_like(getattr(s, k)) for k in s.STATE_NAMES}


def test_valid_buffers_pass_the_checks():
    s = fake_sim()
    for k, t in good_state(s).items():
        assert s._mirror_ptr(t, k, k) == t.data_ptr()


@pytest.mark.parametrize("bad", ["dtype", "size", "contiguity", "device", "type"])
def test_static_scratch_buffers_are_checked(bad):
    s = fake_sim()
    bufs = good_state(s)
    if bad == "dtype":
        bufs["dof_state"] = bufs["dof_state"].double()
    elif bad == "size":
        bufs["impulse_cache"] = bufs["impulse_cache"][:-1]
    elif bad == "contiguity":
        bufs["root_state"] = torch.zeros((13, s.root_state.shape[0])).t()
    elif bad == "device":
        bufs["status"] = torch.zeros(s.status.shape, dtype=torch.int32, device="meta")
    else:
        bufs["dof_actuation"] = np.zeros(s.dof_actuation.shape, np.float32)
    with pytest.raises(ValueError):
        s.step_static_scratch(bufs)


def test_vjp_buffers_are_checked():
    """An int64 tensor where the ABI reads int32 (status), and a gradient buffer one element short,
    are refused before the call."""
    s = fake_sim()
    bufs = {"root_state": s.root_state.clone(), "dof_state": s.dof_state.clone(),
            "dof_actuation": s.dof_actuation.clone(), "impulse_cache": s.impulse_cache.clone(),
            "grad_root_state_in": torch.zeros_like(s.root_state), "grad_dof_state_in": torch.zeros_like(s.dof_state),
            "grad_dof_actuation": torch.zeros_like(s.dof_actuation),
            "grad_impulse_cache_in": torch.zeros_like(s.impulse_cache)}
    assert len(s._ptrs(sim.VJP_FIELDS, bufs)) == len(sim.VJP_FIELDS)
    with pytest.raises(ValueError):
        s._ptrs(sim.VJP_FIELDS, dict(bufs, status=torch.zeros(s.status.shape, dtype=torch.int64)))
    with pytest.raises(ValueError):
        s.step_vjp(dict(bufs, grad_dof_actuation=torch.zeros(s.dof_actuation.numel() - 1)))
    with pytest.raises(ValueError):
        s.step_jvp({"root_state": s.root_state.clone(), "tan_dof_state": torch.zeros((3, 2))})


def test_indexed_setters_check_index_dtype_and_source_size():
    s = fake_sim()
    idx64 = torch.tensor([0, 1])  # int64: would be read as int32 pairs
    with pytest.raises(ValueError):
        s.set_root_state_indexed(torch.zeros((2, 13)), idx64)
    with pytest.raises(ValueError):
        s.set_root_state_indexed(torch.zeros((1, 13)), torch.tensor([0, 1], dtype=torch.int32))
    with pytest.raises(ValueError):
        s.set_dof_state_indexed(torch.zeros((2, 15)), torch.tensor([0, 1], dtype=torch.int32))


@pytest.mark.parametrize("bad", ["dtype", "size", "contiguity", "device", "type"])
def test_step_actuated_buffer_is_checked(bad):
    """The actuation tensor of step_actuated: float32, contiguous, on the handle's device (or pinned
    host memory), with at least N_D elements; anything else raises before the library is called."""
    s = fake_sim()
    act = torch.zeros(s.dof_actuation.shape)
    if bad == "dtype":
        act = act.double()
    elif bad == "size":
        act = act[:-1]
    elif bad == "contiguity":
        act = torch.zeros((2, act.shape[0]))[:, 0]
    elif bad == "device":
        act = torch.zeros(act.shape, device="meta")
    else:
        act = np.zeros(act.shape, np.float32)
    with pytest.raises(ValueError):
        s.step_actuated(act)
