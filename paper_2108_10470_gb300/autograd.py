"""Differentiable env-steps for PyTorch: torch.autograd.Function wrappers around the C ABI.

The carried state is (root state, DOF state, impulse cache); the actuation is the per-step
control. The forward value is the CUDA step kernel; the backward pass is the step's
vector-Jacobian product with the step's constraint and active sets held fixed: the reverse pass
(sim_step_taped records each re-run step's tape, sim_step_adjoint applies the adjoints in reverse
order) where it covers the handle, else sim_step_vjp in forward mode.

`rollout` chains env-steps in segments of `checkpoint` steps, with one of two memory policies per
rollout. Tapes kept: the forward pass records every step's tape (sim_step_taped: the same values
as sim_step, bit for bit) and keeps it on the device, and the backward pass only applies the
adjoints. Recomputation (checkpointing): each segment keeps only its input state, and the
backward pass re-runs its steps with their tapes recorded before applying the adjoints. By default
the tapes are kept when all of the rollout's tapes take at most a quarter of the device's free
memory (1024 Ant-like envs: 18.6 MB per step). The forward pass leaves the handle's views at the
rollout's final state; a backward pass that recomputes restores them afterwards.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import sim as _sim


def _zeros_like_views(s):
    return (torch.zeros_like(s.root_state), torch.zeros_like(s.dof_state), torch.zeros_like(s.impulse_cache))


def _forward_steps(s, root, dof, cache, acts, keep_inputs):
    """Advance the state through len(acts) steps on the handle's own buffers; optionally keep every
    step's input state."""
    s.root_state.copy_(root)
    s.dof_state.copy_(dof)
    s.impulse_cache.copy_(cache)
    inputs = []
    for k in range(acts.shape[0]):
        if keep_inputs:
            inputs.append((s.root_state.clone(), s.dof_state.clone(), s.impulse_cache.clone()))
        s.dof_actuation.copy_(acts[k])
        s.step()
    return (s.root_state.clone(), s.dof_state.clone(), s.impulse_cache.clone()), inputs


def _vjp(s, root, dof, cache, act, g_root, g_dof, g_cache):
    gi_root, gi_dof, gi_cache = _zeros_like_views(s)
    gi_act = torch.zeros_like(s.dof_actuation)
    s.step_vjp({"root_state": root, "dof_state": dof, "dof_actuation": act, "impulse_cache": cache,
                "grad_root_state": g_root.contiguous(), "grad_dof_state": g_dof.contiguous(),
                "grad_impulse_cache": g_cache.contiguous(), "grad_root_state_in": gi_root,
                "grad_dof_state_in": gi_dof, "grad_dof_actuation": gi_act, "grad_impulse_cache_in": gi_cache})
    return gi_root, gi_dof, gi_cache, gi_act


def keep_tapes_by_default(s, steps: int) -> bool:
    """The default policy: keep the tapes when the reverse pass covers the handle and `steps`
    steps' tapes take at most a quarter of the device's free memory."""
    tf = s.tape_floats()
    if tf is None:
        return False
    free, _ = torch.cuda.mem_get_info(s.root_state.device)
    return 4 * tf * steps <= free // 4


class Segment(torch.autograd.Function):
    """`acts.shape[0]` env-steps from (root, dof, cache); returns the final state. With keep_tapes
    the steps' tapes are recorded now and kept for the backward pass."""

    @staticmethod
    def forward(ctx, s, keep_tapes, root, dof, cache, acts):
        ctx.tapes = None
        with torch.no_grad():
            tf = s.tape_floats() if keep_tapes else None
            if tf is not None:
                ctx.tapes = torch.empty((acts.shape[0], max(tf, 1)), dtype=torch.float32, device=root.device)
                s.root_state.copy_(root)
                s.dof_state.copy_(dof)
                s.impulse_cache.copy_(cache)
                s.record_tapes(ctx.tapes, acts.contiguous())
                out = (s.root_state.clone(), s.dof_state.clone(), s.impulse_cache.clone())
            else:
                out, _ = _forward_steps(s, root, dof, cache, acts, keep_inputs=False)
        ctx.s = s
        ctx.save_for_backward(root, dof, cache, acts)
        return out

    @staticmethod
    def backward(ctx, g_root, g_dof, g_cache):
        s = ctx.s
        root, dof, cache, acts = ctx.saved_tensors
        if ctx.tapes is not None:  # tapes kept: the adjoints alone (the handle's views are not touched)
            with torch.no_grad():
                g_acts = torch.zeros_like(acts)
                g = (g_root.contiguous() if g_root is not None else torch.zeros_like(root),
                     g_dof.contiguous() if g_dof is not None else torch.zeros_like(dof),
                     g_cache.contiguous() if g_cache is not None else torch.zeros_like(cache))
                g = s.reverse_rollout(ctx.tapes, acts.contiguous(), g, g_acts, recorded=True)
            ctx.tapes = None
            return None, None, g[0], g[1], g[2], g_acts
        with torch.no_grad():
            # the recomputation steps the handle's own views; they are put back afterwards, so a
            # caller that keeps stepping the handle after backward() continues from where the
            # forward pass (or its own later steps) left it
            kept = (s.root_state.clone(), s.dof_state.clone(), s.impulse_cache.clone(), s.dof_actuation.clone())
            g_acts = torch.zeros_like(acts)
            g = (g_root.contiguous() if g_root is not None else torch.zeros_like(root),
                 g_dof.contiguous() if g_dof is not None else torch.zeros_like(dof),
                 g_cache.contiguous() if g_cache is not None else torch.zeros_like(cache))
            tf = s.tape_floats()
            if tf is not None:
                # reverse pass: the segment re-run with each step's tape recorded, then the steps'
                # adjoints in reverse order
                tapes = torch.empty((acts.shape[0], max(tf, 1)), dtype=torch.float32, device=root.device)
                s.root_state.copy_(root)
                s.dof_state.copy_(dof)
                s.impulse_cache.copy_(cache)
                g = s.reverse_rollout(tapes, acts.contiguous(), g, g_acts)
            else:
                _, inputs = _forward_steps(s, root, dof, cache, acts, keep_inputs=True)
                for k in range(acts.shape[0] - 1, -1, -1):
                    r, d, c = inputs[k]
                    gr, gd, gc, ga = _vjp(s, r, d, c, acts[k], *g)
                    g_acts[k] = ga
                    g = (gr, gd, gc)
            for view, value in zip((s.root_state, s.dof_state, s.impulse_cache, s.dof_actuation), kept):
                view.copy_(value)
        return None, None, g[0], g[1], g[2], g_acts


def step(s: "_sim.Sim", root, dof, cache, act, keep_tapes: Optional[bool] = None):
    """One differentiable env-step: returns (root, dof, cache) after the step."""
    keep = keep_tapes_by_default(s, 1) if keep_tapes is None else bool(keep_tapes)
    return Segment.apply(s, keep, root, dof, cache, act.unsqueeze(0))


def rollout(s: "_sim.Sim", root, dof, cache, acts, checkpoint: int = 16, keep_tapes: Optional[bool] = None):
    """acts: (steps, N_D). Differentiable w.r.t. root, dof, cache and acts, in segments of
    `checkpoint` steps. keep_tapes: True records and keeps every step's tape in the forward pass
    (the backward pass applies the adjoints only), False keeps each segment's input state and
    recomputes the segment in the backward pass, None chooses by keep_tapes_by_default. Both give
    bitwise the same values and gradients."""
    keep = keep_tapes_by_default(s, int(acts.shape[0])) if keep_tapes is None else bool(keep_tapes)
    state = (root, dof, cache)
    for k0 in range(0, acts.shape[0], checkpoint):
        state = Segment.apply(s, keep, *state, acts[k0:k0 + checkpoint])
    return state
