"""Differentiable env-steps for PyTorch: torch.autograd.Function wrappers around the C ABI.

The carried state is (root state, DOF state, impulse cache); the actuation is the per-step
control. The forward value is the CUDA step kernel; the backward pass is the step's
vector-Jacobian product with the step's constraint and active sets held fixed: the reverse pass
(sim_step_taped records each re-run step's tape, sim_step_adjoint applies the adjoints in reverse
order) where it covers the handle, else sim_step_vjp in forward mode.

`rollout` chains env-steps with checkpointing: each segment of `checkpoint` steps keeps only its
input state during the forward pass and, in the backward pass, re-runs its steps (bitwise the same
values) to recover every step's input before applying the adjoints in reverse order. The forward
pass leaves the handle's views at the rollout's final state; the backward pass restores them after
its recomputation.
"""
from __future__ import annotations

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


class Segment(torch.autograd.Function):
    """`acts.shape[0]` env-steps from (root, dof, cache); returns the final state."""

    @staticmethod
    def forward(ctx, s, root, dof, cache, acts):
        with torch.no_grad():
            out, _ = _forward_steps(s, root, dof, cache, acts, keep_inputs=False)
        ctx.s = s
        ctx.save_for_backward(root, dof, cache, acts)
        return out

    @staticmethod
    def backward(ctx, g_root, g_dof, g_cache):
        s = ctx.s
        root, dof, cache, acts = ctx.saved_tensors
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
        return None, g[0], g[1], g[2], g_acts


def step(s: "_sim.Sim", root, dof, cache, act):
    """One differentiable env-step: returns (root, dof, cache) after the step."""
    return Segment.apply(s, root, dof, cache, act.unsqueeze(0))


def rollout(s: "_sim.Sim", root, dof, cache, acts, checkpoint: int = 16):
    """acts: (steps, N_D). Differentiable w.r.t. root, dof, cache and acts; the backward pass
    recomputes each segment of `checkpoint` steps from its saved input state."""
    state = (root, dof, cache)
    for k0 in range(0, acts.shape[0], checkpoint):
        state = Segment.apply(s, *state, acts[k0:k0 + checkpoint])
    return state
