"""Launch plans on the GPU: every kernel variant (lanes per env, rows in shared or global memory,
warps per CTA) and the persistent heterogeneous launch against the FP64 oracle under the same
parity bound as the per-type launches; CUDA-graph replay against direct launches; the autotuner
leaves the state as it found it and its plan stays within the bound."""
import numpy as np
import pytest

from paper_2108_10470_gb300 import workloads as W
from test_gpu_parity import check_rollout, workload

pytestmark = pytest.mark.gpu
SIG, PERSIST, GRAPH = 1, 2, 4


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10470_gb300 import build
    build.build_library()
    torch.cuda.set_device(0)


def variants(cfg, persistent):
    """Every valid (lanes, rows_global, warps) of a type; the persistent launch uses 4 warps."""
    out = []
    for lanes in (8, 16, 32):
        if lanes < cfg["min_lanes"]:
            continue
        for rows in (0, 1):
            for warps in ((4,) if persistent else (1, 2, 4)):
                out.append((lanes, rows, warps))
    return out


def type_configs(w, persistent):
    from paper_2108_10470_gb300 import sim
    s = sim.Sim(w, flags=SIG | (PERSIST if persistent else 0))
    cfgs = [s.type_config(t) for t in range(s.n_types)]
    s.destroy()
    return cfgs


@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("name,n_envs", [("cartpole", 67), ("mixed", 67)])
def test_every_variant_matches_oracle(name, n_envs, persistent):
    """One type's knobs varied at a time (the others at their defaults), one env-step each. Shared
    rows are refused exactly for the type with shape pairs (hand with cube)."""
    from paper_2108_10470_gb300 import sim

    w = workload(name, n_envs)
    flags = SIG | (PERSIST if persistent else 0)
    ran = 0
    for t, cfg in enumerate(type_configs(w, persistent)):
        has_pairs = w.env_actor_count(cfg["first_env"]) == 2
        for lanes, rows, warps in variants(cfg, persistent):
            probe = sim.Sim(w, flags=flags)
            try:
                probe.set_type_config(t, lanes, rows, warps)
                refused = None
            except sim.SimError as err:
                refused = err
            probe.destroy()
            if has_pairs and rows == 0:
                assert refused is not None and refused.code == -1
                continue
            assert refused is None, (t, lanes, rows, warps, refused)
            check_rollout(w, 1, 1e-4, 1e-5, flags=flags,
                          setup=lambda s, t=t, c=(lanes, rows, warps): s.set_type_config(t, *c))
            ran += 1
    assert ran >= (6 if persistent else 18) if name == "cartpole" else ran >= 7


@pytest.mark.parametrize("name,n_envs,steps", [("mixed", 67, 1), ("mixed", 67, 16), ("hand", 37, 16), ("ant", 67, 16),
                                               ("mixed", 16384, 1)])
def test_persistent_matches_oracle(name, n_envs, steps):
    rtol, atol = (1e-4, 1e-5) if steps == 1 else (1e-3, 1e-3)
    check_rollout(workload(name, n_envs), steps, rtol, atol,
                  flags=SIG | PERSIST)


def rollout_views(w, flags, steps, dts=None):
    import torch
    from paper_2108_10470_gb300 import sim

    root, dof, acts = W.seeded_inputs(w, 7, steps)
    s = sim.Sim(w, flags=flags)
    s.root_state.copy_(torch.from_numpy(root))
    s.dof_state.copy_(torch.from_numpy(dof))
    out = []
    for k in range(steps):
        s.dof_actuation.copy_(torch.from_numpy(acts[k]))
        s.step(dt=None if dts is None else dts[k])
        torch.cuda.synchronize()
        out.append({n: getattr(s, n).cpu().numpy().copy() for n in ("root_state", "dof_state", "net_contact_force",
                                                                      "impulse_cache", "contact_pairs", "contact_count")})
    s.destroy()
    return out


@pytest.mark.parametrize("base", [SIG, SIG | PERSIST])
def test_graph_replay_equals_direct_launches(base):
    """Graph replays run the same kernels with the same arguments: identical results, including
    after a change of dt (which recaptures)."""
    w = workload("mixed", 67)
    dts = [1 / 60, 1 / 60, 1 / 120, 1 / 120, 1 / 60]
    a = rollout_views(w, base, 5, dts)
    b = rollout_views(w, base | GRAPH, 5, dts)
    for k in range(5):
        for n in a[k]:
            assert np.array_equal(a[k][n], b[k][n]), (k, n)


def test_persistent_launches_back_to_back():
    """Back-to-back persistent launches step every env every time (the tile counter resets itself):
    each step moves some root of every env and keeps the state finite. From identical inputs the
    first step agrees with the per-type launches within the one-step parity bound (the two launch
    forms round differently in FP32; later steps are compared with the oracle elsewhere, under the
    conditioning-aware bound)."""
    w = workload("mixed", 300)
    a = rollout_views(w, SIG, 6)
    b = rollout_views(w, SIG | PERSIST, 6)
    for n, (rt, at) in (("root_state", (1e-4, 1e-5)), ("dof_state", (1e-4, 1e-5)), ("net_contact_force", (1e-3, 1e-3))):
        np.testing.assert_allclose(b[0][n], a[0][n], rtol=rt, atol=at, err_msg=n)
    assert np.array_equal(b[0]["contact_count"], a[0]["contact_count"])
    rows = np.cumsum([0] + [w.env_actor_count(e) for e in range(w.n_envs)])
    for k in range(1, 6):
        assert np.isfinite(b[k]["root_state"]).all() and np.isfinite(b[k]["dof_state"]).all()
        moved = np.abs(b[k]["root_state"] - b[k - 1]["root_state"]).max(axis=1) > 0
        assert all(moved[rows[e]:rows[e + 1]].any() for e in range(w.n_envs)), f"an env was skipped at step {k}"


@pytest.mark.parametrize("flags", [SIG, SIG | PERSIST])
def test_autotune_keeps_state_and_parity(flags):
    import torch
    from paper_2108_10470_gb300 import sim

    w = workload("mixed", 200)
    root, dof, acts = W.seeded_inputs(w, 0, 1)
    s = sim.Sim(w, flags=flags)
    s.root_state.copy_(torch.from_numpy(root))
    s.dof_state.copy_(torch.from_numpy(dof))
    s.dof_actuation.copy_(torch.from_numpy(acts[0]))
    s.step()
    names = ("root_state", "dof_state", "net_contact_force", "impulse_cache", "contact_pairs", "contact_count",
             "status")
    before = {n: getattr(s, n).cpu().numpy().copy() for n in names}
    ms = s.autotune(reps=3)
    torch.cuda.synchronize()
    assert 0 < ms < 100
    for n in names:
        assert np.array_equal(getattr(s, n).cpu().numpy(), before[n]), n
    chosen = [s.type_config(t) for t in range(s.n_types)]
    s.destroy()

    def setup(sim_obj):
        for t, c in enumerate(chosen):
            sim_obj.set_type_config(t, c["lanes_per_env"], c["rows_global"], c["warps_per_cta"])
    check_rollout(w, 2, 1e-3, 1e-3, flags=flags, setup=setup)
