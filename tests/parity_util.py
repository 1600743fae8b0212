"""Shared helpers of the GPU parity tests: run the same seeded inputs through the CUDA library
(via the C-ABI binding) and through the FP64 oracle, then compare per environment."""
import numpy as np

import oracle
from paper_2108_10470_gb300 import workloads as W


def env_rows(w, per):
    """Row slices of a per-env tensor with `per(env)` rows per env."""
    out, o = [], 0
    for e in range(w.n_envs):
        k = per(e)
        out.append(slice(o, o + k))
        o += k
    return out


def gpu_rollout(w, root, dof, acts, steps, flags=1, setup=None):
    """Run `steps` env-steps through the C ABI; setup(sim) runs once after creation (launch knobs)."""
    import torch
    from paper_2108_10470_gb300 import sim

    s = sim.Sim(w, flags=flags)
    if setup is not None:
        setup(s)
    s.root_state.copy_(torch.from_numpy(root))
    s.dof_state.copy_(torch.from_numpy(dof))
    snaps = []
    for k in range(steps):
        s.dof_actuation.copy_(torch.from_numpy(acts[k]))
        s.step()
        snaps.append(dict(root=s.root_state.cpu().numpy().astype(np.float64),
                          dof=s.dof_state.cpu().numpy().astype(np.float64),
                          net_force=s.net_contact_force.cpu().numpy().astype(np.float64),
                          pairs=s.contact_pairs.cpu().numpy(), n_pairs=s.contact_count.cpu().numpy(),
                          sig=s.signature.cpu().numpy().astype(np.uint32), status=s.status.cpu().numpy(),
                          cache=s.impulse_cache.cpu().numpy().astype(np.float64)))
    s.destroy()
    return snaps


def oracle_rollout(w, root, dof, acts, steps):
    O = oracle.Oracle(w)
    r, d = root.astype(np.float64), dof.astype(np.float64)
    snaps = []
    for k in range(steps):
        out = O.step(r, d, acts[k])
        snaps.append(dict(root=r.copy(), dof=d.copy(), net_force=out["net_force"].copy(), pairs=out["contacts"],
                          n_pairs=out["n_contacts"], sig=out["signature"], failed=out["n_failed"],
                          cache=O.cache.copy()))
    return snaps


def per_env_ok(w, g, o, rtol, atol, key, per):
    """Boolean per env: every component of tensor `key` within atol + rtol*|oracle|."""
    rows = env_rows(w, per)
    a, b = g[key], o[key]
    ok = np.zeros(w.n_envs, bool)
    worst = np.zeros(w.n_envs)
    for e, sl in enumerate(rows):
        ex = np.abs(a[sl] - b[sl]) - (atol + rtol * np.abs(b[sl]))
        worst[e] = ex.max() if ex.size else -1.0
        ok[e] = worst[e] <= 0
    return ok, worst


def compare(w, g, o, rtol, atol, mask):
    """Check root, DOF and net-force parity on the envs in mask; return a report dict."""
    rep = {}
    for key, per in (("root", w.env_actor_count), ("dof", w.env_jdof), ("net_force", w.env_body)):
        ok, worst = per_env_ok(w, g, o, rtol, atol, key, per)
        rep[key] = (ok, worst)
    return rep


def _ulp(a, direction):
    return np.nextafter(a.astype(np.float32), np.float32(direction * np.inf)).astype(np.float64)


def fp32_scales(w, root, dof, acts, steps, rtol=1e-4, atol=1e-5):
    """Per step, tensor and env: the largest deviation from the FP64 oracle of four single-precision
    evaluations of the same oracle algorithm (inputs as given, and nudged by one float32 ulp in
    three patterns). This is the env's FP32 conditioning scale: how far any faithful FP32
    evaluation of the method can land from the FP64 result."""
    base = oracle_rollout(w, root, dof, acts, steps)
    runs = []
    for pert in range(4):
        O = oracle.Oracle(w)
        r, d = root.astype(np.float64), dof.astype(np.float64)
        if pert in (1, 2):
            s = 1 if pert == 1 else -1
            r[:, :3] = _ulp(r[:, :3], s)
            d[:, 0] = _ulp(d[:, 0], -s)
        elif pert == 3:
            r[:, 3:7] = _ulp(r[:, 3:7], 1)
            d[:, 1] = _ulp(d[:, 1], 1)
        snaps = []
        for k in range(steps):
            nf = O.step_f32(r, d, acts[k])
            snaps.append(dict(root=r.copy(), dof=d.copy(), net_force=nf))
        runs.append(snaps)
    scales = []
    per = {"root": w.env_actor_count, "dof": w.env_jdof, "net_force": w.env_body}
    for k in range(steps):
        sk = {}
        for key, pf in per.items():
            rows = env_rows(w, pf)
            s = np.zeros(w.n_envs)
            for e, sl in enumerate(rows):
                if sl.stop > sl.start:
                    s[e] = max(np.abs(run[k][key][sl] - base[k][key][sl]).max() for run in runs)
            sk[key] = s
        # fraction of components within the strict bound, lowest over the FP32 evaluations
        sk["strict_frac"] = {key: min(float(np.mean(np.abs(run[k][key] - base[k][key]) <=
                                                    atol + rtol * np.abs(base[k][key]))) for run in runs)
                             if base[k][key].size else 1.0 for key in per}
        # per component: the largest deviation of the four FP32 evaluations from FP64
        sk["component"] = {key: np.max([np.abs(run[k][key] - base[k][key]) for run in runs], axis=0)
                           for key in per}
        scales.append(sk)
    return base, scales
