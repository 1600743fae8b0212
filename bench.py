"""Throughput of the GB300 articulated-body step (env-steps/s), one JSON line on stdout.

A step is one sim_step(1/60 s, 2 substeps) over the whole batch (default: the Ant-like workload,
4096 environments), preceded by the device-to-device copy of that step's pre-generated actions
into the DOF actuation view. Inputs are resident in HBM before the timed region; L2 is flushed
(256 MiB memset) between timed steps, outside each step's event pair.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload ant|humanoid|cartpole|hand|mixed] [--envs E]
                  [--persistent] [--graph] [--autotune]
  python bench.py --impl reference ...   # the FP64 CPU oracle timed on the host cores

Under torchrun (N > 1) every rank simulates its own E environments on its own GPU (weak scaling:
environments never interact, so there is no collective on the data path); the timed region is
bracketed by barriers and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
METRIC = "env-steps/sec on 1 GB300 (Ant-like, 4096 envs) vs oracle; adjoint steps/sec"
PAIR_SLOTS = 5  # contact candidates per capsule-box pair


def env_candidates(w, e) -> int:
    """Contact candidates of env e: ground candidates of every shape (sphere 1, capsule 2, box 8)
    plus PAIR_SLOTS per capsule-box pair across actors."""
    from paper_2108_10470_gb300 import workloads as W
    models = w.actor_models(e)
    caps = [sum(int(t == W.SHAPE_CAPSULE) for t in m.shape_type) for m in models]
    boxes = [sum(int(t == W.SHAPE_BOX) for t in m.shape_type) for m in models]
    pairs = sum(caps[i] * boxes[j] + boxes[i] * caps[j] for i in range(len(models)) for j in range(i + 1, len(models)))
    return sum(m.contact_cap for m in models) + PAIR_SLOTS * pairs


def algo_bytes_per_step(w) -> int:
    """HBM bytes one step must move over all envs. Read: root (13 f32 per actor), DOF state (2 per
    joint DOF), actuation (1 per joint DOF), impulse cache (3 per candidate + 2 per joint DOF).
    Written: root, DOF state, net contact force (3 per body), impulse cache, contact list (3 i32
    per candidate), count / status / signature."""
    total = 0
    for e in range(w.n_envs):
        A, J, B, C = w.env_actor_count(e), w.env_jdof(e), w.env_body(e), env_candidates(w, e)
        cache = 3 * C + 2 * J
        total += 4 * ((13 * A + 2 * J + J + cache) + (13 * A + 2 * J + 3 * B + cache + 3 * C + 3))
    return total


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """Slowest rank's time (all ranks call this; a no-op on one rank)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank: int) -> int:
    """Each rank simulates its own environments from its own seed (weak scaling)."""
    return 1000 * rank


def weak_value(world: int, n_envs: int, steps: int, seconds: float) -> float:
    """Whole-job env-steps/s: every rank advanced n_envs envs by `steps` steps."""
    return world * n_envs * steps / seconds


KERNEL_SOURCES = ("step_kernel.cuh", "sim_internal.h", "kernels_shared.cu", "kernels_global.cu",
                  "kernels_persistent.cu")


def kernel_source_hash() -> str:
    """First 16 hex digits of the SHA-256 of the step kernels' sources (a profile summary whose
    hash differs describes other code and is not used)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2108_10470_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_fields(kernel: str, wname: str):
    """(fields, table rows, captured env count) of the committed ncu summary of this kernel and
    workload whose kernel sources match the current ones; (None, None, None) if there is none."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_{wname}[0-9]*.md"))):
        try:
            text = open(path).read().splitlines()
            fields = dict(ln.split(":", 1) for ln in text[:6] if ":" in ln)
            if fields.get("kernel_source_sha256_16", "").strip() != kernel_source_hash():
                continue
            rows = {}
            for ln in text:
                cells = [c.strip() for c in ln.split("|")]
                if len(cells) > 4 and cells[2].startswith("`"):
                    rows[cells[2].strip("`")] = cells[3]
            return fields, rows, int(os.path.basename(path)[len(kernel) + 1 + len(wname):-3])
        except (OSError, ValueError):
            continue
    return None, None, None


def profiled_fma_pipe_pct(kernel: str, wname: str):
    """FMA-pipe utilisation (% of peak, active cycles) from the committed ncu summary, or None."""
    _, rows, _ = profile_fields(kernel, wname)
    try:
        return float(rows["sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active"].split()[0])
    except (TypeError, KeyError, ValueError, IndexError):
        return None


def sample_inputs(w, idx, root, dof, acts):
    """The seeded inputs of a subset of envs, taken from the whole batch's arrays (so the subset sees
    exactly the inputs the GPU run gives those envs)."""
    ra = np.cumsum([0] + [w.env_actor_count(e) for e in range(w.n_envs)])
    rd = np.cumsum([0] + [w.env_jdof(e) for e in range(w.n_envs)])
    r = np.concatenate([root[ra[e]:ra[e + 1]] for e in idx])
    d = np.concatenate([dof[rd[e]:rd[e + 1]] for e in idx])
    a = np.concatenate([acts[:, rd[e]:rd[e + 1]] for e in idx], axis=1)
    return r, d, a


def window_flops(w, root, dof, acts, warm, steps, sample=64):
    """Algorithmic flops per env-step over the steps warm .. warm + steps - 1 of the seeded
    trajectory (the bench's timed window), counted by the oracle's operation-counting scalar on a
    strided sample of the batch's envs (the step's cost grows with the ground contacts made)."""
    import oracle
    idx = list(range(0, w.n_envs, max(1, w.n_envs // sample)))[:sample]
    ws = w.subset(idx)
    r, d, a = sample_inputs(w, idx, root, dof, acts)
    O = oracle.Oracle(ws)
    r, d = r.astype(np.float64), d.astype(np.float64)
    for k in range(warm):
        O.step(r, d, a[k])
    total = sum(O.step_flops(r, d, a[warm + k]) for k in range(steps))
    return total / (steps * len(idx)), f"steps {warm}..{warm + steps - 1}, {len(idx)} envs (every {w.n_envs // len(idx)}th)"


def profiled_traffic(kernel: str, wname: str, n_envs: int):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu summary of this
    workload (profiles/<kernel>_<workload><envs>.md), scaled to n_envs; None if there is none or
    the kernel sources changed since."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_{wname}[0-9]*.md"))):
        try:
            fields = dict(ln.split(":", 1) for ln in open(path).read().splitlines()[:6] if ":" in ln)
            if fields.get("kernel_source_sha256_16", "").strip() != kernel_source_hash():
                continue
            captured = int(os.path.basename(path)[len(kernel) + 1 + len(wname):-3])
            return float(fields["traffic_bytes_per_launch"]) * n_envs / captured
        except (OSError, KeyError, ValueError):
            continue
    return None


def workload(name, n_envs):
    from paper_2108_10470_gb300 import workloads as W
    return {"ant": W.ant_workload, "humanoid": W.humanoid_workload, "cartpole": W.cartpole_workload,
            "hand": W.hand_workload, "mixed": W.mixed_workload}[name](n_envs)


def describe(w):
    return (f"{w.name}-like, {w.n_envs} envs, dt {w.dt:.6f} s, {w.substeps} substeps, "
            f"{w.params.pos_iters}/{w.params.vel_iters} solver iterations, seeded synthetic inputs")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(wname, n_envs, budget_s=15.0):
    """The FP64 oracle, as it stands, on the host cores: env-steps/s on a bounded sample of the
    same workload, plus its operation count per env-step (the algorithmic flops of the step)."""
    import oracle
    from paper_2108_10470_gb300 import workloads as W

    w = workload(wname, n_envs)
    threads = os.cpu_count() or 1
    O = oracle.Oracle(w)
    n_act = 100  # action steps drawn from the seed; the timed sample cycles through them
    root, dof, acts = W.seeded_inputs(w, 0, n_act)
    r, d = root.astype(np.float64), dof.astype(np.float64)
    t0 = time.perf_counter()
    O.step(r, d, acts[0], n_threads=threads)
    one = max(time.perf_counter() - t0, 1e-4)
    n_steps = int(max(2, min(5000, budget_s / one)))
    t0 = time.perf_counter()
    for k in range(1, 1 + n_steps):
        O.step(r, d, acts[k % n_act], n_threads=threads)
    el = time.perf_counter() - t0
    value = n_envs * n_steps / el
    return {"value": value, "unit": "env-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{n_steps} env-steps of all {n_envs} envs after 1 warm-up step ({el:.1f} s, "
                      f"{threads} threads)"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, same workload / metric / unit."""
    if rank != 0:
        return
    import oracle
    from paper_2108_10470_gb300 import workloads as W

    w = workload(args.workload, args.envs)
    threads = os.cpu_count() or 1
    sample_envs = min(args.envs, 1024)
    ws = w.subset(list(range(sample_envs)))
    O = oracle.Oracle(ws)
    root, dof, acts = W.seeded_inputs(ws, 0, args.warmup + args.steps)
    r, d = root.astype(np.float64), dof.astype(np.float64)
    for k in range(args.warmup):
        O.step(r, d, acts[k], n_threads=threads)
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.step(r, d, acts[args.warmup + k], n_threads=threads)
    el = time.perf_counter() - t0
    value = sample_envs * args.steps / el
    line = {"metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": describe(w), "n_envs": args.envs,
                       "sample": f"each step advances the first {sample_envs} of the {args.envs} envs"},
            "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"{sample_envs} envs x {args.steps} timed env-steps"},
            "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2108_10470_gb300 import build, sim, workloads as W

    build.build_library()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = workload(args.workload, args.envs)
    K, Wm = args.steps, args.warmup
    flags = (sim.SIM_FLAG_PERSISTENT if args.persistent else 0) | (sim.SIM_FLAG_GRAPH if args.graph else 0)
    s = sim.Sim(w, flags=flags)
    stream = torch.cuda.current_stream()
    root, dof, acts = W.seeded_inputs(w, rank_seed(rank), Wm + K)
    s.root_state.copy_(torch.from_numpy(root))
    s.dof_state.copy_(torch.from_numpy(dof))
    act_dev = torch.from_numpy(acts).to(dev)  # every step's actions resident in HBM
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for k in range(Wm):
        actuated_step(s, act_dev[k])
        if args.autotune and k == Wm // 2:  # tune on a mid-warm-up state; the state is left unchanged
            s.autotune(reps=5)
    torch.cuda.synchronize()
    plan = {"launch": "persistent" if args.persistent else "per env type", "graph": bool(args.graph),
            "autotuned": bool(args.autotune),
            "types": [{k: c[k] for k in ("lanes_per_env", "rows_global", "warps_per_cta", "n_envs")}
                      for c in (s.type_config(t) for t in range(s.n_types))]}
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    in_place = reads_actions_in_place(s)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for k in range(K):
            flush.zero_()  # L2 flush, outside the step's events
            e0, e1, e2 = ev[k]
            e0.record(stream)
            if not in_place:  # graph and persistent handles: the actions copied into the view
                s.dof_actuation.copy_(act_dev[Wm + k])
            e1.record(stream)
            torch.cuda.nvtx.range_push("timed_step")  # lets ncu --nvtx-include pick timed launches
            if in_place:  # the step kernels read the step's actions from act_dev themselves
                s.step_actuated(act_dev[Wm + k])
            else:
                s.step()
            torch.cuda.nvtx.range_pop()
            e2.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [ev[k][0].elapsed_time(ev[k][2]) for k in range(K)]
    kern_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(K)]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, dev)
    bad = s.sync_status()
    # end-to-end through the C ABI with pinned host buffers (copies inside the timed region)
    n_e2e = min(K, 200)
    h_act = torch.from_numpy(acts[Wm:Wm + n_e2e]).pin_memory().numpy()
    h_root = torch.empty((s.N_A, 13), dtype=torch.float32).pin_memory().numpy()
    h_dof = torch.empty((max(s.N_D, 1), 2), dtype=torch.float32).pin_memory().numpy()
    s.step_host(np.ascontiguousarray(h_act[0]), h_root, h_dof)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for k in range(n_e2e):
        s.step_host(h_act[k], h_root, h_dof)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    launches = s.launches_per_step * K
    n_d, n_a = s.N_D, s.N_A
    s.destroy()
    if rank != 0:
        return
    value = weak_value(world, w.n_envs, K, total_s)
    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": 1e3 * total_s / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": describe(w), "n_envs_per_gpu": w.n_envs, "dt": w.dt, "substeps": w.substeps,
                       "l2": "flushed between timed steps (256 MiB memset outside the step events)",
                       "parallelism": f"replicas x{world} (independent envs per GPU)"},
            "gpu_launches": launches, "nonfinite_envs": bad, "plan": plan,
            "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "e2e": {"value": weak_value(world, w.n_envs, n_e2e, e2e_s), "unit": "env-steps/s",
                    "h2d_bytes_per_step": 4 * n_d, "d2h_bytes_per_step": 4 * (13 * n_a + 2 * n_d),
                    "api": "sim_step_host (pinned host actuation in, root + DOF state out, stream sync)"}}
    kern_avg_s = statistics.mean(kern_ms) / 1e3
    roof = None
    cpu = None
    if world == 1:
        kname = "persistent_step_kernel" if args.persistent else "step_kernel"
        flops_per_env_step, window = window_flops(w, root, dof, acts, Wm, K)
        peak = probe_peak_flops()
        sm_mhz = clocks["sm_mhz"] or 2070.0
        nominal = SM_COUNT_NOMINAL * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6
        achieved = flops_per_env_step * w.n_envs / kern_avg_s
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": args.traffic if args.traffic is not None else profiled_traffic(kname, args.workload, w.n_envs),
                "algorithmic_bytes_per_step": algo_bytes_per_step(w),
                "kernel": kname, "kernel_ms": 1e3 * kern_avg_s,
                "flops_per_env_step": flops_per_env_step, "flops_window": window,
                "peak_basis": "measured: FP32 FMA throughput of sim_probe_fp32_peak on this GPU (all SMs, 8 "
                              "independent FMA chains per thread, 64 warps per SM), of measured",
                "peak_nominal": nominal / 1e12, "frac_of_nominal": achieved / nominal,
                "peak_nominal_basis": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz (median SM clock "
                                      f"sampled in the timed region)",
                "ncu_fma_pipe_pct": profiled_fma_pipe_pct(kname, args.workload)}
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(args.workload, args.envs)
    line["roofline"] = roof
    line["cpu_baseline"] = cpu
    if world == 1 and not args.no_variants and args.workload == "ant" and args.envs == 4096:
        line["variants"] = variants_measure(dev)
        line["configs"] = configs_measure(dev, peak / 1e12 if roof else None)
    if world == 1 and not args.no_adjoint:
        line["adjoint"] = adjoint_measure(dev)
    print(json.dumps(line), flush=True)


def probe_peak_flops() -> float:
    """The GPU's FP32 FMA throughput measured by the library's probe (median of three runs)."""
    from paper_2108_10470_gb300 import sim
    return statistics.median(sim.probe_fp32_peak(20000) for _ in range(3))


def reads_actions_in_place(s) -> bool:
    """Whether sim_step_actuated serves the handle by its step kernel reading a step's actions from
    the caller's tensor (one env type, per-type launch, no captured graph); other handles get the
    actions copied into the actuation view first."""
    from paper_2108_10470_gb300 import sim
    return s.n_types == 1 and not (s.flags & (sim.SIM_FLAG_GRAPH | sim.SIM_FLAG_PERSISTENT))


def actuated_step(s, act):
    """One control step with this step's actions (a device tensor): sim_step_actuated where the
    step kernel reads the actions in place (paper: applying the actuation force tensor, then
    simulating); elsewhere the copy into the actuation view and sim_step (what sim_step_actuated
    enqueues for those handles), so that the events can time the step kernels alone."""
    if reads_actions_in_place(s):
        s.step_actuated(act)
    else:
        s.dof_actuation.copy_(act)
        s.step()


def timed_steps(s, act_dev, warm, steps, flush):
    """Mean device time of `steps` control steps (each: the step's actions applied and sim_step;
    L2 flushed before each, outside the step's events) after `warm` untimed steps."""
    import torch
    for k in range(warm):
        actuated_step(s, act_dev[k % act_dev.shape[0]])
    torch.cuda.synchronize()
    ev = []
    for k in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        actuated_step(s, act_dev[(warm + k) % act_dev.shape[0]])
        e1.record()
        ev.append((e0, e1))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def variants_measure(dev, warm=20, steps=200):
    """The same Ant-like step at 8192 and 16384 envs, and at 4096 envs launched directly and replayed
    as a captured CUDA graph: env-steps/s under the main line's timing protocol, over 200 timed
    steps after 20 warm-up steps (fewer than the main line's, so fewer ground contacts: compare
    these lines with each other)."""
    import torch

    from paper_2108_10470_gb300 import sim, workloads as W

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    out = {}
    for n_envs, flags, key in ((8192, 0, "envs_8192"), (16384, 0, "envs_16384"), (4096, 0, "envs_4096"),
                               (4096, sim.SIM_FLAG_GRAPH, "cuda_graph_4096")):
        w = W.ant_workload(n_envs)
        root, dof, acts = W.seeded_inputs(w, 0, warm + steps)
        s = sim.Sim(w, flags=flags)
        s.root_state.copy_(torch.from_numpy(root))
        s.dof_state.copy_(torch.from_numpy(dof))
        ms = timed_steps(s, torch.from_numpy(acts).to(dev), warm, steps, flush)
        s.destroy()
        out[key] = {"value": n_envs / (ms / 1e3), "ms_per_step": ms}
    out["unit"] = "env-steps/s"
    return out


def config_line(w, dev, flush, warm, steps, flags=0, autotune=False, peak_tflops=None, flops_sample=32, seed=0):
    """One config's env-steps/s under the main line's protocol (L2 flushed between timed steps, CUDA
    events around the action copy and the step), with its FP32 roofline fraction when a peak is
    given (flops counted by the oracle over the same window on a strided sample of envs)."""
    import torch

    from paper_2108_10470_gb300 import sim, workloads as W

    root, dof, acts = W.seeded_inputs(w, seed, warm + steps)
    s = sim.Sim(w, flags=flags)
    s.root_state.copy_(torch.from_numpy(root))
    s.dof_state.copy_(torch.from_numpy(dof))
    act_dev = torch.from_numpy(acts).to(dev)
    if autotune:
        for k in range(warm // 2):
            actuated_step(s, act_dev[k])
        s.autotune(reps=5)
        s.root_state.copy_(torch.from_numpy(root))
        s.dof_state.copy_(torch.from_numpy(dof))
        s.impulse_cache.zero_()
    ms = timed_steps(s, act_dev, warm, steps, flush)
    plan = [{k: c[k] for k in ("lanes_per_env", "rows_global", "warps_per_cta")} for c in
            (s.type_config(t) for t in range(s.n_types))]
    s.destroy()
    out = {"value": w.n_envs / (ms / 1e3), "ms_per_step": ms, "timed_steps": steps, "warmup": warm, "plan": plan}
    if peak_tflops:
        f, window = window_flops(w, root, dof, acts, warm, steps, flops_sample)
        out["roofline"] = {"bound": "alu", "flops_per_env_step": f, "flops_window": window,
                           "achieved": f * w.n_envs / (ms / 1e3) / 1e12, "peak": peak_tflops, "unit": "TFLOP/s",
                           "frac": f * w.n_envs / (ms / 1e3) / 1e12 / peak_tflops,
                           "note": "step time includes applying the step's actions (read in place by the "
                                   "step kernel of a one-type handle, else copied into the actuation view)"}
    return out


def configs_measure(dev, peak_tflops, warm=20, steps=100):
    """The other configurations of the workload set, each under the main line's timing protocol:
    Humanoid-like 4096 envs, hand with cube 4096 envs, cartpole 64 envs over 1000 steps, and the
    heterogeneous 16384-env batch (40 % Ant-like, 30 % Humanoid-like, 30 % hand with cube) as one
    launch per env type (concurrent on forked streams, the default), one persistent launch (default
    and autotuned knobs, and autotuned replayed as a CUDA graph), against the sum of each type's
    envs stepped alone."""
    import torch

    from paper_2108_10470_gb300 import sim, workloads as W

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    out = {"unit": "env-steps/s"}
    out["humanoid_4096"] = config_line(W.humanoid_workload(4096), dev, flush, warm, steps, peak_tflops=peak_tflops)
    out["hand_4096"] = config_line(W.hand_workload(4096), dev, flush, warm, steps, peak_tflops=peak_tflops)
    out["cartpole_64_1000_steps"] = config_line(W.cartpole_workload(64), dev, flush, warm, 1000,
                                                peak_tflops=peak_tflops)
    out["cartpole_64_1000_steps_graph"] = config_line(W.cartpole_workload(64), dev, flush, warm, 1000,
                                                      flags=sim.SIM_FLAG_GRAPH)
    mixed = W.mixed_workload(16384)
    out["mixed_16384_per_type"] = config_line(mixed, dev, flush, warm, steps, peak_tflops=peak_tflops)
    out["mixed_16384_persistent"] = config_line(mixed, dev, flush, warm, steps, flags=sim.SIM_FLAG_PERSISTENT)
    out["mixed_16384_persistent_autotuned"] = config_line(mixed, dev, flush, warm, steps, flags=sim.SIM_FLAG_PERSISTENT,
                                                          autotune=True)
    out["mixed_16384_persistent_autotuned_graph"] = config_line(
        mixed, dev, flush, warm, steps, flags=sim.SIM_FLAG_PERSISTENT | sim.SIM_FLAG_GRAPH, autotune=True)
    # each type's envs of the mixed batch stepped alone (seeded inputs of the same distributions)
    alone = 0.0
    for t, name in enumerate(("ant", "humanoid", "hand")):
        idx = [e for e in range(mixed.n_envs) if int(mixed.env_actor_model[2 * e]) == t]
        ms = config_line(mixed.subset(idx), dev, flush, warm, steps)["ms_per_step"]
        out[f"mixed_16384_{name}_alone_ms"] = ms
        alone += ms
    out["mixed_16384_sum_of_types_alone_ms"] = alone
    for k in ("per_type", "persistent", "persistent_autotuned", "persistent_autotuned_graph"):
        out[f"mixed_16384_{k}_over_sum_of_types_alone"] = out[f"mixed_16384_{k}"]["ms_per_step"] / alone
    return out


def adjoint_measure(dev, n_envs=1024, steps=64, checkpoint=16, reps=2):
    """Adjoint throughput on the differentiable-rollout workload: 1024 Ant-like envs, 64 env-steps,
    loss = mean final root x-velocity, gradients w.r.t. every action and the initial DOF state
    (autograd rollout in segments of 16 steps). value = env-steps differentiated per second of the
    backward pass under the rollout's default memory policy (the forward pass keeps every step's
    tape when the rollout's tapes take at most a quarter of the free device memory: here 1.2 GB);
    the checkpointing policy (each segment re-run with its tapes recorded in the backward pass) is
    measured beside it."""
    import torch

    from paper_2108_10470_gb300 import autograd as AG, sim, workloads as W

    w = W.ant_workload(n_envs)
    s = sim.Sim(w)
    s_reverse = s.tape_floats() is not None
    root, dof, acts = W.seeded_inputs(w, 0, steps)
    r0 = torch.from_numpy(root).to(dev)
    d0 = torch.from_numpy(dof).to(dev).requires_grad_(True)
    c0 = torch.zeros((n_envs, s.cache_len), device=dev)
    A = torch.from_numpy(acts).to(dev).requires_grad_(True)

    def timed(keep):
        fwd, bwd = [], []
        for rep in range(reps + 1):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            rf, _, _ = AG.rollout(s, r0, d0, c0, A, checkpoint=checkpoint, keep_tapes=keep)
            loss = rf[:, 7].mean()
            e[1].record()
            loss.backward()
            e[2].record()
            torch.cuda.synchronize()
            if rep > 0:
                fwd.append(e[0].elapsed_time(e[1]))
                bwd.append(e[1].elapsed_time(e[2]))
            d0.grad = None
            A.grad = None
        return statistics.median(fwd), statistics.median(bwd)

    kept = AG.keep_tapes_by_default(s, steps)
    f_ms, b_ms = timed(None)
    rf_ms, rb_ms = timed(False)
    s.destroy()
    hand = hand_adjoint_measure(dev)
    return {"value": n_envs * steps / (b_ms / 1e3), "unit": "adjoint env-steps/s",
            "workload": f"Ant-like, {n_envs} envs, {steps} env-steps, loss = mean final root x-velocity, gradients "
                        f"w.r.t. actions and initial DOF state, segments of {checkpoint} steps",
            "policy": "tapes kept from the forward pass" if kept else "segments recomputed (checkpointing)",
            "forward_ms": f_ms, "backward_ms": b_ms, "backward_over_forward": b_ms / f_ms,
            "forward_plus_backward_ms": f_ms + b_ms,
            "recompute": {"forward_ms": rf_ms, "backward_ms": rb_ms, "backward_over_forward": rb_ms / rf_ms,
                          "forward_plus_backward_ms": rf_ms + rb_ms},
            "hand": hand,
            "method": ("reverse pass: sim_step_taped records each step's tape (in the forward pass when the tapes "
                       "are kept, else in the backward pass's re-run of each segment), sim_step_adjoint applies "
                       "the steps' adjoints in reverse order" if s_reverse else
                       "forward-mode dual kernel (one env per warp), vector-Jacobian product per env-step")}


def hand_adjoint_measure(dev, n_envs=1024, steps=16, reps=2):
    """The same rollout gradient on the hand-with-cube workload (capsule-box pair contacts: the
    reverse pass's pair instantiation): 1024 envs, 16 steps from the seeded state, tapes kept."""
    import torch

    from paper_2108_10470_gb300 import autograd as AG, sim, workloads as W

    w = W.hand_workload(n_envs)
    s = sim.Sim(w)
    root, dof, acts = W.seeded_inputs(w, 0, steps)
    r0 = torch.from_numpy(root).to(dev)
    d0 = torch.from_numpy(dof).to(dev).requires_grad_(True)
    c0 = torch.zeros((n_envs, s.cache_len), device=dev)
    A = torch.from_numpy(acts).to(dev).requires_grad_(True)
    fwd, bwd = [], []
    for rep in range(reps + 1):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        rf, _, _ = AG.rollout(s, r0, d0, c0, A, checkpoint=steps)
        loss = rf[:, 7].mean()
        e[1].record()
        loss.backward()
        e[2].record()
        torch.cuda.synchronize()
        if rep > 0:
            fwd.append(e[0].elapsed_time(e[1]))
            bwd.append(e[1].elapsed_time(e[2]))
        d0.grad = None
        A.grad = None
    kept = AG.keep_tapes_by_default(s, steps)
    s.destroy()
    f_ms, b_ms = statistics.median(fwd), statistics.median(bwd)
    return {"value": n_envs * steps / (b_ms / 1e3), "unit": "adjoint env-steps/s",
            "workload": f"hand with cube, {n_envs} envs, {steps} env-steps, loss = mean final root x-velocity",
            "policy": "tapes kept from the forward pass" if kept else "segments recomputed (checkpointing)",
            "forward_ms": f_ms, "backward_ms": b_ms, "backward_over_forward": b_ms / f_ms}


def run_adjoint_only(local_rank):
    """The adjoint measurement alone (one GPU): the command the adjoint kernel's profiles are taken on."""
    import torch

    from paper_2108_10470_gb300 import build

    build.build_library()
    torch.cuda.set_device(local_rank)
    adj = adjoint_measure(torch.device("cuda", local_rank))
    line = {"metric": "adjoint env-steps/s (Ant-like, 1024 envs, 64-step rollout gradient)", "value": adj["value"],
            "unit": adj["unit"], "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": adj["workload"]}, "adjoint": adj}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ant", choices=["ant", "humanoid", "cartpole", "hand", "mixed"])
    ap.add_argument("--envs", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--persistent", action="store_true", help="one persistent launch for all env types")
    ap.add_argument("--graph", action="store_true", help="replay each step as a captured CUDA graph")
    ap.add_argument("--autotune", action="store_true", help="autotune the launch knobs during warm-up")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (differentiable rollout) measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the 8192 / 16384-env and CUDA-graph lines")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint (differentiable rollout) measurement and print its line")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per step-kernel launch from an ncu capture of the same kernel")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.adjoint_only:
        run_adjoint_only(local_rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
