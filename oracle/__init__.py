"""FP64 CPU oracle of the batched articulated-body step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of ``bench.py``
may import this package. The CUDA product path never touches it, and the two share no code: this
wrapper marshals a :class:`paper_2108_10470_gb300.workloads.Workload` (model data and seeded
inputs, no physics) into the C++ oracle in ``oracle.cpp`` and returns numpy arrays.

Every pin of the oracle (closed forms, invariants, brute force) lives in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, f) for f in ("oracle.cpp", "oracle_math.hpp", "oracle_opcount.hpp")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

D = ctypes.POINTER(ctypes.c_double)
I32 = ctypes.POINTER(ctypes.c_int32)


class _Models(ctypes.Structure):
    _fields_ = [("n_models", ctypes.c_int32), ("link_off", I32), ("shape_off", I32), ("parent", I32), ("jtype", I32),
                ("axis", D), ("ppos", D), ("pquat", D), ("mass", D), ("com", D), ("inertia", D), ("armature", D),
                ("damping", D), ("lo", D), ("hi", D), ("has_limit", I32), ("is_virtual", I32), ("shape_link", I32),
                ("shape_type", I32), ("shape_size", D), ("shape_pos", D), ("shape_quat", D), ("shape_friction", D),
                ("drive_kp", D), ("drive_kd", D), ("tendon_off", I32), ("tendon_entry_off", I32),
                ("tendon_link", I32), ("tendon_coef", D), ("tendon_stiffness", D), ("tendon_damping", D),
                ("tendon_rest", D), ("tendon_lo", D), ("tendon_hi", D), ("tendon_has_limit", I32)]


class _Params(ctypes.Structure):
    _fields_ = [("gravity", ctypes.c_double * 3), ("pos_iters", ctypes.c_int32), ("vel_iters", ctypes.c_int32),
                ("contact_offset", ctypes.c_double), ("limit_margin", ctypes.c_double),
                ("bias_coef", ctypes.c_double), ("max_depen_vel", ctypes.c_double),
                ("ground_friction", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile liboracle.so with the host compiler (no CUDA). Contraction of a*b+c into fused
    multiply-adds is off, so the oracle rounds the same way on every host (aarch64 gcc contracts by
    default, x86-64 gcc without FMA flags does not)."""
    stale = not os.path.exists(_LIB_PATH) or any(os.path.getmtime(s) > os.path.getmtime(_LIB_PATH) for s in _SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", tmp, os.path.join(_HERE, "oracle.cpp")]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.oracle_create.restype = ctypes.c_void_p
        L.oracle_create.argtypes = [ctypes.POINTER(_Models), I32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.POINTER(_Params)]
        L.oracle_destroy.argtypes = [ctypes.c_void_p]
        L.oracle_sizes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
        L.oracle_env_ngen.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.oracle_env_ngen.restype = ctypes.c_int32
        L.oracle_step.argtypes = [ctypes.c_void_p, D, D, D, D, ctypes.c_double, ctypes.c_int32, D, I32, I32,
                                  ctypes.POINTER(ctypes.c_uint32), ctypes.c_int32]
        L.oracle_step.restype = ctypes.c_int32
        L.oracle_step_flops.argtypes = [ctypes.c_void_p, D, D, D, D, ctypes.c_double, ctypes.c_int32]
        L.oracle_step_ext.argtypes = [ctypes.c_void_p, D, D, D, D, D, D, D, ctypes.c_double, ctypes.c_int32, D, D, D,
                                      I32, I32, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int32]
        L.oracle_step_ext.restype = ctypes.c_int32
        L.oracle_jacobian.argtypes = [ctypes.c_void_p, ctypes.c_int32, D, D, ctypes.c_int32, D]
        L.oracle_jacobian.restype = ctypes.c_int32
        L.oracle_step_flops.restype = ctypes.c_double
        L.oracle_step_f32.argtypes = [ctypes.c_void_p, D, D, D, D, ctypes.c_double, ctypes.c_int32, D]
        L.oracle_step_tangent.argtypes = [ctypes.c_void_p, D, D, D, D, D, D, D, D, ctypes.c_double, ctypes.c_int32,
                                          ctypes.c_int32, D, D, D]
        L.oracle_step_tangent_f32.argtypes = [ctypes.c_void_p, D, D, D, D, D, D, D, D, ctypes.c_double,
                                              ctypes.c_int32, D, D, D]
        L.oracle_step_f32.restype = ctypes.c_int32
        L.oracle_capsule_box.argtypes = [D, D, ctypes.c_double, D, D]
        L.oracle_capsule_box.restype = None
        for fn in ("oracle_aba", "oracle_rnea", "oracle_momentum"):
            getattr(L, fn).argtypes = [ctypes.c_void_p, ctypes.c_int32, D, D, D, D]
            getattr(L, fn).restype = ctypes.c_int32
        for fn in ("oracle_crba", "oracle_energy"):
            getattr(L, fn).argtypes = [ctypes.c_void_p, ctypes.c_int32, D, D, D]
            getattr(L, fn).restype = ctypes.c_int32
        L.oracle_rk4.argtypes = [ctypes.c_void_p, D, D, D, ctypes.c_double, ctypes.c_int32]
        L.oracle_rk4.restype = ctypes.c_int32
        L.oracle_link_pose.argtypes = [ctypes.c_void_p, ctypes.c_int32, D, D, ctypes.c_int32, D]
        L.oracle_link_pose.restype = ctypes.c_int32
        L.oracle_rows.argtypes = [ctypes.c_void_p, ctypes.c_int32, D, D, ctypes.c_int32, D, D, I32, I32, D, D, D,
                                  I32]
        L.oracle_rows.restype = ctypes.c_int32
        L.oracle_opcount_probe.argtypes = [ctypes.c_int32, ctypes.c_int32]
        L.oracle_opcount_probe.restype = ctypes.c_double
        _lib = L
    return _lib


def capsule_box(p0, p1, r, ext):
    """Capsule-box geometry in the box frame: t* and, for slots 0, 1, 2 (t = 0, 1, t*), the
    normal (box -> capsule), separation and contact point."""
    a = np.ascontiguousarray(p0, np.float64)
    b = np.ascontiguousarray(p1, np.float64)
    e = np.ascontiguousarray(ext, np.float64)
    out = np.zeros(25)
    lib().oracle_capsule_box(_dp(a), _dp(b), float(r), _dp(e), _dp(out))
    slots = [dict(n=out[1 + 7 * s:4 + 7 * s].copy(), d=out[4 + 7 * s], x=out[5 + 7 * s:8 + 7 * s].copy())
             for s in range(3)]
    slots.append(dict(clip=bool(out[22]), ta=out[23], tb=out[24]))
    return out[0], slots


def opcount_probe(which: int, n: int = 0) -> float:
    """Operations the counting scalar records for one primitive (see oracle_opcount_probe)."""
    return float(lib().oracle_opcount_probe(int(which), int(n)))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(D)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(I32)


class Oracle:
    """FP64 oracle for one workload (its models, env/actor map and solver parameters)."""

    def __init__(self, w):
        self.w = w
        L = lib()
        ms = w.models
        def cat(name, dt):
            parts = [np.asarray(getattr(m, name), dtype=dt).reshape(-1) for m in ms]
            out = np.ascontiguousarray(np.concatenate(parts), dtype=dt)
            return out if out.size else np.zeros(1, dt)  # keep a valid pointer for empty tables
        link_off = np.zeros(len(ms) + 1, np.int32)
        shape_off = np.zeros(len(ms) + 1, np.int32)
        for i, m in enumerate(ms):
            link_off[i + 1] = link_off[i] + m.n_links
            shape_off[i + 1] = shape_off[i] + m.n_shapes
        keep = dict(link_off=link_off, shape_off=shape_off)
        for name, dt in (("parent", np.int32), ("jtype", np.int32), ("axis", np.float64), ("ppos", np.float64),
                         ("pquat", np.float64), ("mass", np.float64), ("com", np.float64), ("inertia", np.float64),
                         ("armature", np.float64), ("damping", np.float64), ("lo", np.float64), ("hi", np.float64),
                         ("has_limit", np.int32), ("is_virtual", np.int32), ("shape_link", np.int32),
                         ("shape_type", np.int32), ("shape_size", np.float64), ("shape_pos", np.float64),
                         ("shape_quat", np.float64), ("shape_friction", np.float64)):
            keep[name] = cat(name, dt)
        keep["drive_kp"] = np.ascontiguousarray(np.concatenate([m.drive_gains()[0] for m in ms]), np.float64)
        keep["drive_kd"] = np.ascontiguousarray(np.concatenate([m.drive_gains()[1] for m in ms]), np.float64)
        if any(m.tendons for m in ms):
            tl = [t for m in ms for t in (m.tendons or [])]
            keep["tendon_off"] = np.cumsum([0] + [len(m.tendons or []) for m in ms]).astype(np.int32)
            keep["tendon_entry_off"] = np.cumsum([0] + [len(t.links) for t in tl]).astype(np.int32)
            keep["tendon_link"] = np.array([l for t in tl for l in t.links] or [0], np.int32)
            keep["tendon_coef"] = np.array([c for t in tl for c in t.coef] or [0.0], np.float64)
            for name, get in (("tendon_stiffness", lambda t: t.stiffness), ("tendon_damping", lambda t: t.damping),
                              ("tendon_rest", lambda t: t.rest),
                              ("tendon_lo", lambda t: t.limit[0] if t.limit else 0.0),
                              ("tendon_hi", lambda t: t.limit[1] if t.limit else 0.0)):
                keep[name] = np.array([get(t) for t in tl] or [0.0], np.float64)
            keep["tendon_has_limit"] = np.array([int(t.limit is not None) for t in tl] or [0], np.int32)
        md = _Models()
        md.n_models = len(ms)
        for k, v in keep.items():
            setattr(md, k, _ip(v) if v.dtype == np.int32 else _dp(v))
        p = _Params()
        for i in range(3):
            p.gravity[i] = float(w.params.gravity[i])
        p.pos_iters, p.vel_iters = int(w.params.pos_iters), int(w.params.vel_iters)
        p.contact_offset, p.limit_margin = float(w.params.contact_offset), float(w.params.limit_margin)
        p.bias_coef, p.max_depen_vel = float(w.params.bias_coef), float(w.params.max_depen_vel)
        p.ground_friction = float(w.params.ground_friction)
        self._eam = np.ascontiguousarray(w.env_actor_model, dtype=np.int32)
        self._keep = keep
        self.h = L.oracle_create(ctypes.byref(md), _ip(self._eam), w.actors_per_env, w.n_envs, ctypes.byref(p))
        sz = (ctypes.c_int64 * 6)()
        L.oracle_sizes(self.h, sz)
        self.N_A, self.N_D, self.N_B, self.contact_cap, self.max_gen, self.cache_len = [int(x) for x in sz]
        # solver impulse cache (warm start), one row per env; zero = no constraint active before
        self.cache = np.zeros((w.n_envs, max(self.cache_len, 1)))

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_destroy(self.h)
            self.h = None

    # -- batch step -------------------------------------------------------------------------
    def step(self, root: np.ndarray, dof: np.ndarray, act: np.ndarray, dt: Optional[float] = None,
             substeps: Optional[int] = None, n_threads: int = 1, pos_target=None, vel_target=None,
             body_force=None) -> Dict[str, np.ndarray]:
        """One env-step of every env. root (N_A,13), dof (N_D,2) and the solver impulse cache
        self.cache (n_envs, cache_len) are updated IN PLACE (float64 arrays); act is (N_D,);
        pos_target / vel_target (N_D,) are joint drive targets (0 when omitted) and body_force
        (N_B,6) external forces and torques (world axes, at each body's COM). Returns net contact
        forces (N_B,3), the joint forces of the last substep (N_D,), body states after the step
        (N_B,13: link origin, quaternion, velocity of the origin, angular velocity), the last
        substep's contact triples (n_envs, cap, 3), their counts, the per-env constraint-set
        signature and the number of failed envs."""
        dt = self.w.dt if dt is None else dt
        substeps = self.w.substeps if substeps is None else substeps
        assert root.dtype == np.float64 and root.flags.c_contiguous and root.shape == (self.N_A, 13)
        assert dof.dtype == np.float64 and dof.flags.c_contiguous and dof.shape == (self.N_D, 2)
        a = np.ascontiguousarray(act, dtype=np.float64).reshape(self.N_D)
        nf = np.zeros((self.N_B, 3))
        con = np.zeros((self.w.n_envs, self.contact_cap, 3), np.int32)
        nc = np.zeros(self.w.n_envs, np.int32)
        sig = np.zeros(self.w.n_envs, np.uint32)
        conv = [None if x is None else np.ascontiguousarray(x, dtype=np.float64).reshape(n)
                for x, n in ((pos_target, self.N_D), (vel_target, self.N_D), (body_force, self.N_B * 6))]
        pt, vt, bf = [None if x is None or x.size == 0 else _dp(x) for x in conv]  # conv keeps them alive
        df = np.zeros(self.N_D)
        bs = np.zeros((self.N_B, 13))
        bad = lib().oracle_step_ext(self.h, _dp(root), _dp(dof) if self.N_D else None, _dp(self.cache),
                                    _dp(a) if self.N_D else None, pt, vt, bf, float(dt), int(substeps),
                                    _dp(nf) if self.N_B else None, _dp(df) if self.N_D else None,
                                    _dp(bs) if self.N_B else None, _ip(con), _ip(nc),
                                    sig.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), int(n_threads))
        return dict(net_force=nf, dof_force=df, body_state=bs, contacts=con, n_contacts=nc, signature=sig,
                    n_failed=int(bad))

    def jacobian(self, env, root, dof, link):
        """World-axis Jacobian (6, env generalized DOFs) of env-local link `link`: rows [angular
        velocity; velocity of the link origin]."""
        root, dof = self._c(root), self._c(dof)
        out = np.zeros((6, self.ngen(env)))
        assert lib().oracle_jacobian(self.h, env, _dp(root), _dp(dof), link, _dp(out)) == 0
        return out

    def step_flops(self, root, dof, act, dt=None, substeps=None) -> float:
        """Floating-point operations of one env-step over all envs (state advanced in place)."""
        dt = self.w.dt if dt is None else dt
        substeps = self.w.substeps if substeps is None else substeps
        a = np.ascontiguousarray(act, dtype=np.float64).reshape(self.N_D)
        return float(lib().oracle_step_flops(self.h, _dp(root), _dp(dof) if self.N_D else None, _dp(self.cache),
                                             _dp(a) if self.N_D else None, float(dt), int(substeps)))

    def step_f32(self, root, dof, act, dt=None, substeps=None):
        """The identical step evaluated in single precision (conditioning probe; state and
        self.cache updated in place like step). Returns the net contact forces."""
        dt = self.w.dt if dt is None else dt
        substeps = self.w.substeps if substeps is None else substeps
        a = np.ascontiguousarray(act, dtype=np.float64).reshape(self.N_D)
        nf = np.zeros((self.N_B, 3))
        lib().oracle_step_f32(self.h, _dp(root), _dp(dof) if self.N_D else None, _dp(self.cache),
                              _dp(a) if self.N_D else None, float(dt), int(substeps), _dp(nf) if self.N_B else None)
        return nf

    def step_tangent(self, root, dof, act, droot, ddof, dact, dcache, dt=None, substeps=None, n_threads=1,
                     single=False, pos_target=None, vel_target=None, body_force=None):
        """One env-step in forward-mode dual numbers. root, dof and self.cache advance in place like
        step; droot (N_A,13), ddof (N_D,2) and dcache (n_envs, cache_len) hold the input tangent and
        are overwritten with the output tangent; dact (N_D,) is the actuation tangent; pos_target /
        vel_target (N_D,) are drive targets and body_force (N_B,6) external forces and torques
        (constants; 0 when omitted). single=True evaluates the
        identical derivative in single precision (conditioning probe). Returns the number of failed
        envs."""
        dt = self.w.dt if dt is None else dt
        substeps = self.w.substeps if substeps is None else substeps
        for x, shape in ((root, (self.N_A, 13)), (droot, (self.N_A, 13)), (dof, (self.N_D, 2)), (ddof, (self.N_D, 2)),
                         (dcache, self.cache.shape)):
            assert x.dtype == np.float64 and x.flags.c_contiguous and x.shape == shape
        a = np.ascontiguousarray(act, dtype=np.float64).reshape(self.N_D)
        da = np.ascontiguousarray(dact, dtype=np.float64).reshape(self.N_D)
        nd = self.N_D > 0
        args = (self.h, _dp(root), _dp(dof) if nd else None, _dp(self.cache), _dp(a) if nd else None, _dp(droot),
                _dp(ddof) if nd else None, _dp(dcache), _dp(da) if nd else None, float(dt), int(substeps))
        tg = [None if x is None else np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
              for x in (pos_target, vel_target, body_force)]  # kept alive through the call
        assert all(x is None or x.size == n for x, n in zip(tg, (self.N_D, self.N_D, self.N_B * 6)))
        tp = [None if x is None or x.size == 0 else _dp(x) for x in tg]
        if single:
            return int(lib().oracle_step_tangent_f32(*args, *tp))
        return int(lib().oracle_step_tangent(*args, int(n_threads), *tp))

    def rk4(self, root, dof, act, dt, nsteps) -> int:
        """Contact-free RK4 reference integration in place; returns 0, or -2 (nothing done) for
        models with ball joints."""
        a = np.ascontiguousarray(act, dtype=np.float64).reshape(self.N_D)
        return int(lib().oracle_rk4(self.h, _dp(root), _dp(dof) if self.N_D else None, _dp(a) if self.N_D else None,
                                    float(dt), int(nsteps)))

    # -- single-env helpers (root: (actors_per_env,13), dof: (env joint DOFs,2), float64) ---------
    def ngen(self, env=0) -> int:
        return int(lib().oracle_env_ngen(self.h, env))

    @staticmethod
    def _c(x):
        return np.ascontiguousarray(x, dtype=np.float64)

    def aba(self, env, root, dof, tau):
        root, dof, tau = self._c(root), self._c(dof), self._c(tau)
        out = np.zeros(self.ngen(env))
        assert lib().oracle_aba(self.h, env, _dp(root), _dp(dof), _dp(tau), _dp(out)) == 0
        return out

    def crba(self, env, root, dof):
        root, dof = self._c(root), self._c(dof)
        n = self.ngen(env)
        out = np.zeros((n, n))
        lib().oracle_crba(self.h, env, _dp(root), _dp(dof), _dp(out))
        return out

    def rnea(self, env, root, dof, qdd):
        root, dof, qdd = self._c(root), self._c(dof), self._c(qdd)
        out = np.zeros(self.ngen(env))
        lib().oracle_rnea(self.h, env, _dp(root), _dp(dof), _dp(qdd), _dp(out))
        return out

    def energy(self, env, root, dof):
        root, dof = self._c(root), self._c(dof)
        out = np.zeros(2)
        lib().oracle_energy(self.h, env, _dp(root), _dp(dof), _dp(out))
        return out

    def momentum(self, env, root, dof, qdd):
        root, dof, qdd = self._c(root), self._c(dof), self._c(qdd)
        out = np.zeros(12)
        lib().oracle_momentum(self.h, env, _dp(root), _dp(dof), _dp(qdd), _dp(out))
        return out[:6], out[6:]

    def link_pose(self, env, root, dof, link):
        root, dof = self._c(root), self._c(dof)
        out = np.zeros(12)
        assert lib().oracle_link_pose(self.h, env, _dp(root), _dp(dof), int(link), _dp(out)) == 0
        return out[:9].reshape(3, 3), out[9:]

    def rows(self, env, root, dof, cap=256):
        root, dof = self._c(root), self._c(dof)
        n = self.ngen(env)
        J = np.zeros((cap, n)); d = np.zeros(cap); A = np.zeros(cap)
        kind = np.zeros(cap, np.int32); link = np.zeros(cap, np.int32)
        x = np.zeros((cap, 3)); k = np.zeros((cap, 3)); info = np.zeros((cap, 3), np.int32)
        R = lib().oracle_rows(self.h, env, _dp(root), _dp(dof), cap, _dp(J), _dp(d), _ip(kind), _ip(link), _dp(x),
                              _dp(k), _dp(A), _ip(info))
        assert R >= 0
        return dict(J=J[:R], d=d[:R], kind=kind[:R], link=link[:R], x=x[:R], k=k[:R], A=A[:R], info=info[:R])
