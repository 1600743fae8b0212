"""Thin Python binding of the C ABI in include/sim.h (argument marshalling only).

Every step of the physics runs in the CUDA library ``libartsim.so``; this module only converts a
:class:`~paper_2108_10470_gb300.workloads.Workload` into ``sim_model_desc`` structs, calls the
entry points of the same names, and wraps the library-owned device views as zero-copy torch
tensors (paper, Sec. "Tensor API": physics buffers wrapped as framework tensors without copying).
There is no fallback: if the library is missing or no GPU is visible, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from .build import LIB_PATH

SIM_OK = 0
ERRORS = {-1: "SIM_ERR_INVALID_ARG", -2: "SIM_ERR_TOPOLOGY", -3: "SIM_ERR_CUDA", -4: "SIM_ERR_CAPACITY",
          -5: "SIM_ERR_TIMEOUT", -6: "SIM_ERR_NONFINITE", -7: "SIM_ERR_HANDLE", -8: "SIM_ERR_NO_DEVICE"}
SIM_FLAG_SIGNATURE = 1
SIM_FLAG_PERSISTENT = 2
SIM_FLAG_GRAPH = 4
SIM_FLAG_BODY_FORCES = 8
SIM_FLAG_RIGID_BODY_STATE = 16
SIM_FLAG_DOF_FORCE = 32
SIM_FLAG_ROW_SOLVER = 64
SIM_FLAG_TANGENT_VJP = 128
(SIM_VIEW_ROOT_STATE, SIM_VIEW_DOF_STATE, SIM_VIEW_DOF_ACTUATION, SIM_VIEW_NET_CONTACT_FORCE,
 SIM_VIEW_CONTACT_PAIRS, SIM_VIEW_CONTACT_COUNT, SIM_VIEW_SIGNATURE, SIM_VIEW_STATUS,
 SIM_VIEW_IMPULSE_CACHE, SIM_VIEW_DOF_POSITION_TARGET, SIM_VIEW_DOF_VELOCITY_TARGET, SIM_VIEW_DOF_FORCE,
 SIM_VIEW_RIGID_BODY_STATE, SIM_VIEW_RIGID_BODY_FORCE) = range(14)
EXPORTED = ("sim_create", "sim_step", "sim_step_actuated", "sim_step_host", "sim_get_view", "sim_set_root_state_indexed",
            "sim_set_dof_state_indexed", "sim_set_stream", "sim_sync_status", "sim_get_sizes", "sim_destroy",
            "sim_error_string", "sim_last_error_message", "sim_probe_fp32_peak", "sim_step_static_scratch",
            "sim_get_type_config", "sim_set_type_config", "sim_autotune", "sim_step_vjp", "sim_step_jvp",
            "sim_get_max_dims", "sim_compute_mass_matrix", "sim_compute_jacobian", "sim_tape_size",
            "sim_step_taped", "sim_step_adjoint")

F = ctypes.POINTER(ctypes.c_float)


def _host_ptr(a: Optional[np.ndarray], need: int) -> Optional[int]:
    """Address of a float32, C-contiguous host array of at least `need` elements (None passes
    through as a null pointer)."""
    if a is None:
        return None
    if a.dtype != np.float32 or not a.flags.c_contiguous or a.size < need:
        raise ValueError(f"host buffer must be float32, C-contiguous, >= {need} elements")
    try:
        return ctypes.addressof(ctypes.c_char.from_buffer(a))  # writable buffers
    except (TypeError, ValueError):
        return a.ctypes.data  # read-only or empty arrays
I32 = ctypes.POINTER(ctypes.c_int32)
U8 = ctypes.POINTER(ctypes.c_uint8)


class sim_model_desc(ctypes.Structure):
    _fields_ = [("n_links", ctypes.c_int32), ("parent", I32), ("joint_type", I32), ("joint_axis", F),
                ("parent_pos", F), ("parent_quat", F), ("mass", F), ("com", F), ("inertia", F), ("armature", F),
                ("damping", F), ("limit_lo", F), ("limit_hi", F), ("has_limit", U8), ("is_virtual", U8),
                ("n_shapes", ctypes.c_int32), ("shape_link", I32), ("shape_type", I32), ("shape_size", F),
                ("shape_pos", F), ("shape_quat", F), ("shape_friction", F), ("drive_stiffness", F),
                ("drive_damping", F), ("n_tendons", ctypes.c_int32), ("tendon_joint_count", I32), ("tendon_link", I32),
                ("tendon_coef", F), ("tendon_stiffness", F), ("tendon_damping", F), ("tendon_rest_length", F),
                ("tendon_limit_lo", F), ("tendon_limit_hi", F), ("tendon_has_limit", U8)]


class sim_params(ctypes.Structure):
    _fields_ = [("gravity", ctypes.c_float * 3), ("pos_iters", ctypes.c_int32), ("vel_iters", ctypes.c_int32),
                ("contact_offset", ctypes.c_float), ("limit_margin", ctypes.c_float), ("bias_coef", ctypes.c_float),
                ("max_depen_vel", ctypes.c_float), ("ground_friction", ctypes.c_float), ("flags", ctypes.c_int32)]


class sim_view(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("ndim", ctypes.c_int32), ("shape", ctypes.c_int64 * 3),
                ("strides", ctypes.c_int64 * 3), ("dtype", ctypes.c_int32), ("device", ctypes.c_int32)]


_lib = None


class sim_state_buffers(ctypes.Structure):
    """Caller-owned device state of sim_step_static_scratch (one pointer per view)."""
    _fields_ = [("root_state", ctypes.c_void_p), ("dof_state", ctypes.c_void_p), ("dof_actuation", ctypes.c_void_p),
                ("net_contact_force", ctypes.c_void_p), ("impulse_cache", ctypes.c_void_p),
                ("contact_pairs", ctypes.c_void_p), ("contact_count", ctypes.c_void_p), ("signature", ctypes.c_void_p),
                ("status", ctypes.c_void_p)]


VJP_FIELDS = ("root_state", "dof_state", "dof_actuation", "impulse_cache", "grad_root_state", "grad_dof_state",
              "grad_impulse_cache", "grad_root_state_in", "grad_dof_state_in", "grad_dof_actuation",
              "grad_impulse_cache_in", "status")
JVP_FIELDS = ("root_state", "dof_state", "dof_actuation", "impulse_cache", "tan_root_state", "tan_dof_state",
              "tan_dof_actuation", "tan_impulse_cache", "root_state_out", "dof_state_out", "impulse_cache_out",
              "tan_root_state_out", "tan_dof_state_out", "tan_impulse_cache_out", "status")


class sim_vjp_buffers(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in VJP_FIELDS]


class sim_jvp_buffers(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in JVP_FIELDS]


ADJ_FIELDS = ("grad_root_state", "grad_dof_state", "grad_impulse_cache", "grad_root_state_in", "grad_dof_state_in",
              "grad_dof_actuation", "grad_impulse_cache_in", "status")


class sim_adjoint_buffers(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in ADJ_FIELDS]


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libartsim.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; build it with paper_2108_10470_gb300.build")
    L = ctypes.CDLL(path)
    L.sim_create.argtypes = [ctypes.POINTER(sim_model_desc), ctypes.c_int32, I32, ctypes.c_int32, ctypes.c_int32,
                             ctypes.POINTER(sim_params), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    L.sim_step.argtypes = [ctypes.c_void_p, ctypes.c_float, ctypes.c_int32]
    L.sim_step_actuated.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_int32]
    L.sim_step_host.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float,
                                ctypes.c_int32]
    L.sim_get_view.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(sim_view)]
    L.sim_set_root_state_indexed.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
    L.sim_set_dof_state_indexed.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
    L.sim_set_stream.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.sim_sync_status.argtypes = [ctypes.c_void_p, I32]
    L.sim_get_sizes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
    L.sim_destroy.argtypes = [ctypes.c_void_p]
    L.sim_error_string.argtypes = [ctypes.c_int]
    L.sim_error_string.restype = ctypes.c_char_p
    L.sim_last_error_message.argtypes = []
    L.sim_last_error_message.restype = ctypes.c_char_p
    L.sim_probe_fp32_peak.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    L.sim_step_static_scratch.argtypes = [ctypes.c_void_p, ctypes.POINTER(sim_state_buffers), ctypes.c_float,
                                          ctypes.c_int32]
    L.sim_get_type_config.argtypes = [ctypes.c_void_p, ctypes.c_int32, I32]
    L.sim_set_type_config.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.sim_autotune.argtypes = [ctypes.c_void_p, ctypes.c_float, ctypes.c_int32, ctypes.c_int32,
                               ctypes.POINTER(ctypes.c_double)]
    L.sim_step_vjp.argtypes = [ctypes.c_void_p, ctypes.POINTER(sim_vjp_buffers), ctypes.c_float, ctypes.c_int32]
    L.sim_step_jvp.argtypes = [ctypes.c_void_p, ctypes.POINTER(sim_jvp_buffers), ctypes.c_float, ctypes.c_int32]
    L.sim_get_max_dims.argtypes = [ctypes.c_void_p, I32, I32]
    L.sim_compute_mass_matrix.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.sim_compute_jacobian.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.sim_tape_size.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
    L.sim_step_taped.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_int32]
    L.sim_step_adjoint.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(sim_adjoint_buffers),
                                   ctypes.c_float, ctypes.c_int32]
    _lib = L  # every other entry point returns int, ctypes' default restype
    return L


class SimError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.sim_error_string(code).decode()
        extra = lib.sim_last_error_message().decode()
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({msg}){' - ' + extra if extra else ''}")
        self.code = code


def check(code: int, where: str) -> int:
    if code != SIM_OK:
        raise SimError(code, where)
    return code


def _f32(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(-1) if shape is None else
                             np.asarray(a, dtype=np.float32).reshape(shape))
    return a if a.size else np.zeros(1, np.float32)


class _DevArray:
    """__cuda_array_interface__ wrapper around a library-owned view (kept alive by the tensor)."""

    _TYPESTR = {0: "<f4", 1: "<i4", 2: "<u4"}

    def __init__(self, v: sim_view, owner):
        shape = tuple(int(v.shape[i]) for i in range(v.ndim))
        self.__cuda_array_interface__ = {"shape": shape, "typestr": self._TYPESTR[v.dtype],
                                         "data": (int(v.data or 0), False), "version": 2, "strides": None}
        self.owner = owner


def params_struct(p, flags: int = 0) -> sim_params:
    s = sim_params()
    for i in range(3):
        s.gravity[i] = float(p.gravity[i])
    s.pos_iters, s.vel_iters = int(p.pos_iters), int(p.vel_iters)
    s.contact_offset, s.limit_margin = float(p.contact_offset), float(p.limit_margin)
    s.bias_coef, s.max_depen_vel = float(p.bias_coef), float(p.max_depen_vel)
    s.ground_friction = float(p.ground_friction)
    s.flags = int(flags)
    return s


def model_structs(models):
    """sim_model_desc array for a list of workloads.Model (float32 copies kept alive)."""
    keep = []
    arr = (sim_model_desc * len(models))()
    for i, m in enumerate(models):
        d = arr[i]
        d.n_links = m.n_links
        fields = dict(parent=np.ascontiguousarray(m.parent, np.int32), joint_type=np.ascontiguousarray(m.jtype, np.int32),
                      joint_axis=_f32(m.axis), parent_pos=_f32(m.ppos), parent_quat=_f32(m.pquat), mass=_f32(m.mass),
                      com=_f32(m.com), inertia=_f32(m.inertia), armature=_f32(m.armature), damping=_f32(m.damping),
                      limit_lo=_f32(m.lo), limit_hi=_f32(m.hi),
                      has_limit=np.ascontiguousarray(m.has_limit, np.uint8),
                      is_virtual=np.ascontiguousarray(m.is_virtual, np.uint8))
        d.n_shapes = m.n_shapes
        if m.n_shapes:
            fields.update(shape_link=np.ascontiguousarray(m.shape_link, np.int32),
                          shape_type=np.ascontiguousarray(m.shape_type, np.int32), shape_size=_f32(m.shape_size),
                          shape_pos=_f32(m.shape_pos), shape_quat=_f32(m.shape_quat),
                          shape_friction=_f32(m.shape_friction))
        if m.drive_kp is not None or m.drive_kd is not None:
            kp, kd = m.drive_gains()
            fields.update(drive_stiffness=_f32(kp), drive_damping=_f32(kd))
        if m.tendons:
            tl = m.tendons
            d.n_tendons = len(tl)
            fields.update(tendon_joint_count=np.array([len(t.links) for t in tl], np.int32),
                          tendon_link=np.array([l for t in tl for l in t.links], np.int32),
                          tendon_coef=_f32([c for t in tl for c in t.coef]),
                          tendon_stiffness=_f32([t.stiffness for t in tl]), tendon_damping=_f32([t.damping for t in tl]),
                          tendon_rest_length=_f32([t.rest for t in tl]),
                          tendon_limit_lo=_f32([t.limit[0] if t.limit else 0.0 for t in tl]),
                          tendon_limit_hi=_f32([t.limit[1] if t.limit else 0.0 for t in tl]),
                          tendon_has_limit=np.array([int(t.limit is not None) for t in tl], np.uint8))
        for k, a in fields.items():
            keep.append(a)
            ctype = dict(sim_model_desc._fields_)[k]
            setattr(d, k, a.ctypes.data_as(ctype))
    return arr, keep


class Sim:
    """A simulation of one workload's environments on the current CUDA device.

    Views (torch tensors aliasing library memory, valid until :meth:`destroy`):
    ``root_state`` (N_A, 13), ``dof_state`` (N_D, 2), ``dof_actuation`` (N_D,),
    ``net_contact_force`` (N_B, 3), ``contact_pairs`` (n_envs, C, 3), ``contact_count``,
    ``signature``, ``status``, ``impulse_cache``, ``dof_position_target`` / ``dof_velocity_target``
    (N_D,), ``dof_force`` (N_D,), ``rigid_body_state`` (N_B, 13), ``rigid_body_force`` (N_B, 6).
    """

    def __init__(self, w, stream=None, flags: int = 0):
        import torch  # device memory and streams only

        L = load()
        self.w = w
        self.flags = int(flags)
        self._torch = torch
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        arr, keep = model_structs(w.models)
        self._keep = (arr, keep)
        eam = np.ascontiguousarray(w.env_actor_model, np.int32)
        p = params_struct(w.params, flags)
        h = ctypes.c_void_p()
        check(L.sim_create(arr, len(w.models), eam.ctypes.data_as(I32), w.actors_per_env, w.n_envs, ctypes.byref(p),
                           ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h)), "sim_create")
        self.h = h
        sz = (ctypes.c_int64 * 7)()
        check(L.sim_get_sizes(h, sz), "sim_get_sizes")
        self.N_A, self.N_D, self.N_B, self.pair_cap, self.cache_len, self.n_types, self.launches_per_step = \
            [int(x) for x in sz]
        names = ["root_state", "dof_state", "dof_actuation", "net_contact_force", "contact_pairs", "contact_count",
                 "signature", "status", "impulse_cache", "dof_position_target", "dof_velocity_target", "dof_force",
                 "rigid_body_state", "rigid_body_force"]
        for which, name in enumerate(names):
            setattr(self, name, self.view(which))

    def view(self, which: int):
        v = sim_view()
        check(load().sim_get_view(self.h, which, ctypes.byref(v)), "sim_get_view")
        t = self._torch.as_tensor(_DevArray(v, self), device=f"cuda:{v.device}")
        return t

    def step(self, dt: Optional[float] = None, substeps: Optional[int] = None):
        check(load().sim_step(self.h, float(self.w.dt if dt is None else dt),
                              int(self.w.substeps if substeps is None else substeps)), "sim_step")

    def step_actuated(self, act, dt: Optional[float] = None, substeps: Optional[int] = None):
        """The step with this step's DOF actuation forces taken from `act` (paper: applying the
        actuation force tensor, then simulating): a float32, contiguous torch tensor of at least N_D
        elements, on the handle's device (or in pinned host memory), which the step kernels read
        in place; the actuation view ends holding the forces, as after writing it and calling step.
        Other tensors are refused with ValueError before anything is launched."""
        torch = self._torch
        need = self.dof_actuation.numel()
        if isinstance(act, torch.Tensor) and act.device.type == "cpu" and act.is_pinned():
            if act.dtype != torch.float32 or not act.is_contiguous() or act.numel() < need:
                raise ValueError("act: a pinned host tensor must be float32, contiguous, with at least N_D elements")
            ptr = act.data_ptr()
        else:
            ptr = self._dev_ptr(act, "act", (torch.float32,), need)
        check(load().sim_step_actuated(self.h, ptr, float(self.w.dt if dt is None else dt),
                                       int(self.w.substeps if substeps is None else substeps)), "sim_step_actuated")

    def step_host(self, act: np.ndarray, root_out: Optional[np.ndarray], dof_out: Optional[np.ndarray],
                  dt: Optional[float] = None, substeps: Optional[int] = None):
        """End-to-end step from host buffers (float32, C-contiguous, at least the view's size; pinned
        memory is faster). The addresses go to the library as plain integers (a few hundred ns per
        buffer, against microseconds for ctypes pointer objects: this call runs every control step)."""
        check(load().sim_step_host(self.h, _host_ptr(act, self.N_D), _host_ptr(root_out, 13 * self.N_A),
                                   _host_ptr(dof_out, 2 * self.N_D), float(self.w.dt if dt is None else dt),
                                   int(self.w.substeps if substeps is None else substeps)), "sim_step_host")

    STATE_NAMES = ("root_state", "dof_state", "dof_actuation", "net_contact_force", "impulse_cache", "contact_pairs",
                   "contact_count", "signature", "status")

    # view whose dtype and size each caller-owned buffer of the VJP / JVP / static-scratch calls mirrors
    MIRRORS = {"root_state": "root_state", "dof_state": "dof_state", "dof_actuation": "dof_actuation",
               "impulse_cache": "impulse_cache", "net_contact_force": "net_contact_force",
               "contact_pairs": "contact_pairs", "contact_count": "contact_count", "signature": "signature",
               "status": "status"}

    def _dev_ptr(self, t, name: str, dtypes, need: int) -> int:
        """Address of a caller-owned device tensor after checking what the C ABI assumes of it: a
        torch tensor of one of `dtypes`, contiguous, on the handle's device, with at least `need`
        elements. Raises ValueError (before anything is launched) otherwise."""
        torch = self._torch
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name}: expected a torch tensor, got {type(t).__name__}")
        if t.dtype not in dtypes:
            raise ValueError(f"{name}: dtype {t.dtype}, expected {' or '.join(str(d) for d in dtypes)}")
        if t.device != self.root_state.device:
            raise ValueError(f"{name}: on {t.device}, the simulation is on {self.root_state.device}")
        if not t.is_contiguous():
            raise ValueError(f"{name}: must be contiguous")
        if t.numel() < need:
            raise ValueError(f"{name}: {t.numel()} elements, at least {need} needed")
        return t.data_ptr()

    def _mirror_ptr(self, t, name: str, view: str) -> int:
        """_dev_ptr for a buffer laid out like the view `view` (same dtype family and size)."""
        torch = self._torch
        v = getattr(self, view)
        dtypes = (torch.float32,) if v.dtype == torch.float32 else (torch.int32, getattr(torch, "uint32", torch.int32))
        return self._dev_ptr(t, name, dtypes, v.numel())

    def step_static_scratch(self, bufs: dict, dt: Optional[float] = None, substeps: Optional[int] = None):
        """The step on caller-owned device tensors (keys STATE_NAMES, each shaped and typed like the
        view of the same name), with the library's built-in scratch array: the call allocates no
        device memory."""
        io = sim_state_buffers(*[ctypes.c_void_p(self._mirror_ptr(bufs[k], k, k)) for k in self.STATE_NAMES])
        check(load().sim_step_static_scratch(self.h, ctypes.byref(io), float(self.w.dt if dt is None else dt),
                                             int(self.w.substeps if substeps is None else substeps)),
              "sim_step_static_scratch")

    def type_config(self, t: int) -> dict:
        """Launch knobs of env type t (see sim_get_type_config)."""
        out = (ctypes.c_int32 * 6)()
        check(load().sim_get_type_config(self.h, t, out), "sim_get_type_config")
        keys = ("lanes_per_env", "rows_global", "warps_per_cta", "n_envs", "min_lanes", "first_env")
        return dict(zip(keys, [int(x) for x in out]))

    def set_type_config(self, t: int, lanes_per_env: int, rows_global: int, warps_per_cta: int = 4):
        check(load().sim_set_type_config(self.h, t, lanes_per_env, rows_global, warps_per_cta), "sim_set_type_config")

    def autotune(self, reps: int = 5, dt: Optional[float] = None, substeps: Optional[int] = None) -> float:
        """Pick the fastest launch knobs on the current state (left unchanged); ms per step."""
        ms = ctypes.c_double(0.0)
        check(load().sim_autotune(self.h, float(self.w.dt if dt is None else dt),
                                  int(self.w.substeps if substeps is None else substeps), reps, ctypes.byref(ms)),
              "sim_autotune")
        return float(ms.value)

    def max_dims(self):
        n, l = ctypes.c_int32(0), ctypes.c_int32(0)
        check(load().sim_get_max_dims(self.h, ctypes.byref(n), ctypes.byref(l)), "sim_get_max_dims")
        return int(n.value), int(l.value)

    def compute_mass_matrix(self):
        """(n_envs, n_max, n_max) joint-space inertia at the current state (a new tensor)."""
        n, _ = self.max_dims()
        out = self._torch.zeros((self.w.n_envs, n, n), device=self.root_state.device)
        check(load().sim_compute_mass_matrix(self.h, ctypes.c_void_p(out.data_ptr())), "sim_compute_mass_matrix")
        return out

    def compute_jacobian(self):
        """(n_envs, L_max, 6, n_max) world-axis link Jacobians at the current state (a new tensor)."""
        n, lm = self.max_dims()
        out = self._torch.zeros((self.w.n_envs, lm, 6, n), device=self.root_state.device)
        check(load().sim_compute_jacobian(self.h, ctypes.c_void_p(out.data_ptr())), "sim_compute_jacobian")
        return out

    def _ptrs(self, fields, bufs):
        """Checked addresses of the VJP / JVP buffers (each laid out like the view its name ends in;
        missing or None entries pass as NULL)."""
        out = []
        for f in fields:
            t = bufs.get(f)
            if t is None:
                out.append(None)
                continue
            view = next(v for v in ("root_state", "dof_state", "dof_actuation", "impulse_cache", "status") if v in f)
            out.append(ctypes.c_void_p(self._mirror_ptr(t, f, view)))
        return out

    def step_vjp(self, bufs: dict, dt: Optional[float] = None, substeps: Optional[int] = None):
        """Vector-Jacobian product of one env-step at bufs' input state (keys VJP_FIELDS; device
        tensors in the views' layouts; missing output gradients count as zero)."""
        b = sim_vjp_buffers(*self._ptrs(VJP_FIELDS, bufs))
        check(load().sim_step_vjp(self.h, ctypes.byref(b), float(self.w.dt if dt is None else dt),
                                  int(self.w.substeps if substeps is None else substeps)), "sim_step_vjp")

    def step_jvp(self, bufs: dict, dt: Optional[float] = None, substeps: Optional[int] = None):
        """Jacobian-vector product of one env-step (keys JVP_FIELDS)."""
        b = sim_jvp_buffers(*self._ptrs(JVP_FIELDS, bufs))
        check(load().sim_step_jvp(self.h, ctypes.byref(b), float(self.w.dt if dt is None else dt),
                                  int(self.w.substeps if substeps is None else substeps)), "sim_step_jvp")

    def tape_floats(self, substeps: Optional[int] = None) -> Optional[int]:
        """Floats of one recorded step's tape, or None if the reverse pass does not cover this
        handle (an env type whose adjoint arena does not fit a CTA): the derivative then runs in
        forward mode (step_vjp)."""
        sub = int(self.w.substeps if substeps is None else substeps)
        cache = self.__dict__.setdefault("_tape_floats", {})
        if sub not in cache:
            out = ctypes.c_int64(0)
            rc = load().sim_tape_size(self.h, sub, ctypes.byref(out))
            if rc in (-1, -4):
                cache[sub] = None
            else:
                check(rc, "sim_tape_size")
                cache[sub] = int(out.value)
        return cache[sub]

    def step_taped(self, tape, dt: Optional[float] = None, substeps: Optional[int] = None):
        """sim_step on the handle's views that also records the step's tape (a float32 device
        tensor of at least tape_floats() elements)."""
        sub = int(self.w.substeps if substeps is None else substeps)
        need = self.tape_floats(sub)
        if need is None:
            raise ValueError("the reverse pass does not cover this handle")
        p = self._dev_ptr(tape, "tape", (self._torch.float32,), need)
        check(load().sim_step_taped(self.h, ctypes.c_void_p(p), float(self.w.dt if dt is None else dt), sub),
              "sim_step_taped")

    def step_adjoint(self, tape, bufs: dict, dt: Optional[float] = None, substeps: Optional[int] = None):
        """Vector-Jacobian product of the step recorded in `tape` (keys ADJ_FIELDS; output
        gradients may be missing or None: zero)."""
        sub = int(self.w.substeps if substeps is None else substeps)
        need = self.tape_floats(sub)
        if need is None:
            raise ValueError("the reverse pass does not cover this handle")
        p = self._dev_ptr(tape, "tape", (self._torch.float32,), need)
        b = sim_adjoint_buffers(*self._ptrs(ADJ_FIELDS, bufs))
        check(load().sim_step_adjoint(self.h, ctypes.c_void_p(p), ctypes.byref(b), float(self.w.dt if dt is None else dt),
                                      sub), "sim_step_adjoint")

    def _tape_rows(self, tapes, acts):
        """Checks tapes (steps x >= tape_floats(), row-strided) and acts (steps x N_D) once; returns
        (steps, address of tape 0, tape row stride in floats)."""
        f32 = (self._torch.float32,)
        steps = int(acts.shape[0])
        need = self.tape_floats()
        if need is None:
            raise ValueError("the reverse pass does not cover this handle")
        tstride = int(tapes.stride(0)) if tapes.dim() > 1 else need
        self._dev_ptr(tapes, "tapes", f32, need + tstride * (steps - 1))
        self._dev_ptr(acts, "acts", f32, self.dof_actuation.numel() * steps)
        return steps, tapes.data_ptr(), tstride

    def record_tapes(self, tapes, acts):
        """len(acts) steps from the handle's current state, step k with actuation acts[k] and its
        tape recorded in tapes[k] (sim_step_taped); the views end at the last step's state."""
        steps, t0, tstride = self._tape_rows(tapes, acts)
        L = load()
        dt, sub = float(self.w.dt), int(self.w.substeps)
        for k in range(steps):
            self.dof_actuation.copy_(acts[k])
            check(L.sim_step_taped(self.h, ctypes.c_void_p(t0 + 4 * tstride * k), dt, sub), "sim_step_taped")

    def reverse_rollout(self, tapes, acts, grads, g_acts, recorded: bool = False):
        """The reverse pass of len(acts) steps: unless `recorded` (tapes[k] already hold the steps,
        from record_tapes), each step is first re-run from the handle's current state with its tape
        recorded in tapes[k]; then the adjoints in reverse order from the final-state gradients
        grads = (root, dof, cache), the actuation gradients written into g_acts[k]. Returns the
        initial-state gradients. Every buffer is checked once here, then passed to the library as
        plain addresses (the per-step calls run in a loop of a few microseconds)."""
        torch = self._torch
        f32 = (torch.float32,)
        steps, t0, tstride = self._tape_rows(tapes, acts)
        self._dev_ptr(g_acts, "g_acts", f32, self.dof_actuation.numel() * steps)
        views = ("root_state", "dof_state", "impulse_cache")
        g = [self._mirror_ptr(x, f"grad {v}", v) for x, v in zip(grads, views)]
        sets = [tuple(torch.empty_like(getattr(self, v)) for v in views) for _ in range(2)]
        L = load()
        dt, sub = float(self.w.dt), int(self.w.substeps)
        nd = self.dof_actuation.numel()
        if not recorded:
            self.record_tapes(tapes, acts)
        b = sim_adjoint_buffers()
        out = grads
        for k in range(steps - 1, -1, -1):
            out = sets[k % 2]
            b.grad_root_state, b.grad_dof_state, b.grad_impulse_cache = g
            b.grad_root_state_in, b.grad_dof_state_in, b.grad_impulse_cache_in = [x.data_ptr() for x in out]
            b.grad_dof_actuation = g_acts.data_ptr() + 4 * nd * k
            b.status = None
            check(L.sim_step_adjoint(self.h, ctypes.c_void_p(t0 + 4 * tstride * k), ctypes.byref(b), dt, sub),
                  "sim_step_adjoint")
            g = [x.data_ptr() for x in out]
        return out

    def set_root_state_indexed(self, src, actor_idx):
        """src: (n, 13) float32 root states; actor_idx: n int32 actor indices (device tensors)."""
        n = int(actor_idx.numel())
        pi = self._dev_ptr(actor_idx, "actor_idx", (self._torch.int32,), n)
        ps = self._dev_ptr(src, "src", (self._torch.float32,), 13 * n)
        check(load().sim_set_root_state_indexed(self.h, ctypes.c_void_p(ps), ctypes.c_void_p(pi), n),
              "sim_set_root_state_indexed")

    def set_dof_state_indexed(self, src, env_idx):
        """src: n rows of (largest env DOF count) x 2 float32; env_idx: n int32 env indices."""
        n = int(env_idx.numel())
        if not hasattr(self, "_max_jdof"):
            self._max_jdof = max((self.w.env_jdof(e) for e in range(self.w.n_envs)), default=0)
        pi = self._dev_ptr(env_idx, "env_idx", (self._torch.int32,), n)
        ps = self._dev_ptr(src, "src", (self._torch.float32,), 2 * self._max_jdof * n)
        check(load().sim_set_dof_state_indexed(self.h, ctypes.c_void_p(ps), ctypes.c_void_p(pi), n),
              "sim_set_dof_state_indexed")

    def set_stream(self, stream):
        self._stream = stream
        check(load().sim_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), "sim_set_stream")

    def sync_status(self) -> int:
        bad = ctypes.c_int32(0)
        rc = load().sim_sync_status(self.h, ctypes.byref(bad))
        if rc not in (SIM_OK, -6):
            check(rc, "sim_sync_status")
        return int(bad.value)

    def destroy(self):
        if getattr(self, "h", None):
            check(load().sim_destroy(self.h), "sim_destroy")
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def probe_fp32_peak(iters: int = 20000, stream=None) -> float:
    """Measured FP32 FMA throughput of the current GPU (FLOP/s)."""
    out = ctypes.c_double(0.0)
    check(load().sim_probe_fp32_peak(ctypes.c_void_p(stream.cuda_stream if stream is not None else 0), int(iters),
                                     ctypes.byref(out)), "sim_probe_fp32_peak")
    return float(out.value)
