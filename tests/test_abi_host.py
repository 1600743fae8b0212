"""Host-side checks of the C ABI (no GPU): the library loads, exports every entry point that
include/sim.h declares, and rejects malformed models before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2108_10470_gb300 import build, sim, workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sim.h")


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return sim.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(sim_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("sim_create", "sim_step", "sim_get_view", "sim_set_root_state_indexed", "sim_set_dof_state_indexed",
              "sim_sync_status", "sim_destroy", "sim_error_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(sim.EXPORTED) == declared_functions()


def create(lib, models, n_envs=2, params=None, eam=None):
    arr, keep = sim.model_structs(models)
    p = sim.params_struct(params or W.Params())
    eam = np.zeros(n_envs, np.int32) if eam is None else np.asarray(eam, np.int32)
    h = ctypes.c_void_p()
    rc = lib.sim_create(arr, len(models), eam.ctypes.data_as(sim.I32), 1, n_envs, ctypes.byref(p), None, ctypes.byref(h))
    return rc, h


def test_valid_model_reaches_device_check(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible; this checks the no-device path")
    rc, _ = create(lib, [W.ant()])
    assert rc == -8  # SIM_ERR_NO_DEVICE: validation passed, no device


def bad(model, **kw):
    import dataclasses
    m = dataclasses.replace(model)
    for k, v in kw.items():
        setattr(m, k, v)
    return m


@pytest.mark.parametrize("case,code", [
    ("root_parent", -2), ("forward_parent", -2), ("root_joint", -2), ("joint_type", -2),
    ("neg_mass", -1), ("free_root_massless", -1), ("inertia_not_psd", -1), ("nan_axis", -1),
    ("zero_axis", -1), ("limits_swapped", -1), ("shape_type", -1), ("shape_on_virtual", -1),
    ("shape_size", -1), ("too_many_links", -4), ("ball_root", -2), ("ball_limit", -1), ("ball_drive", -1),
    ("ball_tendon", -1),
])
def test_malformed_models_rejected(lib, case, code):
    m = W.ant()
    if case == "root_parent":
        p = m.parent.copy(); p[0] = 0; m = bad(m, parent=p)
    elif case == "forward_parent":
        p = m.parent.copy(); p[3] = 5; m = bad(m, parent=p)
    elif case == "root_joint":
        j = m.jtype.copy(); j[0] = W.JOINT_REVOLUTE; m = bad(m, jtype=j)
    elif case == "joint_type":
        j = m.jtype.copy(); j[2] = 7; m = bad(m, jtype=j)
    elif case == "neg_mass":
        x = m.mass.copy(); x[3] = -1.0; m = bad(m, mass=x)
    elif case == "free_root_massless":
        x = m.mass.copy(); x[0] = 0.0; m = bad(m, mass=x)
    elif case == "inertia_not_psd":
        x = m.inertia.copy(); x[2] = [1.0, 1.0, 1.0, 5.0, 0.0, 0.0]; m = bad(m, inertia=x)
    elif case == "nan_axis":
        x = m.axis.copy(); x[1, 0] = np.nan; m = bad(m, axis=x)
    elif case == "zero_axis":
        x = m.axis.copy(); x[1] = 0.0; m = bad(m, axis=x)
    elif case == "limits_swapped":
        lo, hi = m.lo.copy(), m.hi.copy(); lo[1], hi[1] = 1.0, -1.0; m = bad(m, lo=lo, hi=hi)
    elif case == "shape_type":
        x = m.shape_type.copy(); x[0] = 9; m = bad(m, shape_type=x)
    elif case == "shape_on_virtual":
        v = m.is_virtual.copy(); v[1] = 1; m = bad(m, is_virtual=v)
    elif case == "shape_size":
        x = m.shape_size.copy(); x[1, 0] = 0.0; m = bad(m, shape_size=x)
    elif case == "too_many_links":
        rng = np.random.default_rng(0)
        m = W.random_tree(rng, 33, True)
    elif case == "ball_root":  # a ball joint attaches a child, never the root
        j = m.jtype.copy(); j[0] = W.JOINT_SPHERICAL; m = bad(m, jtype=j)
    elif case in ("ball_limit", "ball_drive", "ball_tendon"):  # ball joints take no limits, drives or tendons
        j = m.jtype.copy(); j[1] = W.JOINT_SPHERICAL
        m = bad(m, jtype=j, gear=np.concatenate([m.gear[:1], [1.0, 1.0], m.gear[1:]]))
        if case == "ball_limit":
            assert m.has_limit[1]
        else:
            h = m.has_limit.copy(); h[1] = 0; m = bad(m, has_limit=h)
            if case == "ball_drive":
                kp = np.zeros(m.n_links); kp[1] = 10.0; m = bad(m, drive_kp=kp, drive_kd=np.zeros(m.n_links))
            else:
                m = bad(m, tendons=[W.Tendon([1, 2], [1.0, 1.0], 1.0, 0.0, 0.0, None)])
    rc, _ = create(lib, [m])
    assert rc == code


def test_bad_batch_arguments(lib):
    rc, _ = create(lib, [W.ant()], n_envs=0)
    assert rc == -1
    rc, _ = create(lib, [W.ant()], n_envs=2, eam=[0, 1])  # model index out of range
    assert rc == -1
    rc, _ = create(lib, [W.ant()], params=W.Params(pos_iters=0))
    assert rc == -1


def test_handle_errors(lib):
    assert lib.sim_step(None, ctypes.c_float(0.01), 1) == -7
    assert lib.sim_destroy(None) == -7
    v = sim.sim_view()
    assert lib.sim_get_view(ctypes.c_void_p(12345), 0, ctypes.byref(v)) == -7
    assert lib.sim_error_string(-4) == b"environment exceeds kernel capacity"
