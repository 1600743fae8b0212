"""Small hand-built scenes shared by the oracle pins and the GPU tests."""
import numpy as np

from paper_2108_10470_gb300 import workloads as W


def two_actor_env(cap_pos, cap_quat, box_pos, params=None):
    """Fixed-base actor holding one capsule (radius 0.02, half length 0.1) and a free 0.2 kg box
    (half extents 0.05)."""
    b = W._Builder("holder")
    root = b.link(-1, W.JOINT_FIXED, mass=1.0, inertia=(0.1, 0.1, 0.1, 0, 0, 0))
    for p, q in zip(cap_pos, cap_quat):
        b.shape(root, W.SHAPE_CAPSULE, (0.02, 0.1), pos=p, quat=q)
    holder = b.build()
    box = W.free_box(0.05, 0.05, 0.05, mass=0.2)
    w = W.Workload("pair", [holder, box], np.array([0, 1], np.int32), 2, 1, params or W.Params())
    root_st = np.zeros((2, 13))
    root_st[:, 6] = 1.0
    root_st[1, 0:3] = box_pos
    return w, root_st
