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



def capsule_chain(n_links=17, radius=0.03, half_len=0.08, pitch=0.2, density=1000.0, gear=1.0):
    """A floating chain of n_links capsules along x joined end to end by hinges about their y axis
    (limits +-45 deg), lying on the ground: 17 links (32 lanes per env), 22 generalized DOFs, two
    contacts per capsule lying flat, so a substep can have more constraint rows (3 per contact,
    1 per limit) than a shared Y region sized for 32 rows holds. Each link's origin is its hinge;
    its capsule is centred half a pitch further along x."""
    m, inertia = W.capsule_mass_x(radius, half_len, density)
    bld = W._Builder("capsule_chain")
    prev = bld.link(-1, W.JOINT_FREE, mass=m, com=(pitch / 2, 0.0, 0.0), inertia=inertia)
    bld.shape(prev, W.SHAPE_CAPSULE, (radius, half_len), pos=(pitch / 2, 0.0, 0.0))
    for _ in range(n_links - 1):
        prev = bld.link(prev, W.JOINT_REVOLUTE, axis=(0.0, 1.0, 0.0), ppos=(pitch, 0.0, 0.0), mass=m,
                        com=(pitch / 2, 0.0, 0.0), inertia=inertia, armature=0.05, damping=0.2,
                        limit=(-np.pi / 4, np.pi / 4), gear=gear)
        bld.shape(prev, W.SHAPE_CAPSULE, (radius, half_len), pos=(pitch / 2, 0.0, 0.0))
    # the chain straight, 5 mm above the ground at q = 0; hinge noise lifts parts of it
    return bld.build(root_pos=(0.0, 0.0, radius + 0.005), dof_noise=0.05)

