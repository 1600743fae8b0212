"""Synthetic articulation models and seeded inputs shaped like the paper's benchmark tasks.

The paper measures Ant, Humanoid and Shadow Hand environments (Sec. "Characterising Simulation
Performance"; simulation set-up table: Ant and Humanoid run joint torques at a 1/120 s simulation
step under a 1/60 s control step). Its robot assets are not available, so this module builds
synthetic models with the shapes and sizes of those workloads, plus the small models the physics
pins need (pendulum, cartpole, free box, free sphere, random trees).

This module holds model data and random draws only: no step of the physics method. Both the CUDA
path and the FP64 oracle consume what it produces.

Conventions shared by every consumer (a data format, not code):
  * joint types: 0 free root, 1 fixed, 2 revolute, 3 prismatic (link 0 is the root: free or fixed);
  * shape types: 0 sphere (size[0] = r), 1 capsule (size = r, half segment length; axis = local x),
    2 box (size = half extents);
  * quaternions are (x, y, z, w); inertia is (xx, yy, zz, xy, xz, yz) about the COM in link axes;
  * root state rows are [p 3 | quat 4 | v 3 | omega 3] in world axes, v being the velocity of the
    root origin; DOF state rows are [q, qd] (paper's "Physics state tensors" table).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

JOINT_FREE, JOINT_FIXED, JOINT_REVOLUTE, JOINT_PRISMATIC, JOINT_SPHERICAL = 0, 1, 2, 3, 4
# DOFs of each joint type (a ball joint: rotation vector and angular velocity, 3 each)
JOINT_NDOF = {JOINT_FREE: 0, JOINT_FIXED: 0, JOINT_REVOLUTE: 1, JOINT_PRISMATIC: 1, JOINT_SPHERICAL: 3}
SHAPE_SPHERE, SHAPE_CAPSULE, SHAPE_BOX = 0, 1, 2
IDENT_Q = (0.0, 0.0, 0.0, 1.0)


@dataclasses.dataclass
class Tendon:
    """Fixed tendon of one articulation: length l = sum_k coef[k] q(links[k]) over 1-DOF joints, a
    spring-damper on the length (force -stiffness (l - rest) - damping l_dot, applied to each joint
    as coef[k] times it) and optional length limits lo <= l <= hi."""
    links: List[int]
    coef: List[float]
    stiffness: float = 0.0
    damping: float = 0.0
    rest: float = 0.0
    limit: Optional[tuple] = None


@dataclasses.dataclass
class Model:
    """One articulation: links 0..L-1 with parent[i] < i, plus collision shapes."""

    name: str
    parent: np.ndarray
    jtype: np.ndarray
    axis: np.ndarray
    ppos: np.ndarray
    pquat: np.ndarray
    mass: np.ndarray
    com: np.ndarray
    inertia: np.ndarray
    armature: np.ndarray
    damping: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    has_limit: np.ndarray
    is_virtual: np.ndarray
    shape_link: np.ndarray
    shape_type: np.ndarray
    shape_size: np.ndarray
    shape_pos: np.ndarray
    shape_quat: np.ndarray
    shape_friction: np.ndarray
    gear: np.ndarray          # per joint DOF (action scale of the workload, not physics)
    root_pos: np.ndarray      # nominal root position of the initial state
    dof_noise: float = 0.0    # half-width of the uniform initial joint-position noise
    drive_kp: Optional[np.ndarray] = None  # per link: joint drive stiffness (None: no drives)
    drive_kd: Optional[np.ndarray] = None  # per link: joint drive damping
    tendons: Optional[List[Tendon]] = None   # fixed tendons (None: none)

    def drive_gains(self):
        """(kp, kd) per link, zeros where no drive is set."""
        z = np.zeros(self.n_links)
        kp = z if self.drive_kp is None else np.asarray(self.drive_kp, np.float64)
        kd = z if self.drive_kd is None else np.asarray(self.drive_kd, np.float64)
        return kp, kd

    @property
    def n_links(self) -> int:
        return int(self.parent.shape[0])

    @property
    def n_shapes(self) -> int:
        return int(self.shape_link.shape[0])

    @property
    def free_root(self) -> bool:
        return int(self.jtype[0]) == JOINT_FREE

    @property
    def n_jdof(self) -> int:
        return int(sum(JOINT_NDOF[int(t)] for t in self.jtype))

    def dof_links(self) -> List[int]:
        """The link of every joint DOF, in DOF order (a ball joint's link three times)."""
        return [i for i in range(self.n_links) for _ in range(JOINT_NDOF[int(self.jtype[i])])]

    @property
    def n_gen(self) -> int:
        return self.n_jdof + (6 if self.free_root else 0)

    @property
    def n_body(self) -> int:
        return int(np.sum(self.is_virtual == 0))

    @property
    def contact_cap(self) -> int:
        per = {SHAPE_SPHERE: 1, SHAPE_CAPSULE: 2, SHAPE_BOX: 8}
        return int(sum(per[int(t)] for t in self.shape_type))


class _Builder:
    """Accumulates links and shapes, then freezes them into a Model."""

    def __init__(self, name: str):
        self.name = name
        self.links: List[dict] = []
        self.shapes: List[dict] = []
        self.gear: List[float] = []
        self.tendons: List[Tendon] = []

    def tendon(self, links, coef, stiffness=0.0, damping=0.0, rest=0.0, limit=None):
        self.tendons.append(Tendon(list(links), [float(c) for c in coef], float(stiffness), float(damping),
                                   float(rest), limit))

    def link(self, parent, jtype, *, axis=(0, 0, 1), ppos=(0, 0, 0), pquat=IDENT_Q, mass=0.0, com=(0, 0, 0),
             inertia=(0, 0, 0, 0, 0, 0), armature=0.0, damping=0.0, limit=None, virtual=False, gear=1.0,
             drive=(0.0, 0.0)) -> int:
        lo, hi = (limit if limit is not None else (0.0, 0.0))
        self.links.append(dict(parent=parent, jtype=jtype, axis=axis, ppos=ppos, pquat=pquat, mass=mass, com=com,
                               inertia=inertia, armature=armature, damping=damping, lo=lo, hi=hi,
                               has_limit=int(limit is not None), is_virtual=int(virtual), kp=float(drive[0]),
                               kd=float(drive[1])))
        self.gear.extend([gear] * JOINT_NDOF[jtype])
        return len(self.links) - 1

    def shape(self, link, stype, size, pos=(0, 0, 0), quat=IDENT_Q, friction=1.0):
        sz = list(size) + [0.0] * (3 - len(size))
        self.shapes.append(dict(link=link, type=stype, size=sz, pos=pos, quat=quat, friction=friction))

    def build(self, root_pos=(0, 0, 0), dof_noise=0.0) -> Model:
        L = self.links
        S = self.shapes
        def f(k, w=None):
            a = np.array([l[k] for l in L], dtype=np.float64)
            return a.reshape(len(L), w) if w else a

        def sf(k, w=None):
            a = np.array([s[k] for s in S], dtype=np.float64)
            return a.reshape(len(S), w) if w else a

        return Model(
            name=self.name,
            parent=np.array([l["parent"] for l in L], dtype=np.int32),
            jtype=np.array([l["jtype"] for l in L], dtype=np.int32),
            axis=f("axis", 3), ppos=f("ppos", 3), pquat=f("pquat", 4), mass=f("mass"), com=f("com", 3),
            inertia=f("inertia", 6), armature=f("armature"), damping=f("damping"), lo=f("lo"), hi=f("hi"),
            has_limit=np.array([l["has_limit"] for l in L], dtype=np.int32),
            is_virtual=np.array([l["is_virtual"] for l in L], dtype=np.int32),
            shape_link=np.array([s["link"] for s in S], dtype=np.int32),
            shape_type=np.array([s["type"] for s in S], dtype=np.int32),
            shape_size=sf("size", 3) if S else np.zeros((0, 3)), shape_pos=sf("pos", 3) if S else np.zeros((0, 3)),
            shape_quat=sf("quat", 4) if S else np.zeros((0, 4)),
            shape_friction=sf("friction") if S else np.zeros((0,)),
            gear=np.array(self.gear, dtype=np.float64),
            root_pos=np.array(root_pos, dtype=np.float64),
            dof_noise=float(dof_noise),
            drive_kp=f("kp") if any(l["kp"] for l in L) else None,
            drive_kd=f("kd") if any(l["kd"] for l in L) else None,
            tendons=list(self.tendons) if self.tendons else None)


# ------------------------------------------------------------------------------------------------
# Mass properties of primitive solids (uniform density), used only to fill model tables.
def sphere_mass(r, rho):
    m = rho * 4.0 / 3.0 * math.pi * r ** 3
    i = 0.4 * m * r * r
    return m, (i, i, i, 0.0, 0.0, 0.0)


def capsule_mass_x(r, half_len, rho):
    """Capsule with its axis along local x: segment length 2*half_len, radius r."""
    L = 2.0 * half_len
    mc = rho * math.pi * r * r * L
    mh = rho * 4.0 / 3.0 * math.pi * r ** 3
    ia = mc * r * r / 2.0 + mh * 2.0 * r * r / 5.0
    ip = mc * (L * L / 12.0 + r * r / 4.0) + mh * (2.0 * r * r / 5.0 + L * L / 4.0 + 3.0 * L * r / 8.0)
    return mc + mh, (ia, ip, ip, 0.0, 0.0, 0.0)


def capsule_mass_along(r, half_len, rho, axis):
    """Capsule inertia for an axis that is one of the link's coordinate axes (0=x, 1=y, 2=z)."""
    m, (ia, ip, _, _, _, _) = capsule_mass_x(r, half_len, rho)
    d = [ip, ip, ip]
    d[axis] = ia
    return m, (d[0], d[1], d[2], 0.0, 0.0, 0.0)


def box_mass(hx, hy, hz, m):
    return m, (m * (hy * hy + hz * hz) / 3.0, m * (hx * hx + hz * hz) / 3.0, m * (hx * hx + hy * hy) / 3.0, 0.0, 0.0, 0.0)


def quat_axis_angle(axis, ang):
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    s = math.sin(ang / 2.0)
    return (a[0] * s, a[1] * s, a[2] * s, math.cos(ang / 2.0))


# Capsule axis is local x; these quaternions turn it onto -z or +y.
Q_X_TO_NEG_Z = quat_axis_angle((0, 1, 0), math.pi / 2)
Q_X_TO_Y = quat_axis_angle((0, 0, 1), math.pi / 2)


# ------------------------------------------------------------------------------------------------
# Models.
def pendulum(mass=0.5, length=1.0) -> Model:
    """Fixed pivot + uniform thin rod hanging along -z, hinge about y (no shapes)."""
    b = _Builder("pendulum")
    b.link(-1, JOINT_FIXED, mass=1.0, inertia=(1, 1, 1, 0, 0, 0))
    i_perp = mass * length * length / 12.0
    b.link(0, JOINT_REVOLUTE, axis=(0, 1, 0), mass=mass, com=(0, 0, -length / 2.0),
           inertia=(i_perp, i_perp, 1e-6, 0, 0, 0))
    return b.build()


def ball_pendulum(mass=0.5, length=1.0, inertia=None, com=None, name="ball_pendulum") -> Model:
    """Fixed pivot + a body on a ball joint (3 DOF: rotation vector, angular velocity in the body
    frame); by default the uniform thin rod of `pendulum` hanging along -z (no shapes)."""
    b = _Builder(name)
    b.link(-1, JOINT_FIXED, mass=1.0, inertia=(1, 1, 1, 0, 0, 0))
    i_perp = mass * length * length / 12.0
    b.link(0, JOINT_SPHERICAL, mass=mass, com=(0, 0, -length / 2.0) if com is None else com,
           inertia=(i_perp, i_perp, 1e-6, 0, 0, 0) if inertia is None else inertia)
    return b.build()


def cartpole(hanging=False, with_limits=False) -> Model:
    """Fixed rail, prismatic cart (1 kg) along x, revolute pole (0.5 kg uniform rod, 1 m) about y.

    hanging=False puts the pole COM 0.5 m above the pivot (the control task); hanging=True puts it
    below (the free-oscillation pin).
    """
    b = _Builder("cartpole_hanging" if hanging else "cartpole")
    b.link(-1, JOINT_FIXED, mass=1.0, inertia=(1, 1, 1, 0, 0, 0))
    cart = b.link(0, JOINT_PRISMATIC, axis=(1, 0, 0), mass=1.0, inertia=box_mass(0.2, 0.1, 0.05, 1.0)[1],
                  limit=(-4.0, 4.0) if with_limits else None, gear=10.0)
    i_perp = 0.5 * 1.0 / 12.0
    zc = -0.5 if hanging else 0.5
    b.link(cart, JOINT_REVOLUTE, axis=(0, 1, 0), mass=0.5, com=(0, 0, zc), inertia=(i_perp, i_perp, 1e-6, 0, 0, 0),
           gear=0.0)
    return b.build(root_pos=(0.0, 0.0, 2.0), dof_noise=0.2)


ANT_TORSO_R = 0.25
ANT_LEG_R = 0.08
ANT_THIGH = 0.28
ANT_SHIN = 0.40
ANT_KNEE_TILT = math.pi / 4  # shin points outward and 45 degrees down at q = 0


def ant(density=5.0, armature=1.0, damping=1.0, gear=15.0, friction=1.0, ball_hips=False, tendons=False) -> Model:
    """Ant-like quadruped: floating sphere torso (r 0.25, 0.33 kg), four legs at azimuths
    45/135/225/315 degrees, each a hip hinge about z (+-30 deg) carrying a 0.28 m thigh capsule and a
    knee hinge about the horizontal axis perpendicular to the leg (+-70 deg) carrying a 0.40 m shin
    capsule (radius 0.08). 9 links, 8 joint DOF, 14 generalized DOF. With ball_hips, each hip is a
    ball joint (3 DOF, no limits): 16 joint DOF, 22 generalized DOF. With tendons (hinge hips only):
    a spring-damper tendon on leg 0's hip and knee, a length-limited tendon on the knees of legs 1
    and 2, and an equality tendon on the hips of legs 2 and 3."""
    b = _Builder("ball_ant" if ball_hips else ("tendon_ant" if tendons else "ant"))
    mt, it = sphere_mass(ANT_TORSO_R, density)
    torso = b.link(-1, JOINT_FREE, mass=mt, inertia=it)
    b.shape(torso, SHAPE_SPHERE, (ANT_TORSO_R,), friction=friction)
    for k in range(4):
        phi = math.radians(45 + 90 * k)
        m1, i1 = capsule_mass_x(ANT_LEG_R, ANT_THIGH / 2, density)
        thigh = b.link(torso, JOINT_SPHERICAL if ball_hips else JOINT_REVOLUTE, axis=(0, 0, 1),
                       ppos=(ANT_TORSO_R * math.cos(phi), ANT_TORSO_R * math.sin(phi), 0.0),
                       pquat=quat_axis_angle((0, 0, 1), phi), mass=m1, com=(ANT_THIGH / 2, 0, 0), inertia=i1,
                       armature=armature, damping=damping,
                       limit=None if ball_hips else (-math.radians(30), math.radians(30)), gear=gear)
        b.shape(thigh, SHAPE_CAPSULE, (ANT_LEG_R, ANT_THIGH / 2), pos=(ANT_THIGH / 2, 0, 0), friction=friction)
        m2, i2 = capsule_mass_x(ANT_LEG_R, ANT_SHIN / 2, density)
        shin = b.link(thigh, JOINT_REVOLUTE, axis=(0, 1, 0), ppos=(ANT_THIGH, 0, 0),
                      pquat=quat_axis_angle((0, 1, 0), ANT_KNEE_TILT), mass=m2, com=(ANT_SHIN / 2, 0, 0), inertia=i2,
                      armature=armature, damping=damping, limit=(-math.radians(70), math.radians(70)), gear=gear)
        b.shape(shin, SHAPE_CAPSULE, (ANT_LEG_R, ANT_SHIN / 2), pos=(ANT_SHIN / 2, 0, 0), friction=friction)
    if tendons and not ball_hips:  # leg k: thigh link 1 + 2k, shin link 2 + 2k
        b.tendon([1, 2], (1.0, -0.5), stiffness=30.0, damping=2.0, rest=0.1)
        b.tendon([4, 6], (1.0, 1.0), limit=(-0.1, 0.1))
        b.tendon([5, 7], (1.0, -1.0), limit=(0.0, 0.0))
    # lowest point at q = 0: shin tip minus its radius; start it 5 mm above the ground
    z0 = ANT_SHIN * math.sin(ANT_KNEE_TILT) + ANT_LEG_R + 0.005
    return b.build(root_pos=(0.0, 0.0, z0), dof_noise=0.1)


def humanoid(density=1000.0, damping=0.5, friction=1.0, ball_joints=False) -> Model:
    """Humanoid-like biped: 13 bodies (capsules and spheres) on a floating torso, 21 revolute DOF.
    Multi-axis joints (abdomen 3, hips 3, ankles 2, shoulders 2) are chains of 1-DOF hinges through
    massless virtual links; the head is welded to the torso by a fixed joint. Gears 50-150 N m,
    armature 0.1 * gear / 50 kg m^2 (0.1-0.3: with lighter rotors, e.g. 0.02 * gear / 50, random
    150 N m torques drive joint rates to ~100 rad/s, where the explicit 1/120 s substeps diverge in
    the FP64 oracle and on the GPU alike). 23 links, 21 joint DOF, 27 generalized DOF. With
    ball_joints, the abdomen and the hips are ball joints (3 DOF each, no limits) instead of hinge
    chains: 17 links, 21 joint DOF."""
    b = _Builder("ball_humanoid" if ball_joints else "humanoid")
    deg = math.radians
    ARM = 0.1

    def hinge(parent, axis, limit, gear, ppos=(0, 0, 0), body=None):
        """body=None -> virtual link; else (mass, com, inertia)."""
        if body is None:
            return b.link(parent, JOINT_REVOLUTE, axis=axis, ppos=ppos, armature=ARM * gear / 50, damping=damping,
                          limit=(deg(limit[0]), deg(limit[1])), virtual=True, gear=gear)
        m, c, inn = body
        return b.link(parent, JOINT_REVOLUTE, axis=axis, ppos=ppos, mass=m, com=c, inertia=inn,
                      armature=ARM * gear / 50, damping=damping, limit=(deg(limit[0]), deg(limit[1])), gear=gear)

    mt, it = capsule_mass_along(0.07, 0.07, density, 1)
    torso = b.link(-1, JOINT_FREE, mass=mt, inertia=it)
    b.shape(torso, SHAPE_CAPSULE, (0.07, 0.07), quat=Q_X_TO_Y, friction=friction)
    mh, ih = sphere_mass(0.09, density)
    head = b.link(torso, JOINT_FIXED, ppos=(0, 0, 0.19), mass=mh, inertia=ih)
    b.shape(head, SHAPE_SPHERE, (0.09,), friction=friction)
    def ball(parent, gear, ppos, body):
        m, c, inn = body
        return b.link(parent, JOINT_SPHERICAL, ppos=ppos, mass=m, com=c, inertia=inn, armature=ARM * gear / 50,
                      damping=damping, gear=gear)

    # abdomen z, y, x -> pelvis
    mp, ip = capsule_mass_along(0.09, 0.07, density, 1)
    if ball_joints:
        pelvis = ball(torso, 100, (0, 0, -0.26), (mp, (0, 0, 0), ip))
    else:
        v = hinge(torso, (0, 0, 1), (-45, 45), 100, ppos=(0, 0, -0.26))
        v = hinge(v, (0, 1, 0), (-75, 30), 100)
        pelvis = hinge(v, (1, 0, 0), (-35, 35), 100, body=(mp, (0, 0, 0), ip))
    b.shape(pelvis, SHAPE_CAPSULE, (0.09, 0.07), quat=Q_X_TO_Y, friction=friction)
    for side in (-1.0, 1.0):
        # hip x, z, y -> thigh
        m, inn = capsule_mass_along(0.06, 0.17, density, 2)
        if ball_joints:
            thigh = ball(pelvis, 125, (0, 0.1 * side, -0.04), (m, (0, 0, -0.17), inn))
        else:
            v = hinge(pelvis, (1, 0, 0), (-25, 5) if side < 0 else (-5, 25), 125, ppos=(0, 0.1 * side, -0.04))
            v = hinge(v, (0, 0, 1), (-60, 35) if side < 0 else (-35, 60), 125)
            thigh = hinge(v, (0, 1, 0), (-110, 20), 150, body=(m, (0, 0, -0.17), inn))
        b.shape(thigh, SHAPE_CAPSULE, (0.06, 0.17), pos=(0, 0, -0.17), quat=Q_X_TO_NEG_Z, friction=friction)
        # knee -> shin
        m, inn = capsule_mass_along(0.049, 0.15, density, 2)
        shin = hinge(thigh, (0, 1, 0), (-160, -2), 100, ppos=(0, 0, -0.40), body=(m, (0, 0, -0.15), inn))
        b.shape(shin, SHAPE_CAPSULE, (0.049, 0.15), pos=(0, 0, -0.15), friction=friction, quat=Q_X_TO_NEG_Z)
        # ankle y, x -> foot (capsule pointing forward)
        v = hinge(shin, (0, 1, 0), (-50, 50), 75, ppos=(0, 0, -0.36))
        m, inn = capsule_mass_along(0.04, 0.07, density, 0)
        foot = hinge(v, (1, 0, 0), (-35, 35), 50, body=(m, (0.05, 0, -0.03), inn))
        b.shape(foot, SHAPE_CAPSULE, (0.04, 0.07), pos=(0.05, 0, -0.03), friction=friction)
    for side in (-1.0, 1.0):
        # shoulder (2) -> upper arm, elbow -> lower arm
        v = hinge(torso, (1, 0, 0), (-85, 60) if side < 0 else (-60, 85), 75, ppos=(0, 0.17 * side, 0.06))
        m, inn = capsule_mass_along(0.04, 0.14, density, 2)
        upper = hinge(v, (0, 1, 0), (-85, 60), 75, body=(m, (0, 0, -0.14), inn))
        b.shape(upper, SHAPE_CAPSULE, (0.04, 0.14), pos=(0, 0, -0.14), quat=Q_X_TO_NEG_Z, friction=friction)
        m, inn = capsule_mass_along(0.031, 0.13, density, 2)
        lower = hinge(upper, (0, 1, 0), (-90, 50), 50, ppos=(0, 0, -0.29), body=(m, (0, 0, -0.13), inn))
        b.shape(lower, SHAPE_CAPSULE, (0.031, 0.13), pos=(0, 0, -0.13), quat=Q_X_TO_NEG_Z, friction=friction)
    # lowest point at q = 0: foot capsule bottom = torso - (0.26 + 0.04 + 0.40 + 0.36 + 0.03 + 0.04)
    z0 = 0.26 + 0.04 + 0.40 + 0.36 + 0.03 + 0.04 + 0.005
    return b.build(root_pos=(0.0, 0.0, z0), dof_noise=0.1)


HAND_HEIGHT = 0.5   # palm centre above the ground
CUBE_HALF = 0.0325  # 6.5 cm cube


def hand(density=1000.0, armature=0.01, damping=0.05, gear=0.5, friction=1.0, coupled=False) -> Model:
    """Fixed-base five-finger hand, palm up, shaped like the paper's 24-DOF Shadow Hand: wrist 2 DOF,
    index / middle / ring 4 DOF each (abduction + three flexions), little 5 (metacarpal + 4), thumb
    5; multi-axis joints are chains through massless virtual links; every joint is limited to
    +-90 degrees. Capsule palm and phalanges (radius 1 cm), 16 shapes. 25 links, 24 DOF.
    coupled=True adds a fixed tendon per long finger holding its middle and distal flexions equal
    (length q_middle - q_distal with limits [0, 0]), as the Shadow Hand couples them."""
    b = _Builder("hand")
    lim = (-math.pi / 2, math.pi / 2)

    def hinge(parent, axis, ppos=(0, 0, 0), body=None):
        if body is None:
            return b.link(parent, JOINT_REVOLUTE, axis=axis, ppos=ppos, armature=armature, damping=damping,
                          limit=lim, virtual=True, gear=gear)
        m, c, inn = body
        return b.link(parent, JOINT_REVOLUTE, axis=axis, ppos=ppos, mass=m, com=c, inertia=inn, armature=armature,
                      damping=damping, limit=lim, gear=gear)

    def phalanx(parent, axis, ppos, half, r=0.01):
        m, inn = capsule_mass_x(r, half, density)
        link = hinge(parent, axis, ppos, body=(m, (half, 0, 0), inn))
        b.shape(link, SHAPE_CAPSULE, (r, half), pos=(half, 0, 0), friction=friction)
        return link

    forearm = b.link(-1, JOINT_FIXED, mass=1.0, inertia=(0.01, 0.01, 0.01, 0, 0, 0))
    v = hinge(forearm, (0, 1, 0))
    mp, ip = capsule_mass_x(0.025, 0.035, density)
    palm = hinge(v, (1, 0, 0), body=(mp, (0, 0, 0), ip))
    b.shape(palm, SHAPE_CAPSULE, (0.025, 0.035), friction=friction)
    lens = (0.0225, 0.0125, 0.01)  # half lengths of proximal, middle, distal phalanges

    def finger(parent, base):
        a = hinge(parent, (0, 0, 1), base)  # abduction (virtual)
        p = phalanx(a, (0, 1, 0), (0, 0, 0), lens[0])
        m = phalanx(p, (0, 1, 0), (2 * lens[0], 0, 0), lens[1])
        d = phalanx(m, (0, 1, 0), (2 * lens[1], 0, 0), lens[2])
        if coupled:
            b.tendon([m, d], (1.0, -1.0), limit=(0.0, 0.0))

    for y in (0.033, 0.011, -0.011):  # index, middle, ring
        finger(palm, (0.06, y, 0.0))
    mm_, im_ = capsule_mass_x(0.01, 0.015, density)
    meta = hinge(palm, (1, 0, 0), (0.03, -0.033, 0.0), body=(mm_, (0.015, 0, 0), im_))  # little metacarpal
    finger(meta, (0.03, 0.0, 0.0))
    # thumb: base rotation (virtual) and metacarpal, then three flexions
    t0 = hinge(palm, (1, 0, 0), (0.0, 0.045, 0.0))
    tm = hinge(t0, (0, 0, 1), body=(mm_, (0.015, 0, 0), im_))
    tp = phalanx(tm, (0, 1, 0), (0.03, 0, 0), lens[0])
    tq = phalanx(tp, (0, 1, 0), (2 * lens[0], 0, 0), lens[1])
    phalanx(tq, (0, 1, 0), (2 * lens[1], 0, 0), lens[2])
    return b.build(root_pos=(0.0, 0.0, HAND_HEIGHT), dof_noise=0.1)


def cube(mass=0.1, friction=1.0) -> Model:
    """Free 6.5 cm, 0.1 kg cube resting 2 mm above the hand's palm."""
    m = free_box(CUBE_HALF, CUBE_HALF, CUBE_HALF, mass=mass, friction=friction,
                 z=HAND_HEIGHT + 0.025 + CUBE_HALF + 0.002)
    m.name = "cube"
    m.root_pos = np.array([0.03, 0.0, HAND_HEIGHT + 0.025 + CUBE_HALF + 0.002])
    return m


def free_box(hx=0.1, hy=0.1, hz=0.1, mass=1.0, friction=1.0, z=None) -> Model:
    b = _Builder("box")
    m, inn = box_mass(hx, hy, hz, mass)
    r = b.link(-1, JOINT_FREE, mass=m, inertia=inn)
    b.shape(r, SHAPE_BOX, (hx, hy, hz), friction=friction)
    return b.build(root_pos=(0.0, 0.0, hz if z is None else z))


def free_sphere(r=0.1, mass=1.0, friction=1.0, z=None) -> Model:
    b = _Builder("sphere")
    m, inn = sphere_mass(r, 1.0)
    inn = tuple(x * mass / m for x in inn)
    rl = b.link(-1, JOINT_FREE, mass=mass, inertia=inn)
    b.shape(rl, SHAPE_SPHERE, (r,), friction=friction)
    return b.build(root_pos=(0.0, 0.0, r if z is None else z))


def random_tree(rng: np.random.Generator, n_links: int, floating: bool, name="random_tree",
                allow_fixed=True, ball_joints=False) -> Model:
    """Random tree (parent[i] < i) with mixed revolute / prismatic / fixed joints (and ball joints
    when ball_joints), random offsets, orientations, axes and SPD inertias; no shapes. The draws of
    a tree without ball joints do not change with the option."""
    b = _Builder(name)

    def rand_inertia():
        # principal moments satisfying the triangle inequality, rotated by a random rotation
        a = rng.uniform(0.02, 0.25, size=3)  # d = (a0+a1, a1+a2, a0+a2) obeys the triangle inequality
        d = np.array([a[0] + a[1], a[1] + a[2], a[0] + a[2]])
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        x, y, z, w = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                      [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                      [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
        I = R @ np.diag(d) @ R.T
        return (I[0, 0], I[1, 1], I[2, 2], I[0, 1], I[0, 2], I[1, 2])

    def rand_quat():
        q = rng.normal(size=4)
        return tuple(q / np.linalg.norm(q))

    def rand_axis():
        a = rng.normal(size=3)
        return tuple(a / np.linalg.norm(a))

    b.link(-1, JOINT_FREE if floating else JOINT_FIXED, mass=float(rng.uniform(0.5, 2.0)),
           com=tuple(rng.uniform(-0.1, 0.1, 3)), inertia=rand_inertia())
    for i in range(1, n_links):
        par = int(rng.integers(0, i))
        choices = [JOINT_REVOLUTE, JOINT_REVOLUTE, JOINT_PRISMATIC] + ([JOINT_FIXED] if allow_fixed else []) + \
            ([JOINT_SPHERICAL, JOINT_SPHERICAL] if ball_joints else [])
        jt = int(rng.choice(choices))
        b.link(par, jt, axis=rand_axis(), ppos=tuple(rng.uniform(-0.4, 0.4, 3)), pquat=rand_quat(),
               mass=float(rng.uniform(0.2, 2.0)), com=tuple(rng.uniform(-0.2, 0.2, 3)), inertia=rand_inertia(),
               armature=float(rng.uniform(0.0, 0.1)))
    return b.build()


# ------------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    """Solver parameters (paper's simulation-parameter table: gravity, position / velocity
    iterations, max bias coefficient, friction, rest / contact offsets) with this project's values."""

    gravity: Sequence[float] = (0.0, 0.0, -9.81)
    pos_iters: int = 4
    vel_iters: int = 1
    contact_offset: float = 0.02
    limit_margin: float = 0.1
    bias_coef: float = 1.0
    max_depen_vel: float = 5.0
    ground_friction: float = 1.0


@dataclasses.dataclass
class Workload:
    """A batch of environments: env e holds actors env_actor_model[e*A:(e+1)*A] (indices into
    models), plus the step's dt / substeps."""

    name: str
    models: List[Model]
    env_actor_model: np.ndarray
    actors_per_env: int
    n_envs: int
    params: Params
    dt: float = 1.0 / 60.0
    substeps: int = 2

    def actor_models(self, env: int) -> List[Model]:
        """The env's actors in order (entries of -1 pad envs that have fewer actors)."""
        A = self.actors_per_env
        return [self.models[int(m)] for m in self.env_actor_model[env * A:(env + 1) * A] if m >= 0]

    @property
    def n_actors(self) -> int:
        return int(np.sum(np.asarray(self.env_actor_model) >= 0))

    def env_actor_count(self, env: int) -> int:
        return len(self.actor_models(env))

    def env_jdof(self, env: int) -> int:
        return sum(m.n_jdof for m in self.actor_models(env))

    def env_body(self, env: int) -> int:
        return sum(m.n_body for m in self.actor_models(env))

    @property
    def n_dof(self) -> int:
        return sum(self.env_jdof(e) for e in range(self.n_envs)) if len(self.models) > 1 else \
            self.n_envs * self.env_jdof(0)

    @property
    def n_body(self) -> int:
        return sum(self.env_body(e) for e in range(self.n_envs)) if len(self.models) > 1 else \
            self.n_envs * self.env_body(0)

    def subset(self, envs: Sequence[int]) -> "Workload":
        A = self.actors_per_env
        idx = np.concatenate([np.arange(e * A, (e + 1) * A) for e in envs]) if len(envs) else np.zeros(0, np.int64)
        return dataclasses.replace(self, env_actor_model=self.env_actor_model[idx].copy(), n_envs=len(envs))


def homogeneous(name: str, model: Model, n_envs: int, params: Optional[Params] = None, dt=1.0 / 60.0,
                substeps=2) -> Workload:
    return Workload(name=name, models=[model], env_actor_model=np.zeros(n_envs, dtype=np.int32), actors_per_env=1,
                    n_envs=n_envs, params=params or Params(), dt=dt, substeps=substeps)


def hand_tendon_workload(n_envs=64) -> Workload:
    """The hand with coupled middle / distal flexions (four equality tendons) holding a free cube."""
    return Workload(name="hand_tendon", models=[hand(coupled=True), cube()],
                    env_actor_model=np.tile(np.array([0, 1], np.int32), n_envs), actors_per_env=2, n_envs=n_envs,
                    params=Params())


def hand_workload(n_envs=64) -> Workload:
    """Fixed-base 24-DOF hand holding a free cube (two actors per env: box-capsule contacts)."""
    return Workload(name="hand", models=[hand(), cube()],
                    env_actor_model=np.tile(np.array([0, 1], np.int32), n_envs), actors_per_env=2,
                    n_envs=n_envs, params=Params())


def mixed_workload(n_envs=16384, fractions=(0.4, 0.3, 0.3)) -> Workload:
    """Heterogeneous batch: Ant-like, Humanoid-like and hand-with-cube envs in the given
    proportions (contiguous blocks, in that order). Envs with one actor pad the second slot
    with -1."""
    n_ant = int(round(fractions[0] * n_envs))
    n_hum = int(round(fractions[1] * n_envs))
    n_hand = n_envs - n_ant - n_hum
    eam = np.concatenate([np.tile([0, -1], n_ant), np.tile([1, -1], n_hum), np.tile([2, 3], n_hand)]).astype(np.int32)
    return Workload(name="mixed", models=[ant(), humanoid(), hand(), cube()], env_actor_model=eam,
                    actors_per_env=2, n_envs=n_envs, params=Params())


def cartpole_workload(n_envs=64) -> Workload:
    """Plain step, smallest case: 64 cartpoles, no contacts, dt 1/60 s, 2 substeps."""
    return homogeneous("cartpole", cartpole(), n_envs)


def ant_workload(n_envs=4096) -> Workload:
    """Ant-like locomotion: 4096 envs, dt 1/60 s, 2 substeps, 4 position + 1 velocity iterations."""
    return homogeneous("ant", ant(), n_envs)


def humanoid_workload(n_envs=4096) -> Workload:
    """Humanoid-like locomotion: 4096 envs, dt 1/60 s, 2 substeps, 4/1 iterations."""
    return homogeneous("humanoid", humanoid(), n_envs)


# ------------------------------------------------------------------------------------------------
# Seeded inputs. One numpy Generator(PCG64(seed)) per workload; draw order: initial DOF noise
# (env-major, DOF-minor), then actions (step-major, env, DOF).
def initial_state(w: Workload, rng: np.random.Generator):
    """Root states (N_A, 13) and DOF states (N_D, 2), float32. Roots start at their model's nominal
    position with identity orientation and zero velocity; joint positions are uniform in
    +-dof_noise, clipped into the joint limits; joint velocities are zero."""
    root = np.zeros((w.n_actors, 13), dtype=np.float32)
    dofs = []
    row = 0
    for e in range(w.n_envs):
        for m in w.actor_models(e):
            r = root[row]
            r[0:3] = m.root_pos
            r[6] = 1.0
            row += 1
    for e in range(w.n_envs):
        for m in w.actor_models(e):
            nj = m.n_jdof
            q = rng.uniform(-m.dof_noise, m.dof_noise, size=nj) if nj else np.zeros(0)
            for j, li in enumerate(m.dof_links()):
                if m.has_limit[li]:  # 1-DOF joints only
                    q[j] = min(max(q[j], m.lo[li]), m.hi[li])
            d = np.zeros((nj, 2))
            d[:, 0] = q
            dofs.append(d)
    dof = np.concatenate(dofs).astype(np.float32) if dofs else np.zeros((0, 2), np.float32)
    return root, dof


def env_gear(w: Workload) -> np.ndarray:
    """Per joint DOF action scale (N_D,), float32."""
    g = [np.concatenate([m.gear for m in w.actor_models(e)]) for e in range(w.n_envs)]
    return np.concatenate(g).astype(np.float32) if g else np.zeros(0, np.float32)


def actions(w: Workload, rng: np.random.Generator, n_steps: int) -> np.ndarray:
    """DOF actuation forces (n_steps, N_D) float32: uniform [-1, 1] times the DOF's gear."""
    g = env_gear(w)
    a = rng.uniform(-1.0, 1.0, size=(n_steps, g.shape[0]))
    return (a * g[None, :]).astype(np.float32)


def seeded_inputs(w: Workload, seed: int, n_steps: int):
    """(root, dof, actions) for a workload, from numpy Generator(PCG64(seed))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    root, dof = initial_state(w, rng)
    act = actions(w, rng, n_steps)
    return root, dof, act
