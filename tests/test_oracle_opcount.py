"""Pins of the oracle's operation-counting scalar, which supplies the flops of the roofline.

The counter is defined to count every floating-point add, subtract, multiply, divide, square root,
sine, cosine and arctangent the oracle executes (accumulations included: a dot product of length
n that starts from zero is n multiplies and n adds), and nothing else (negations, absolute values
and comparisons are free). Each expected count below is derived by hand from the definition of
the routine, not read off the code:
  * dot of 3-vectors: 3 mul + 2 add = 5; cross product: 6 mul + 3 sub = 9;
  * 3x3 matrix times vector: 3 rows x (3 mul + 2 add) = 15; 3x3 product: 9 entries x 5 = 45;
  * quaternion product: 16 mul + 12 add/sub = 28;
  * quaternion exponential of a rotation vector th: |th|^2 (5), its root (1), the half angle (1,
    used twice: 2), sine and cosine (2), sin / |th| (1), three scalings (3): 14;
  * 6x6 matrix times spatial vector, accumulated from zero: 6 x (6 mul + 6 add) = 72; 6x6 product
    36 x 12 = 432; spatial dot product 12;
  * Cholesky factor of an n x n SPD matrix: column j costs j multiply-subtract pairs and a square
    root for the pivot, and j pairs and a division for each of the n - 1 - j entries below it,
    (2j + 1)(n - j) in all, sum over j = n(n + 1)(2n + 1) / 6; the forward and back substitutions
    cost 2i + 1 per row, 2 n^2 together.
On the whole step, the projected Gauss-Seidel solve's cost per iteration is pinned by differences
of the step count between solver settings (everything before and after the solve is identical):
one more position iteration of a contact-free body adds the delta-buffer update (n multiply-adds,
2n), and one more velocity iteration adds nothing; with one active limit row on a one-DOF pendulum
moving away from its limit (separation positive throughout, so the speculative target -sep/h_it
costs 2 operations), a position iteration costs the row (separation d + J dq: 2n + 1; target: 2;
J v: 2n; (target - J v) / A added to the impulse: 3; impulse change and v += W dl: 1 + 2n; 6n + 7)
plus the delta-buffer update (2n), and a velocity iteration 6n + 7 (target -sep/h: 2).
A skipped operation type, a helper counted twice or a solver loop miscounted fails one of these."""
import numpy as np
import pytest

import oracle
from paper_2108_10470_gb300 import workloads as W

SINGLE = {0: "add", 1: "sub", 2: "mul", 3: "div", 4: "sqrt", 5: "sin", 6: "cos", 7: "atan2"}
FREE = {8: "negation", 9: "fabs", 10: "comparison"}
HELPERS = {20: 5, 21: 9, 22: 15, 23: 45, 24: 28, 25: 14, 26: 72, 27: 432, 28: 12}


@pytest.mark.parametrize("which", sorted(SINGLE))
def test_each_operation_type_counts_once(which):
    assert oracle.opcount_probe(which) == 1, SINGLE[which]


@pytest.mark.parametrize("which", sorted(FREE))
def test_sign_flips_and_comparisons_are_free(which):
    assert oracle.opcount_probe(which) == 0, FREE[which]


@pytest.mark.parametrize("which,expected", sorted(HELPERS.items()))
def test_helper_counts_match_their_definitions(which, expected):
    assert oracle.opcount_probe(which) == expected


@pytest.mark.parametrize("n", [1, 2, 3, 6, 14, 27])
def test_cholesky_counts_match_closed_forms(n):
    assert oracle.opcount_probe(29, n) == n * (n + 1) * (2 * n + 1) // 6
    assert oracle.opcount_probe(30, n) == 2 * n * n


def step_count(model, root, dof, act, pos_iters, vel_iters, gravity):
    p = W.Params(gravity=gravity, pos_iters=pos_iters, vel_iters=vel_iters)
    w = W.homogeneous("probe", model, 1, params=p, substeps=1)
    O = oracle.Oracle(w)
    r, d = root.astype(np.float64).copy(), dof.astype(np.float64).copy()
    return O.step_flops(r, d, act)


def test_solver_iteration_cost_without_rows():
    """A free sphere far above the ground (no contacts, n = 6 generalized velocities)."""
    m = W.free_sphere(z=3.0)
    root = np.array([[0, 0, 3.0, 0, 0, 0, 1, 0.1, -0.2, 0.3, 0.5, 0.2, -0.1]])
    dof, act = np.zeros((0, 2)), np.zeros(0)
    c = {(p, v): step_count(m, root, dof, act, p, v, (0, 0, -9.81)) for p, v in ((4, 1), (5, 1), (4, 2))}
    n = 6
    assert c[(5, 1)] - c[(4, 1)] == 2 * n
    assert c[(4, 2)] - c[(4, 1)] == 0


def limited_pendulum():
    b = W._Builder("limited_pendulum")
    b.link(-1, W.JOINT_FIXED, mass=1.0, inertia=(1, 1, 1, 0, 0, 0))
    b.link(0, W.JOINT_REVOLUTE, axis=(0, 1, 0), mass=0.5, com=(0, 0, -0.5), inertia=(0.04, 0.04, 1e-6, 0, 0, 0),
           limit=(-0.5, 0.5))
    return b.build()


def test_solver_iteration_cost_of_one_limit_row():
    """The pendulum 0.05 rad inside its lower limit's margin, moving away from it at 1 rad/s in
    zero gravity: one active limit row whose impulse stays zero."""
    m = limited_pendulum()
    root = np.array([[0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0]], np.float64)
    dof = np.array([[-0.45, 1.0]])
    act = np.zeros(1)
    c = {(p, v): step_count(m, root, dof, act, p, v, (0, 0, 0)) for p, v in ((4, 1), (5, 1), (4, 2))}
    n = 1
    assert c[(5, 1)] - c[(4, 1)] == (6 * n + 7) + 2 * n
    assert c[(4, 2)] - c[(4, 1)] == 6 * n + 7


def test_step_count_is_additive_over_envs():
    """Envs are independent: a batch's count is the sum of its envs' counts."""
    w = W.ant_workload(6)
    root, dof, acts = W.seeded_inputs(w, 2, 1)
    whole = oracle.Oracle(w).step_flops(root.astype(np.float64), dof.astype(np.float64), acts[0])
    parts = 0.0
    for e in range(w.n_envs):
        ws = w.subset([e])
        parts += oracle.Oracle(ws).step_flops(root[e:e + 1].astype(np.float64), dof[8 * e:8 * e + 8].astype(np.float64),
                                              acts[0][8 * e:8 * e + 8])
    assert whole == parts > 0
