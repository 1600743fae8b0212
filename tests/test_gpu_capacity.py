"""GPU parity at the kernel's capacity limits and across lane widths: random articulated trees (mixed
revolute / prismatic joints, random frames, axes and inertias) with 32 links and 31 joint DOFs on
a fixed base, 27 links and 32 generalized DOFs on a floating base, and a batch mixing tree sizes
that map to 8, 16 and 32 lanes per env."""
import numpy as np
import pytest

from paper_2108_10470_gb300 import workloads as W
from test_gpu_parity import check_rollout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10470_gb300 import build
    build.build_library()
    torch.cuda.set_device(0)


def tree(seed, n_links, floating):
    m = W.random_tree(np.random.default_rng(seed), n_links, floating, allow_fixed=False)
    m.armature = np.full(m.n_links, 0.05)  # keep the joint-space inertia well conditioned
    return m


@pytest.mark.parametrize("n_links,floating", [(32, False), (27, True)])
@pytest.mark.parametrize("steps,rtol,atol", [(1, 1e-4, 1e-5), (16, 1e-3, 1e-3)])
def test_largest_trees(n_links, floating, steps, rtol, atol):
    m = tree(11, n_links, floating)
    assert m.n_links <= 32 and m.n_gen <= 32 and (m.n_gen == 32 or m.n_links == 32)
    w = W.homogeneous("tree", m, 37)
    check_rollout(w, steps, rtol, atol, min_same=1.0)


def test_mixed_lane_widths():
    models = [tree(1, 5, False), tree(2, 12, False), tree(3, 24, True)]  # 8, 16 and 32 lanes
    eam = np.array([i % 3 for i in range(60)], np.int32)
    w = W.Workload("trees", models, eam, 1, 60, W.Params())
    check_rollout(w, 4, 1e-3, 1e-3, min_same=1.0)
