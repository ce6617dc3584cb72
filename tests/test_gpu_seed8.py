"""Seeding with 8-connectivity (the pixel graph of the paper's DiLiGenT
experiments and of its connectivity ablation): GPU labels and K equal the
oracle's bit for bit."""
import math

import numpy as np
import pytest

import oracle as O
from synth import generators as G, make_workload

from gpu_util import dev, integrator
from paper_2510_11508_gb300 import ni

pytestmark = pytest.mark.gpu


def _check(normals, mask, camera, theta):
    H, W = mask.shape
    n, m = dev(normals, mask)
    it = integrator(H, W, camera, {"theta_c_deg": theta}, validate=0, connectivity=8, batched=0)
    lab, K = it.seed_components(n, m)
    ref, Kr = O.seed_components(normals, mask, theta, 8)
    assert K == Kr
    np.testing.assert_array_equal(lab.cpu().numpy().reshape(-1), ref)
    return K


@pytest.mark.parametrize("name", ["c1", "c2", "c3_small"])
def test_labels_8_bit_exact_on_workloads(name):
    w = make_workload(name)
    K = _check(w.normals, w.mask, w.camera, w.params["theta_c_deg"])
    _, K4 = O.seed_components(w.normals, w.mask, w.params["theta_c_deg"], 4)
    print(name, "K0 8-connected", K, "4-connected", K4)
    assert K <= K4


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (37, 1), (2, 2), (33, 47), (16, 32), (17, 33), (100, 131)])
@pytest.mark.parametrize("theta", [None, 2.0, 3.5, 179.0])
def test_labels_8_bit_exact_random_fields(H, W, theta):
    nrm, mask, cam = G.random_normal_field(H, W, n_dirs=3, jitter_deg=1.5, hole_frac=0.3,
                                           seed=H * 1000 + W + 7)
    _check(nrm, mask, cam, theta)


def test_checkerboard_joins_through_diagonals_only():
    """Valid pixels on one colour of a checkerboard have no 4-neighbours: every
    component comes from diagonal edges (tile borders included)."""
    H, W = 70, 97
    nrm, _, cam = G.random_normal_field(H, W, n_dirs=2, jitter_deg=0.5, hole_frac=0.0, seed=3, block=9)
    v, u = np.mgrid[0:H, 0:W]
    mask = ((u + v) % 2 == 0).astype(np.uint8)
    K = _check(nrm, mask, cam, 5.0)
    _, K4 = O.seed_components(nrm, mask, 5.0, 4)
    assert K4 == int(mask.sum()) and K < K4 // 10


def test_diagonal_threshold_ties_at_one_ulp():
    """Diagonal dots one float32 ulp above / at / below cos(theta_c); the axis
    neighbours are masked out, so only diagonal edges decide."""
    theta = 3.5
    c = math.cos(theta * (math.pi / 180.0))
    cz = np.float32(c)
    zs = [np.nextafter(cz, np.float32(2)), cz, np.nextafter(cz, np.float32(0))]
    H, W = 24, 40
    rng = np.random.default_rng(1)
    nrm = np.zeros((H, W, 4), np.float32)
    nrm[..., 2] = 1.0
    v, u = np.mgrid[0:H, 0:W]
    mask = ((u + v) % 2 == 0).astype(np.uint8)
    for j in range(1, W, 2):             # odd columns tilted: every diagonal dot equals the chosen z
        z = zs[rng.integers(3)]
        nrm[:, j, 0] = np.float32(math.sqrt(1 - float(z) ** 2))
        nrm[:, j, 2] = z
    cam = {"camera": 0, "fx": 1.0, "fy": 1.0, "cx": 0.0, "cy": 0.0}
    _check(nrm, mask, cam, theta)


def test_full_size_c3_labels_8():
    w = make_workload("c3")
    K = _check(w.normals, w.mask, w.camera, w.params["theta_c_deg"])
    print("c3 K0 8-connected =", K)
