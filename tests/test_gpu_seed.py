"""Seeding (Sec. 3.3): GPU labels and K must equal the oracle's bit for bit."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from synth import generators as G, make_workload

from gpu_util import dev, integrator

pytestmark = pytest.mark.gpu


def _check(normals, mask, camera, theta):
    H, W = mask.shape
    n, m = dev(normals, mask)
    it = integrator(H, W, camera, {"theta_c_deg": theta}, validate=0)
    lab, K = it.seed_components(n, m)
    ref, Kr = O.seed_components(normals, mask, theta)
    assert K == Kr
    np.testing.assert_array_equal(lab.cpu().numpy().reshape(-1), ref)
    return K


@pytest.mark.parametrize("name", ["c1", "c2", "c3_small", "c5_small"])
def test_labels_bit_exact_on_workloads(name):
    w = make_workload(name)
    K = _check(w.normals, w.mask, w.camera, w.params["theta_c_deg"])
    print(name, "K0 =", K)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (37, 1), (33, 47), (16, 32), (17, 33), (100, 131)])
@pytest.mark.parametrize("theta", [None, 2.0, 3.5, 179.0])
def test_labels_bit_exact_random_fields(H, W, theta):
    nrm, mask, cam = G.random_normal_field(H, W, n_dirs=3, jitter_deg=1.5, hole_frac=0.15,
                                           seed=H * 1000 + W)
    _check(nrm, mask, cam, theta)


def test_empty_mask():
    nrm, mask, cam = G.random_normal_field(20, 20, seed=1)
    mask[:] = 0
    assert _check(nrm, mask, cam, 3.0) == 0


def test_threshold_ties_at_one_ulp():
    """Dots exactly one float32 ulp above / at / below cos(theta_c)."""
    theta = 3.5
    c = math.cos(theta * (math.pi / 180.0))
    cz = np.float32(c)
    zs = [np.nextafter(cz, np.float32(2)), cz, np.nextafter(cz, np.float32(0))]
    H, W = 24, 40
    rng = np.random.default_rng(0)
    nrm = np.zeros((H, W, 4), np.float32)
    nrm[..., 2] = 1.0
    # alternate columns tilted so that horizontal dots equal the chosen z exactly
    for j in range(1, W, 2):
        z = zs[rng.integers(3)]
        nrm[:, j, 0] = np.float32(math.sqrt(1 - float(z) ** 2))
        nrm[:, j, 2] = z
    mask = np.ones((H, W), np.uint8)
    cam = {"camera": 0, "fx": 1.0, "fy": 1.0, "cx": 0.0, "cy": 0.0}
    _check(nrm, mask, cam, theta)


def test_full_size_c3_labels():
    w = make_workload("c3")
    K = _check(w.normals, w.mask, w.camera, w.params["theta_c_deg"])
    print("c3 K0 =", K)
