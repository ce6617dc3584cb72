"""Merging (Sec. 3.5): with identical residual magnitudes as input, the GPU's
new partition equals the oracle's bit for bit (ties broken by edge id)."""
import numpy as np
import pytest
import torch

import oracle as O
from synth import generators as G, make_workload

from gpu_util import dev, integrator

pytestmark = pytest.mark.gpu


def _chi_field(H, W, seed, ties=True):
    rng = np.random.default_rng(seed)
    chi = np.abs(rng.normal(0, 1e-3, (H, W, 2))).astype(np.float32)
    if ties:
        chi.reshape(-1)[::5] = chi.reshape(-1)[0]
    return chi


@pytest.mark.parametrize("name", ["c3_small", "c2"])
def test_merge_bit_exact_two_rounds(name):
    w = make_workload(name)
    H, W = w.mask.shape
    p = dict(w.params, theta_c_deg=2.0)
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, p)
    lab, K = it.seed_components(n, m)
    it.solve_components()
    cam = O.Camera.from_dict(w.camera)
    geo = O.geometry(w.normals, w.mask, cam)
    ref_lab, Kr = O.seed_components(w.normals, w.mask, 2.0)
    for rnd in range(2):
        chi = _chi_field(H, W, 10 + rnd)
        e = O.inter_edges(geo, ref_lab)
        chi_e = chi.reshape(-1)[2 * geo.a[e] + geo.d[e]]
        ref_lab, Kr, _ = O.merge_labels(ref_lab, Kr, geo, e, chi_e)
        lab, K = it.merge_residuals(torch.from_numpy(chi).cuda())
        print(name, "round", rnd, "K", K, Kr)
        assert K == Kr
        np.testing.assert_array_equal(lab.cpu().numpy().reshape(-1), ref_lab)


def test_merge_leaves_logdepth_unchanged():
    w = make_workload("c3_small")
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, w.params)
    it.seed_components(n, m)
    it.solve_components()
    it.solve_scales(3)
    z0 = it.logdepth().cpu().numpy()
    lab, K = it.merge()
    z1 = it.logdepth().cpu().numpy()
    assert np.max(np.abs(z0 - z1)) < 1e-5
