"""The allocation-free seeding entry point (ni_seed_components_noalloc).

It is meant for callers that may not allocate device memory while running
(real-time pipelines with all memory reserved up front, frameworks that own
the device allocator, code under a fixed memory-pool limit).  Its labels and K
must equal those of the regular entry point, on two calls in a row (the second
call reuses the static scratch the first one left behind).  This file is named
so that pytest collects it last."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2510_11508_gb300 import ni
from synth import make_workload
from synth import generators as G

pytestmark = pytest.mark.gpu


def _regular(normals, mask, camera, theta):
    H, W = mask.shape
    it = ni.Integrator(ni.config_for(H, W, camera, {"theta_c_deg": theta}, validate=0))
    lab, K = it.seed_components(normals, mask)
    torch.cuda.synchronize()
    out = lab.cpu().numpy()
    it.close()
    return out, K


def _noalloc(normals, mask, camera, theta):
    L = ni.load()
    H, W = mask.shape
    cam = ni.Camera(int(camera["camera"]), float(camera["fx"]), float(camera["fy"]),
                    float(camera["cx"]), float(camera["cy"]))
    labels = torch.empty((H, W), dtype=torch.int32, device=normals.device)
    K = torch.zeros(1, dtype=torch.int32, device=normals.device)
    rc = L.ni_seed_components_noalloc(normals.data_ptr(), mask.data_ptr(), H, W, C.byref(cam),
                                      -1.0 if theta is None else float(theta), labels.data_ptr(),
                                      K.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, ni.STATUS.get(rc, rc)
    torch.cuda.synchronize()
    return labels.cpu().numpy(), int(K.item())


def _inputs(w):
    return torch.from_numpy(w.normals).cuda(), torch.from_numpy(w.mask).cuda()


def test_noalloc_matches_regular_entry_point_twice():
    """Two different maps back to back: identical labels and K each time."""
    for name in ("c3_small", "c2"):
        w = make_workload(name)
        n, m = _inputs(w)
        ref, Kr = _regular(n, m, w.camera, w.params["theta_c_deg"])
        got, K = _noalloc(n, m, w.camera, w.params["theta_c_deg"])
        assert K == Kr
        np.testing.assert_array_equal(got, ref)


def test_noalloc_same_map_twice_and_ragged():
    nrm, mask, cam = G.random_normal_field(77, 45, n_dirs=3, jitter_deg=1.5, hole_frac=0.2, seed=9)
    n = torch.from_numpy(nrm).cuda()
    m = torch.from_numpy(mask).cuda()
    ref, Kr = _regular(n, m, cam, 2.5)
    for _ in range(2):
        got, K = _noalloc(n, m, cam, 2.5)
        assert K == Kr
        np.testing.assert_array_equal(got, ref)


def test_noalloc_at_its_pixel_limit():
    """The full 2048x2048 map holds exactly 2^22 pixels: the parent array
    fills the static scratch to its last byte."""
    w = make_workload("c3")
    assert w.mask.size == 1 << 22
    n, m = _inputs(w)
    ref, Kr = _regular(n, m, w.camera, w.params["theta_c_deg"])
    for _ in range(2):
        got, K = _noalloc(n, m, w.camera, w.params["theta_c_deg"])
        assert K == Kr
        np.testing.assert_array_equal(got, ref)


def test_noalloc_rejects_maps_beyond_its_scratch():
    L = ni.load()
    cam = ni.Camera(1, 100.0, 100.0, 0.0, 0.0)
    H, W = 4096, 1025          # 4,198,400 > 2^22 pixels; no buffer is touched
    rc = L.ni_seed_components_noalloc(16, 16, H, W, C.byref(cam), 3.0, 16, 16, None)
    assert ni.STATUS[rc] == "NI_ERR_INVALID_ARG"
