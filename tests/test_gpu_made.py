"""ni_min_made (the minimum theoretical MADE of a decomposition, supplementary
material, the section on the components found for different theta_c) against
the oracle's min_made on the same inputs."""
import time

import numpy as np
import pytest
import torch

import oracle as O
from synth import make_workload

from gpu_util import dev, integrator
from paper_2510_11508_gb300 import ni

pytestmark = pytest.mark.gpu


def _close(gpu, ref, scale):
    """FP64 on both sides; only the order of the sums differs."""
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    assert np.array_equal(np.isnan(gpu), np.isnan(ref))
    ok = ~np.isnan(ref)
    np.testing.assert_allclose(gpu[ok], ref[ok], rtol=1e-10, atol=1e-13 * scale)


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _depth(z, camera):
    z = np.asarray(z, np.float64)
    return np.exp(z) if camera == O.PERSP else z


@pytest.mark.parametrize("name", ["c1", "c2", "c3_small"])
def test_min_made_of_the_fill_matches_oracle(name):
    """The decomposition and fill of the GPU path, scored by both sides."""
    w = make_workload(name)
    H, W = w.mask.shape
    cam = w.camera["camera"]
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, w.params)
    labels, K = it.seed_components(n, m)
    z = it.solve_components()
    gt = _t(w.depth_gt)
    made, per, scale = it.min_made(z, gt, labels, K, z_is_log=True, per_component=True)
    zc, lc = z.cpu().numpy(), labels.cpu().numpy()
    g32 = gt.cpu().numpy()
    ref, ref_per, ref_scale = O.min_made(_depth(zc, cam), g32, lc, K, cam)
    gscale = float(np.nanmean(np.abs(g32)))
    print(name, "K", K, "min MADE", made, "oracle", ref)
    _close([made], [ref], gscale)
    _close(per.cpu().numpy(), ref_per, gscale)
    # the scales may differ where a component's error is flat; both must reach the minimum
    s = scale.cpu().numpy()
    d = _depth(zc, cam).reshape(-1)
    g = g32.reshape(-1).astype(np.float64)
    ok = (lc.reshape(-1) >= 0) & np.isfinite(d) & np.isfinite(g)
    for c in range(0, K, max(1, K // 25)):
        sel = ok & (lc.reshape(-1) == c)
        if not sel.any():
            continue
        e = np.abs(s[c] * d[sel] - g[sel]) if cam == O.PERSP else np.abs(d[sel] + s[c] - g[sel])
        assert e.mean() == pytest.approx(ref_per[c], rel=1e-10, abs=1e-13 * gscale)


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_global_made_of_the_output_matches_oracle(name):
    """labels = None: the reconstruction's MADE after the best global scale."""
    w = make_workload(name)
    H, W = w.mask.shape
    cam = w.camera["camera"]
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, w.params)
    depth, labels, st = it.integrate(n, m)
    gt = _t(w.depth_gt)
    made = it.min_made(depth, gt, None, z_is_log=False)
    ref, _, _ = O.min_made(depth.cpu().numpy(), gt.cpu().numpy(), None, 1, cam)
    fine = it.min_made(depth, gt, labels, st["K_final"], z_is_log=False)
    ref_fine, _, _ = O.min_made(depth.cpu().numpy(), gt.cpu().numpy(), labels.cpu().numpy(), st["K_final"], cam)
    print(name, "MADE", made, "oracle", ref, "per final component", fine, ref_fine)
    _close([made, fine], [ref, ref_fine], float(np.nanmean(np.abs(w.depth_gt))))
    assert fine <= made * (1 + 1e-12)


@pytest.mark.parametrize("camera", [O.PERSP, O.ORTHO])
@pytest.mark.parametrize("shape", [(1, 2), (37, 53), (130, 257)])
def test_min_made_ragged_excluded_and_empty(camera, shape):
    """Odd sizes, NaN and non-positive depths, excluded labels, empty
    components, ties and repeated values."""
    H, W = shape
    rng = np.random.default_rng(H * 1000 + W + camera)
    used = max(1, (H * W) // 40)
    K = min(H * W, used + 3)                                   # components past `used` stay empty
    lab = rng.integers(-1, used, (H, W)).astype(np.int32)
    g = rng.uniform(0.5, 4.0, (H, W)).astype(np.float32)
    z = rng.normal(scale=0.3, size=(H, W)).astype(np.float32)
    if H * W > 2:
        z.reshape(-1)[:: 17] = np.nan
        g.reshape(-1)[3:: 29] = -1.0 if camera == O.PERSP else np.inf
        z.reshape(-1)[5:: 31] = z.reshape(-1)[5]                  # repeated values
        g.reshape(-1)[5:: 31] = g.reshape(-1)[5]
    cam = {"camera": camera, "fx": 100.0, "fy": 100.0, "cx": W / 2, "cy": H / 2}
    it = integrator(H, W, cam, {"theta_c_deg": 3.5})
    for z_is_log in (True, False):
        zz = z if z_is_log or camera == O.ORTHO else np.exp(z).astype(np.float32)
        made, per, scale = it.min_made(_t(zz), _t(g), _t(lab, torch.int32), K, z_is_log=z_is_log,
                                       per_component=True)
        d = _depth(zz, camera) if z_is_log else np.asarray(zz, np.float64)
        ref, ref_per, ref_scale = O.min_made(d, g, lab, K, camera)
        _close([made], [ref], 1.0)
        _close(per.cpu().numpy(), ref_per, 1.0)
        assert np.array_equal(np.isnan(scale.cpu().numpy()), np.isnan(ref_scale))


def test_min_made_closed_form_and_errors():
    cam = {"camera": 1, "fx": 10.0, "fy": 10.0, "cx": 1.0, "cy": 0.5}
    it = integrator(1, 2, cam, {"theta_c_deg": 3.5})
    d, g = _t(np.array([[1.0, 1.0]])), _t(np.array([[1.0, 3.0]]))
    assert it.min_made(d, g, None, z_is_log=False) == 1.0        # any scale in [1, 3]: E = 2 over 2 pixels
    d, g = _t(np.array([[1.0, 3.0]])), _t(np.array([[2.0, 3.0]]))
    assert it.min_made(d, g, None, z_is_log=False) == 0.5        # weighted median of (2, 1) with weights (1, 3)
    assert np.isnan(it.min_made(_t(np.full((1, 2), np.nan)), g, None, z_is_log=False))
    with pytest.raises(ni.NIError) as ei:                         # label >= K: rejected by the kernel's check
        it.min_made(d, g, _t(np.array([[0, 2]]), torch.int32), 2, z_is_log=False)
    assert ei.value.status == 1
    with pytest.raises(ni.NIError):
        it.min_made(d, g, _t(np.array([[0, 0]]), torch.int32), 0, z_is_log=False)
    # the handle stays usable after the rejected calls
    assert it.min_made(d, g, _t(np.array([[0, 1]]), torch.int32), 2, z_is_log=False) == 0.0


def test_min_made_full_size_c3():
    """2048 x 2048 (2.7e6 counted pixels): the decomposition of the seeding and
    fill, timed (CUDA events) and compared with the oracle."""
    w = make_workload("c3")
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, w.params)
    labels, K = it.seed_components(n, m)
    z = it.solve_components()
    gt = _t(w.depth_gt)
    it.min_made(z, gt, labels, K)                                 # allocates the scratch
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    wall = time.perf_counter()
    t0.record()
    made, per, _ = it.min_made(z, gt, labels, K, per_component=True)
    t1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall
    ref, ref_per, _ = O.min_made(np.exp(z.cpu().numpy().astype(np.float64)), gt.cpu().numpy(),
                                 labels.cpu().numpy(), K, O.PERSP)
    print(f"C3 K={K} min MADE {made:.6e} (oracle {ref:.6e}); {t0.elapsed_time(t1):.2f} ms on the GPU, "
          f"{1e3 * wall:.2f} ms wall")
    gscale = float(np.nanmean(np.abs(w.depth_gt)))
    _close([made], [ref], gscale)
    _close(per.cpu().numpy(), ref_per, gscale)
