"""8-connectivity past the seeding (fill, relative-scale loop, merging, end to
end) against the 8-connected oracle (the setting of the paper's DiLiGenT
experiments and of its connectivity ablation)."""
import numpy as np
import pytest
import torch

import oracle as O
from synth import make_workload

from gpu_util import PIXEL_TOL, dev, integrator

pytestmark = pytest.mark.gpu


def _p(w, **over):
    return dict(w.params, connectivity=8, **over)


def _max(z, zr, mask, camera):
    """Largest per-pixel error after the island alignment of _rel (8-connected islands)."""
    isl, n = O.islands(mask, 8)
    m = isl >= 0
    worst = 0.0
    if camera == O.PERSP:
        z, zr = np.exp(np.where(m, z, 0.0)), np.exp(np.where(m, zr, 0.0))
    for i in range(n):
        s = isl == i
        if camera == O.PERSP:
            al = z[s] * (np.sum(z[s] * zr[s]) / np.sum(z[s] * z[s]))
            worst = max(worst, float(np.max(np.abs(al - zr[s]) / zr[s])))
        else:
            al = z[s] + np.mean(zr[s] - z[s])
            worst = max(worst, float(np.max(np.abs(al - zr[s]))))
    if camera != O.PERSP and m.any():
        worst /= max(float(np.ptp(zr[m])), 1e-300)
    return worst


def _rel(z, zr, mask, camera):
    m = mask > 0
    if camera == O.PERSP:
        return O.aligned_rel_rmse(np.where(m, np.exp(z), np.nan), np.where(m, np.exp(zr), np.nan), mask, O.PERSP, 8)
    return O.aligned_rel_rmse(np.where(m, z, np.nan), np.where(m, zr, np.nan), mask, O.ORTHO, 8)


@pytest.mark.parametrize("name", ["c1", "c2", "c3_small"])
@pytest.mark.parametrize("irls", [1, 2])
def test_fill_8_matches_oracle(name, irls):
    w = make_workload(name)
    H, W = w.mask.shape
    p = _p(w, n_fill_irls=irls)
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, p, batched=0)
    lab, K = it.seed_components(n, m)
    z = it.solve_components().cpu().numpy()
    geo = O.geometry(w.normals, w.mask, O.Camera.from_dict(w.camera), 8)
    ref_lab, Kr = O.seed_components(w.normals, w.mask, p["theta_c_deg"], 8)
    assert K == Kr
    zr, _ = O.fill_components(geo, ref_lab, Kr, p.get("k", 2.0), irls)
    d = (z - np.nan_to_num(zr).reshape(H, W))[w.mask > 0]
    scale = 1.0 if w.camera["camera"] == 1 else float(np.ptp(w.depth_gt[w.mask > 0]))
    rms = float(np.sqrt(np.mean(d * d))) / scale
    print(name, "irls", irls, "K", K, "fill rms", rms, "max", float(np.abs(d).max()) / scale)
    assert rms <= 1e-4
    assert float(np.abs(d).max()) / scale <= PIXEL_TOL


@pytest.mark.parametrize("name,T", [("c1", 6), ("c2", 8), ("c3_small", 8)])
def test_scale_loop_8_matches_oracle(name, T):
    w = make_workload(name)
    p = _p(w, T=T, dE_max=0.0, can_merge=False)
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, p, batched=0)
    it.seed_components(n, m)
    it.solve_components()
    k, E, z = it.solve_scales(T)
    assert k == T
    ref = O.integrate(w.normals, w.mask, w.camera, O.Params.from_dict(p))
    err = _rel(z.cpu().numpy(), np.nan_to_num(ref["z"]), w.mask, w.camera["camera"])
    mx = _max(z.cpu().numpy(), np.nan_to_num(ref["z"]), w.mask, w.camera["camera"])
    print(name, "rel depth err", err, "max", mx)
    assert err <= 1e-4
    assert mx <= PIXEL_TOL
    np.testing.assert_allclose(E, ref["energies"], rtol=5e-3, atol=1e-9 * max(ref["energies"]))


@pytest.mark.parametrize("name", ["c3_small", "c2"])
def test_merge_8_bit_exact_two_rounds(name):
    w = make_workload(name)
    H, W = w.mask.shape
    p = _p(w, theta_c_deg=2.0)
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, p, batched=0)
    it.seed_components(n, m)
    it.solve_components()
    geo = O.geometry(w.normals, w.mask, O.Camera.from_dict(w.camera), 8)
    ref_lab, Kr = O.seed_components(w.normals, w.mask, 2.0, 8)
    for rnd in range(2):
        rng = np.random.default_rng(20 + rnd)
        chi = np.abs(rng.normal(0, 1e-3, (H, W, 4))).astype(np.float32)
        chi.reshape(-1)[::5] = chi.reshape(-1)[0]          # ties, broken by the edge id 4 a + dir
        e = O.inter_edges(geo, ref_lab)
        chi_e = chi.reshape(-1)[4 * geo.a[e] + geo.d[e]]
        ref_lab, Kr, _ = O.merge_labels(ref_lab, Kr, geo, e, chi_e)
        lab, K = it.merge_residuals(torch.from_numpy(chi).cuda())
        assert K == Kr
        np.testing.assert_array_equal(lab.cpu().numpy().reshape(-1), ref_lab)


@pytest.mark.parametrize("name", ["c1", "c2", "c3_small"])
def test_integrate_8_matches_oracle(name):
    w = make_workload(name)
    H, W = w.mask.shape
    p = _p(w)
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, p, batched=0)
    depth, labels, st = it.integrate(n, m)
    ref = O.integrate(w.normals, w.mask, w.camera, O.Params.from_dict(p))
    zg = np.log(depth.cpu().numpy()) if w.camera["camera"] == 1 else depth.cpu().numpy()
    err = _rel(np.nan_to_num(zg), np.nan_to_num(ref["z"]), w.mask, w.camera["camera"])
    mx = _max(np.nan_to_num(zg), np.nan_to_num(ref["z"]), w.mask, w.camera["camera"])
    print(name, "max", mx, "K0", st["K0"], ref["K0"], "K", st["K_final"], ref["K"], "iters", st["scale_iters"], ref["iters"],
          "err", err)
    assert st["K0"] == ref["K0"]
    assert st["K_final"] == ref["K"] and st["scale_iters"] == ref["iters"]
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
    assert err <= 1e-4
    assert mx <= PIXEL_TOL
