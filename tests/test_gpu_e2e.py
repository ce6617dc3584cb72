"""Algorithm 1 end to end through ni_integrate against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from synth import make_workload

from gpu_util import PIXEL_TOL, dev, integrator, rel_depth_error, rel_depth_max

pytestmark = pytest.mark.gpu


def _run(name, **over):
    w = make_workload(name)
    p = dict(w.params, **over)
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, p)
    depth, labels, st = it.integrate(n, m)
    ref = O.integrate(w.normals, w.mask, w.camera, O.Params.from_dict(p))
    return w, depth.cpu().numpy(), labels.cpu().numpy(), st, ref


@pytest.mark.parametrize("name", ["c1", "c2", "c3_small"])
@pytest.mark.parametrize("precond", [0, 1])
def test_integrate_matches_oracle(name, precond):
    w, depth, labels, st, ref = _run(name, precond=precond)
    zg = np.log(depth) if w.camera["camera"] == 1 else depth
    zr = np.nan_to_num(ref["z"])
    err = rel_depth_error(np.nan_to_num(zg), zr, w.mask, w.camera["camera"])
    mx = rel_depth_max(np.nan_to_num(zg), zr, w.mask, w.camera["camera"])
    print(name, "stats", {k: st[k] for k in ("K0", "K_final", "scale_iters", "fill_iters", "merges")},
          "oracle K0", ref["K0"], "K", ref["K"], "iters", ref["iters"], "err", err, "max", mx)
    assert st["K0"] == ref["K0"]
    assert np.isnan(depth[w.mask == 0]).all()
    if st["K_final"] == ref["K"] and st["scale_iters"] == ref["iters"]:
        np.testing.assert_array_equal(labels, ref["labels"])
        assert err <= 1e-4
        assert mx <= PIXEL_TOL
    else:
        pytest.fail(f"partition or iteration count differs: {st} vs oracle K={ref['K']} iters={ref['iters']}")


def test_integrate_host_equals_device():
    w = make_workload("c2")
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, w.params)
    d_dev, _, _ = it.integrate(n, m)
    nh = torch.from_numpy(w.normals).pin_memory()
    mh = torch.from_numpy(w.mask).pin_memory()
    out = torch.empty((H, W), dtype=torch.float32).pin_memory()
    it.integrate_host(nh, mh, out)
    a, b = d_dev.cpu().numpy(), out.numpy()
    assert np.array_equal(np.isnan(a), np.isnan(b))
    assert np.nanmax(np.abs(a - b) / np.abs(b)) < 1e-5


_C3_REF = {}


@pytest.mark.parametrize("precond", [0, 1])
def test_full_size_c3(precond):
    w = make_workload("c3")
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, w.params, precond=precond)
    depth, labels, st = it.integrate(n, m)
    if "ref" not in _C3_REF:
        _C3_REF["ref"] = O.integrate(w.normals, w.mask, w.camera, O.Params.from_dict(w.params))
    ref = _C3_REF["ref"]
    depth, labels = depth.cpu().numpy(), labels.cpu().numpy()
    err = rel_depth_error(np.nan_to_num(np.log(depth)), np.nan_to_num(ref["z"]), w.mask, 1)
    mx = rel_depth_max(np.nan_to_num(np.log(depth)), np.nan_to_num(ref["z"]), w.mask, 1)
    print("c3 precond", precond, "max", mx, {k: st[k] for k in ("K0", "K_final", "scale_iters", "fill_iters", "ms_fill", "ms_total")},
          "oracle", ref["K0"], ref["K"], ref["iters"], "err", err)
    assert st["K0"] == ref["K0"]
    assert st["K_final"] == ref["K"] and st["scale_iters"] == ref["iters"]
    np.testing.assert_array_equal(labels, ref["labels"])
    assert err <= 1e-4
    assert mx <= PIXEL_TOL


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_pixel_level_limit_matches_oracle(name):
    """theta_c = None: every pixel is its own component (the paper's pixel-level
    setting); the relative-scale loop then works on the pixel graph itself."""
    w, depth, labels, st, ref = _run(name, theta_c_deg=None)
    zg = np.log(depth) if w.camera["camera"] == 1 else depth
    err = rel_depth_error(np.nan_to_num(zg), np.nan_to_num(ref["z"]), w.mask, w.camera["camera"])
    mx = rel_depth_max(np.nan_to_num(zg), np.nan_to_num(ref["z"]), w.mask, w.camera["camera"])
    print(name, "pixel level", "max", mx, {k: st[k] for k in ("K0", "K_final", "scale_iters", "merges", "ms_scale")},
          "oracle", ref["K0"], ref["K"], ref["iters"], "err", err)
    assert st["K0"] == int(w.mask.sum()) == ref["K0"]
    assert st["K_final"] == ref["K"] and st["scale_iters"] == ref["iters"]
    np.testing.assert_array_equal(labels, ref["labels"])
    assert err <= 1e-4
    assert mx <= PIXEL_TOL


@pytest.mark.parametrize("over", [dict(hard_outliers=True), dict(L=1e-6), dict(L=1e-4, U=1e-2)],
                         ids=["hard", "L1e-6", "L1e-4_U1e-2"])
def test_outlier_variants_match_oracle(over):
    """The outlier reweighting variants of the supplementary ablation: the hard
    threshold and other (L, U) of Eq. 11."""
    w, depth, labels, st, ref = _run("c3_small", **over)
    err = rel_depth_error(np.nan_to_num(np.log(depth)), np.nan_to_num(ref["z"]), w.mask, 1)
    mx = rel_depth_max(np.nan_to_num(np.log(depth)), np.nan_to_num(ref["z"]), w.mask, 1)
    print(over, "max", mx, {k: st[k] for k in ("K0", "K_final", "scale_iters", "merges")}, "oracle", ref["K"], ref["iters"],
          "err", err)
    assert st["K_final"] == ref["K"] and st["scale_iters"] == ref["iters"]
    np.testing.assert_array_equal(labels, ref["labels"])
    assert err <= 1e-4
    assert mx <= PIXEL_TOL


@pytest.mark.parametrize("name,irls", [("c3_small", 1), ("c2", 2)])
def test_residual_bini_variant_matches_oracle(name, irls):
    """The residual-based BiNI weights (bini_residual) in the scale loop (and
    in the second fill sweep) against the oracle's variant."""
    w, depth, labels, st, ref = _run(name, bini_residual=1, n_fill_irls=irls)
    zg = np.log(depth) if w.camera["camera"] == 1 else depth
    err = rel_depth_error(np.nan_to_num(zg), np.nan_to_num(ref["z"]), w.mask, w.camera["camera"])
    mx = rel_depth_max(np.nan_to_num(zg), np.nan_to_num(ref["z"]), w.mask, w.camera["camera"])
    print(name, "residual BiNI", {k: st[k] for k in ("K0", "K_final", "scale_iters", "merges")}, "oracle", ref["K"],
          ref["iters"], "err", err, "max", mx)
    assert st["K_final"] == ref["K"] and st["scale_iters"] == ref["iters"]
    np.testing.assert_array_equal(labels, ref["labels"])
    assert err <= 1e-4
    assert mx <= PIXEL_TOL
