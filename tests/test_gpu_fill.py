"""Component fill (Sec. 3.3, Eqs. 9-10): the GPU's per-component log-depth
against the oracle's minimum-norm least-squares solution.

Tolerance: the accuracy bound is a relative depth RMSE of 1e-4 for the
FP64-reduction path and 1e-3 for the reduced-precision path; an error dz in
log-depth is a relative depth error of dz, so the same numbers bound the RMS of
the log-depth difference (orthographic: relative to the depth range)."""
import numpy as np
import pytest

import oracle as O
from synth import generators as G, make_workload

from gpu_util import PIXEL_TOL, dev, integrator, island_rms

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-3}


def _fill_pair(normals, mask, camera, params, **over):
    H, W = mask.shape
    n, m = dev(normals, mask)
    it = integrator(H, W, camera, params, **over)
    lab, K = it.seed_components(n, m)
    z = it.solve_components().cpu().numpy()
    cam = O.Camera.from_dict(camera)
    geo = O.geometry(normals, mask, cam)
    ref_lab, Kr = O.seed_components(normals, mask, params["theta_c_deg"])
    assert K == Kr
    zr, _ = O.fill_components(geo, ref_lab, Kr, params.get("k", 2.0), params.get("n_fill_irls", 1))
    zr = np.nan_to_num(zr).reshape(mask.shape)
    return z, zr, K


@pytest.mark.parametrize("name", ["c1", "c2", "c3_small"])
@pytest.mark.parametrize("batched", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_fill_matches_oracle(name, batched, precision):
    """Jacobi preconditioner (plain global PCG or batched tile PCG)."""
    w = make_workload(name)
    z, zr, K = _fill_pair(w.normals, w.mask, w.camera, w.params, batched=batched, precision=precision, precond=0)
    m = w.mask > 0
    # per-component zero mean on both sides: compare directly
    d = (z - zr)[m]
    scale = 1.0 if w.camera["camera"] == 1 else float(np.ptp(w.depth_gt[m]))
    rms = float(np.sqrt(np.mean(d * d))) / scale
    print(f"{name} batched={batched} prec={precision} K={K} fill rms={rms:.3e} max={np.abs(d).max():.3e}")
    assert rms <= TOL[precision]
    assert float(np.abs(d).max()) / scale <= PIXEL_TOL


@pytest.mark.parametrize("batched", [0, 1])
def test_fill_exact_plane(batched):
    nrm, mask, z, cam = G.plane_map(40, 53, G.PERSP, normal=(0.3, -0.2, -1.0), d=30.0, dtype=np.float32)
    zf, zr, K = _fill_pair(nrm, mask, cam, {"theta_c_deg": 5.0}, batched=batched, precond=0)
    assert K == 1
    rms, mx = island_rms(zf, np.log(z), mask)
    assert rms < 2e-6, rms


def test_fill_random_ragged_with_holes():
    nrm, mask, cam = G.random_normal_field(45, 77, n_dirs=2, jitter_deg=0.8, hole_frac=0.05, seed=3,
                                           block=9)
    z, zr, K = _fill_pair(nrm, mask, cam, {"theta_c_deg": 3.0}, batched=1, precond=0)
    d = (z - zr)[mask > 0]
    assert np.sqrt(np.mean(d * d)) < 1e-4
    assert float(np.abs(d).max()) <= PIXEL_TOL


def test_fill_irls_sweeps():
    w = make_workload("c3_small")
    p = dict(w.params, n_fill_irls=2)
    z, zr, K = _fill_pair(w.normals, w.mask, w.camera, p, batched=1, precond=0)
    d = (z - zr)[w.mask > 0]
    assert np.sqrt(np.mean(d * d)) < 1e-4
    assert float(np.abs(d).max()) <= PIXEL_TOL


# ---- multigrid-preconditioned batched fill (precond = 1): same answer, fewer iterations

@pytest.mark.parametrize("name", ["c1", "c2", "c3_small"])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("fill_kernels", [0, 1])
def test_fill_multigrid_matches_oracle(name, precision, fill_kernels):
    """Both multigrid drivers: per-phase kernels from a CUDA graph (0) and the
    persistent cooperative kernel (1)."""
    w = make_workload(name)
    z, zr, K = _fill_pair(w.normals, w.mask, w.camera, w.params, batched=1, precond=1, precision=precision,
                          fill_kernels=fill_kernels)
    m = w.mask > 0
    d = (z - zr)[m]
    scale = 1.0 if w.camera["camera"] == 1 else float(np.ptp(w.depth_gt[m]))
    rms = float(np.sqrt(np.mean(d * d))) / scale
    print(f"{name} multigrid prec={precision} K={K} fill rms={rms:.3e} max={np.abs(d).max():.3e}")
    assert rms <= TOL[precision]
    assert float(np.abs(d).max()) / scale <= PIXEL_TOL


def test_fill_multigrid_exact_plane():
    nrm, mask, z, cam = G.plane_map(40, 53, G.PERSP, normal=(0.3, -0.2, -1.0), d=30.0, dtype=np.float32)
    zf, zr, K = _fill_pair(nrm, mask, cam, {"theta_c_deg": 5.0}, batched=1, precond=1)
    assert K == 1
    rms, mx = island_rms(zf, np.log(z), mask)
    assert rms < 2e-6, rms


@pytest.mark.parametrize("H,W", [(45, 77), (1, 93), (97, 1), (2, 2), (33, 65)])
@pytest.mark.parametrize("fill_kernels", [0, 1])
def test_fill_multigrid_ragged_shapes(H, W, fill_kernels):
    nrm, mask, cam = G.random_normal_field(H, W, n_dirs=2, jitter_deg=0.8, hole_frac=0.05, seed=H * W,
                                           block=9)
    z, zr, K = _fill_pair(nrm, mask, cam, {"theta_c_deg": 3.0}, batched=1, precond=1, fill_kernels=fill_kernels)
    d = (z - zr)[mask > 0]
    assert np.sqrt(np.mean(d * d)) < 1e-4 if d.size else True
    assert float(np.abs(d).max()) <= PIXEL_TOL if d.size else True


def test_fill_multigrid_irls_sweeps():
    w = make_workload("c3_small")
    p = dict(w.params, n_fill_irls=2)
    z, zr, K = _fill_pair(w.normals, w.mask, w.camera, p, batched=1, precond=1)
    d = (z - zr)[w.mask > 0]
    assert np.sqrt(np.mean(d * d)) < 1e-4
    assert float(np.abs(d).max()) <= PIXEL_TOL


def test_multigrid_needs_fewer_iterations():
    w = make_workload("c3_small")
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    its = {}
    for pc in (0, 1):
        it = integrator(H, W, w.camera, w.params, batched=1, precond=pc)
        its[pc] = it.integrate(n, m)[2]["fill_iters"]
    print("fill iterations jacobi / multigrid", its)
    assert its[1] * 4 < its[0]


@pytest.mark.parametrize("om", [0.7, 0.8, 0.9, 0.95])
def test_multigrid_knobs_converge(om):
    """Every smoother weight the tuner may pick ends converged on the 2048^2 map
    (components the multigrid PCG leaves stalled are finished by the Jacobi
    fallback); the default weight needs no fallback."""
    w = make_workload("c3")
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, w.params, precond=1, mg_omega=om)
    st = it.integrate(n, m)[2]
    print("c3 multigrid", om, "fill iterations", st["fill_iters"], "fallbacks", st["fill_fallbacks"])
    assert st["fill_unconverged"] == 0
    if om == 0.9:
        assert st["fill_fallbacks"] == 0 and st["fill_iters"] < 400


@pytest.mark.parametrize("name", ["c2", "c3_small"])
def test_multigrid_mean_projection_option(name):
    """mg_flags bit 0 (the residual's component mean projected out before each
    V-cycle): same answer as the oracle."""
    w = make_workload(name)
    z, zr, K = _fill_pair(w.normals, w.mask, w.camera, w.params, batched=1, precond=1, mg_flags=1)
    d = (z - zr)[w.mask > 0]
    scale = 1.0 if w.camera["camera"] == 1 else float(np.ptp(w.depth_gt[w.mask > 0]))
    assert float(np.sqrt(np.mean(d * d))) / scale <= 1e-4
    assert float(np.abs(d).max()) / scale <= PIXEL_TOL


@pytest.mark.parametrize("batched,precond", [(0, 0), (1, 0), (1, 1)])
def test_fill_residual_bini_sweep_matches_oracle(batched, precond):
    """A second fill sweep with the residual-based BiNI weights (bini_residual)."""
    w = make_workload("c3_small")
    p = dict(w.params, n_fill_irls=2)
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, p, batched=batched, precond=precond, bini_residual=1)
    it.seed_components(n, m)
    z = it.solve_components().cpu().numpy()
    cam = O.Camera.from_dict(w.camera)
    geo = O.geometry(w.normals, w.mask, cam)
    lab, K = O.seed_components(w.normals, w.mask, p["theta_c_deg"])
    zr, _ = O.fill_components(geo, lab, K, p.get("k", 2.0), 2, residual=True)
    zr = np.nan_to_num(zr).reshape(H, W)
    zraw, _ = O.fill_components(geo, lab, K, p.get("k", 2.0), 2)
    d = (z - zr)[w.mask > 0]
    sep = float(np.abs(np.nan_to_num(zraw).reshape(H, W) - zr)[w.mask > 0].max())
    print("residual sweep rms", float(np.sqrt(np.mean(d * d))), "max", float(np.abs(d).max()),
          "raw vs residual oracle max", sep)
    assert np.sqrt(np.mean(d * d)) < 1e-4
    assert float(np.abs(d).max()) <= PIXEL_TOL
