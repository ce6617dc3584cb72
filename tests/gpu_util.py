"""Helpers shared by the GPU parity tests (inputs from synth, expectations
from the oracle, results from the CUDA library through its C ABI)."""
import numpy as np
import torch

import oracle as O
from paper_2510_11508_gb300 import ni


def dev(w_normals, w_mask):
    return (torch.from_numpy(np.ascontiguousarray(w_normals, dtype=np.float32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(w_mask, dtype=np.uint8)).cuda())


def integrator(H, W, camera, params=None, **over):
    return ni.Integrator(ni.config_for(H, W, camera, params, **over))


def island_rms(z, zref, mask):
    """RMS and max of z - zref after removing each island's mean difference
    (each island of the mask is determined up to one constant in log-depth)."""
    isl, n = O.islands(mask)
    z = np.asarray(z, np.float64)
    zr = np.asarray(zref, np.float64)
    d = np.zeros_like(zr)
    m = isl >= 0
    for i in range(n):
        s = isl == i
        dd = z[s] - zr[s]
        d[s] = dd - dd.mean()
    return float(np.sqrt(np.mean(d[m] ** 2))), float(np.max(np.abs(d[m])) if m.any() else 0.0)


def rel_depth_error(z, zref, mask, camera):
    """Relative depth RMSE of log-depth (or orthographic depth) z against zref
    after island-wise scale (perspective) or offset (orthographic) alignment."""
    m = mask > 0
    if camera == O.PERSP:
        return O.aligned_rel_rmse(np.where(m, np.exp(z), np.nan), np.where(m, np.exp(zref), np.nan), mask,
                                  O.PERSP)
    return O.aligned_rel_rmse(np.where(m, z, np.nan), np.where(m, zref, np.nan), mask, O.ORTHO)


# Per-pixel bound beside every RMSE bound: after the same island alignment, no
# pixel's relative depth error (perspective) or range-relative error
# (orthographic) may exceed this, so a small component with a wrong scale
# cannot hide inside a small RMSE.
PIXEL_TOL = 1e-3


def rel_depth_max(z, zref, mask, camera):
    """Largest per-pixel relative depth error of log-depth (or orthographic
    depth) z against zref after the island-wise alignment of rel_depth_error:
    max |s* e^z - e^zref| / e^zref (perspective) or max |z + o* - zref| /
    (max - min of zref) (orthographic)."""
    isl, n = O.islands(mask)
    m = isl >= 0
    if not m.any():
        return 0.0
    z = np.asarray(z, np.float64)
    zr = np.asarray(zref, np.float64)
    if camera == O.PERSP:
        z, zr = np.exp(np.where(m, z, 0.0)), np.exp(np.where(m, zr, 0.0))
    worst = 0.0
    for i in range(n):
        s = isl == i
        if camera == O.PERSP:
            den = np.sum(z[s] * z[s])
            al = z[s] * (np.sum(z[s] * zr[s]) / den if den > 0 else 1.0)
            worst = max(worst, float(np.max(np.abs(al - zr[s]) / np.abs(zr[s]))))
        else:
            al = z[s] + np.mean(zr[s] - z[s])
            worst = max(worst, float(np.max(np.abs(al - zr[s]))))
    if camera != O.PERSP:
        worst /= max(float(np.ptp(zr[m])), 1e-300)
    return worst
