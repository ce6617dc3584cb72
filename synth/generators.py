"""Analytic synthetic normal maps for the five benchmark workloads and for tests.

Conventions shared by every generator (they describe the *input*, not the
method):

* The image is H rows by W columns; pixel (u, v) has column u and row v, and
  raster index v * W + u.
* Perspective camera: the ray through pixel (u, v) is
  tau(u, v) = ((u - cx) / fx, (v - cy) / fy, 1) and the 3D point is
  P = z * tau, with z the depth along the optical axis.  Normals are the
  normalised cross product of dP/du and dP/dv, oriented towards the camera.
* Orthographic camera: P = (u, v, z) with unit pixel pitch; normals are
  proportional to (-z_u, -z_v, 1).
* Normals are returned as float32 [H, W, 4] (x, y, z, 0); invalid pixels hold
  zeros.  The mask is uint8 [H, W] (1 = valid).  The ground-truth depth is
  float64 [H, W] with NaN at invalid pixels.

Every random draw comes from numpy's PCG64 generator seeded explicitly, so a
workload is a pure function of its parameters.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional, Tuple

import numpy as np

ORTHO = 0
PERSP = 1


@dataclasses.dataclass
class Workload:
    name: str
    normals: np.ndarray          # float32 [H, W, 4]
    mask: np.ndarray             # uint8 [H, W]
    depth_gt: np.ndarray         # float64 [H, W], NaN where invalid
    camera: Dict[str, float]     # {"camera": 0|1, "fx", "fy", "cx", "cy"}
    params: Dict[str, object]    # method hyper-parameters used with this workload
    description: str = ""
    cells: Optional[np.ndarray] = None  # int32 [H, W] generating cell id (-1 invalid)

    @property
    def H(self) -> int:
        return int(self.mask.shape[0])

    @property
    def W(self) -> int:
        return int(self.mask.shape[1])

    @property
    def n_valid(self) -> int:
        return int(self.mask.sum())


# --------------------------------------------------------------------------
# normals from analytic depth derivatives
# --------------------------------------------------------------------------

def _pack(nx, ny, nz, mask) -> np.ndarray:
    H, W = mask.shape
    out = np.zeros((H, W, 4), np.float32)
    m = mask.astype(bool)
    out[..., 0] = np.where(m, nx, 0.0)
    out[..., 1] = np.where(m, ny, 0.0)
    out[..., 2] = np.where(m, nz, 0.0)
    return out


def _normals_persp(z, zu, zv, u, v, cam):
    """-(dP/du x dP/dv) normalised, with P = z * tau(u, v)."""
    fx, fy, cx, cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    tx = (u - cx) / fx
    ty = (v - cy) / fy
    # dP/du = zu * tau + z * (1/fx, 0, 0); dP/dv = zv * tau + z * (0, 1/fy, 0)
    ax, ay, az = zu * tx + z / fx, zu * ty, zu
    bx, by, bz = zv * tx, zv * ty + z / fy, zv
    nx = -(ay * bz - az * by)
    ny = -(az * bx - ax * bz)
    nz = -(ax * by - ay * bx)
    s = np.sqrt(nx * nx + ny * ny + nz * nz)
    return nx / s, ny / s, nz / s


def _normals_ortho(zu, zv):
    s = np.sqrt(zu * zu + zv * zv + 1.0)
    return -zu / s, -zv / s, 1.0 / s


def _add_noise(nx, ny, nz, sigma, rng, mask):
    if sigma <= 0:
        return nx, ny, nz
    H, W = mask.shape
    e = rng.normal(0.0, sigma, size=(3, H, W))
    nx, ny, nz = nx + e[0], ny + e[1], nz + e[2]
    s = np.sqrt(nx * nx + ny * ny + nz * nz)
    return nx / s, ny / s, nz / s


def _grid(H, W):
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    return u, v


def _persp_cam(H, W, f_scale=1.5):
    f = f_scale * W
    return {"camera": PERSP, "fx": f, "fy": f, "cx": W / 2.0, "cy": H / 2.0}


DEFAULT_PARAMS = dict(theta_c_deg=3.5, k=2.0, L=1e-5, U=1e-3, T=15, dE_max=1e-3,
                      can_merge=False, freq_merging=5, n_fill_irls=1)


def _params(**kw):
    p = dict(DEFAULT_PARAMS)
    p.update(kw)
    return p


# --------------------------------------------------------------------------
# config 1: 64x64 orthographic, plane + two raised hemispheres, no noise
# --------------------------------------------------------------------------

def c1_map() -> Workload:
    H = W = 64
    u, v = _grid(H, W)
    mask = ((u - 31.5) ** 2 + (v - 31.5) ** 2 <= 31.0 ** 2).astype(np.uint8)
    z = 0.1 * u + 0.05 * v
    zu = np.full_like(z, 0.1)
    zv = np.full_like(z, 0.05)
    for (uc, vc, R, step) in ((21.0, 24.0, 20.0, 5.0), (46.0, 45.0, 12.0, 8.0)):
        r2 = (u - uc) ** 2 + (v - vc) ** 2
        inside = np.sqrt(r2) <= R - 0.5
        h = np.sqrt(np.maximum(R * R - r2, 1e-12))
        z = np.where(inside, z + step + h, z)
        zu = np.where(inside, zu - (u - uc) / h, zu)
        zv = np.where(inside, zv - (v - vc) / h, zv)
    nx, ny, nz = _normals_ortho(zu, zv)
    cam = {"camera": ORTHO, "fx": 1.0, "fy": 1.0, "cx": 0.0, "cy": 0.0}
    depth = np.where(mask.astype(bool), z, np.nan)
    return Workload("c1_64_ortho", _pack(nx, ny, nz, mask), mask, depth, cam,
                    _params(theta_c_deg=2.0),
                    "64x64 orthographic disc mask: plane z=0.1u+0.05v with hemispheres "
                    "R=20 (step 5) and R=12 (step 8); exact float32 normals, no noise")


# --------------------------------------------------------------------------
# config 2 family: union-of-ellipses mask, Voronoi cells of Gaussian bumps
# --------------------------------------------------------------------------

def _ellipse_mask(H, W, target, rng, axes=(0.05, 0.14), centre_spread=0.25):
    mask = np.zeros((H, W), bool)
    u, v = _grid(H, W)
    s = min(H, W)
    tries = 0
    while mask.sum() < target and tries < 10000:
        tries += 1
        cu = W / 2 + rng.uniform(-centre_spread, centre_spread) * W
        cv = H / 2 + rng.uniform(-centre_spread, centre_spread) * H
        a = rng.uniform(*axes) * s
        b = rng.uniform(*axes) * s
        th = rng.uniform(0, math.pi)
        c, sn = math.cos(th), math.sin(th)
        du, dv = u - cu, v - cv
        x = (c * du + sn * dv) / a
        y = (-sn * du + c * dv) / b
        mask |= (x * x + y * y) <= 1.0
    return mask


def _nearest_site(points_uv, sites_uv):
    """Index of the nearest site for each point (Voronoi assignment)."""
    from scipy.spatial import cKDTree
    tree = cKDTree(sites_uv)
    try:
        _, idx = tree.query(points_uv, k=1, workers=-1)
    except TypeError:  # very old scipy
        _, idx = tree.query(points_uv, k=1)
    return idx.astype(np.int32)


def c2_type_map(H=512, W=612, n_cells=8, target_valid=40000, seed=1002, noise=0.01,
                name="c2_512x612_persp", params=None) -> Workload:
    """Voronoi cells of smooth Gaussian-bump surfaces on piecewise-constant depth
    offsets inside a union-of-ellipses mask (occlusion steps at cell borders)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cam = _persp_cam(H, W)
    semi = math.sqrt(target_valid / (4.0 * math.pi)) / min(H, W)
    mask = _ellipse_mask(H, W, target_valid, rng, axes=(0.6 * semi, 1.4 * semi))
    vv, uu = np.nonzero(mask)
    pts = np.stack([uu, vv], 1).astype(np.float64)
    pick = rng.choice(len(pts), size=n_cells, replace=False)
    sites = pts[pick]
    cell_of = _nearest_site(pts, sites)
    z = np.zeros(len(pts))
    zu = np.zeros(len(pts))
    zv = np.zeros(len(pts))
    order = np.argsort(cell_of, kind="stable")
    bounds = np.searchsorted(cell_of[order], np.arange(n_cells + 1))
    for c in range(n_cells):
        sel = order[bounds[c]:bounds[c + 1]]
        o = rng.uniform(50.0, 150.0)
        z[sel] = o
        if len(sel) == 0:
            continue
        for _ in range(3):
            # amplitude in pixel-pitch units at the patch depth (o / f depth units)
            A = rng.uniform(5.0, 30.0) * o / cam["fx"]
            sg = rng.uniform(10.0, 40.0)
            mu = pts[sel[rng.integers(len(sel))]]
            du = pts[sel, 0] - mu[0]
            dv = pts[sel, 1] - mu[1]
            g = A * np.exp(-(du * du + dv * dv) / (2 * sg * sg))
            z[sel] -= g                      # bumps protrude towards the camera
            zu[sel] += g * du / (sg * sg)
            zv[sel] += g * dv / (sg * sg)
    Z = np.full((H, W), np.nan)
    ZU = np.zeros((H, W))
    ZV = np.zeros((H, W))
    C = np.full((H, W), -1, np.int32)
    Z[vv, uu] = z
    ZU[vv, uu] = zu
    ZV[vv, uu] = zv
    C[vv, uu] = cell_of
    u, v = _grid(H, W)
    Zs = np.where(mask, Z, 100.0)
    nx, ny, nz = _normals_persp(Zs, ZU, ZV, u, v, cam)
    nx, ny, nz = _add_noise(nx, ny, nz, noise, rng, mask)
    m8 = mask.astype(np.uint8)
    return Workload(name, _pack(nx, ny, nz, m8), m8, Z, cam,
                    params if params is not None else _params(theta_c_deg=3.5),
                    f"{H}x{W} perspective, {n_cells} Voronoi cells of 3 Gaussian bumps "
                    f"on offsets U(50,150), noise {noise}", C)


# --------------------------------------------------------------------------
# config 3: power-law cells of quadric patches
# --------------------------------------------------------------------------

def _power_law_sizes(n, smin, smax, alpha, rng):
    q = (np.arange(n) + rng.uniform(0, 1, n)) / n
    r = (smin / smax) ** alpha
    return smin / (1.0 - q * (1.0 - r)) ** (1.0 / alpha)


def c3_map(H=2048, W=2048, n_cells=120, target_valid=2.5e6, seed=1003, noise=0.02,
           smin=20.0, smax=3e5, name="c3_2048_persp", params=None) -> Workload:
    """Power-diagram cells with power-law target areas; each cell is a random
    quadric patch at its own depth offset (steps at borders); the background
    outside every cell's disc is invalid."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cam = _persp_cam(H, W)
    scale = (H * W) / (2048.0 * 2048.0)
    sizes = _power_law_sizes(n_cells, max(smin, 4.0), smax * scale, 0.12, rng)
    sizes = np.clip(sizes * (1.25 * target_valid / sizes.sum()), smin, smax * scale)
    sizes = sizes[rng.permutation(n_cells)]
    order = np.argsort(-sizes, kind="stable")
    w = np.zeros(n_cells)
    sites = np.zeros((n_cells, 2))
    placed = []
    for j in order:
        w[j] = sizes[j] / math.pi
        rj = math.sqrt(w[j])
        best = None
        for _ in range(200):
            p = np.array([rng.uniform(rj * 0.3, W - rj * 0.3), rng.uniform(rj * 0.3, H - rj * 0.3)])
            ok = True
            for i in placed:
                if (p[0] - sites[i, 0]) ** 2 + (p[1] - sites[i, 1]) ** 2 - w[i] < -0.25 * w[j]:
                    ok = False
                    break
            if ok:
                best = p
                break
            if best is None:
                best = p
        sites[j] = best
        placed.append(j)
    # power diagram assignment, chunked over rows
    cell = np.full((H, W), -1, np.int32)
    u1 = np.arange(W, dtype=np.float64)
    rows = max(1, int(4e6 // (W * n_cells)) or 1)
    for r0 in range(0, H, rows):
        r1 = min(H, r0 + rows)
        vv = np.arange(r0, r1, dtype=np.float64)[:, None, None]
        uu = u1[None, :, None]
        pd = (uu - sites[None, None, :, 0]) ** 2 + (vv - sites[None, None, :, 1]) ** 2 - w[None, None, :]
        j = np.argmin(pd, axis=2)
        mn = np.take_along_axis(pd, j[..., None], 2)[..., 0]
        cell[r0:r1] = np.where(mn < 0, j, -1)
    mask = cell >= 0
    u, v = _grid(H, W)
    Z = np.full((H, W), np.nan)
    ZU = np.zeros((H, W))
    ZV = np.zeros((H, W))
    f = cam["fx"]
    d = rng.uniform(50.0, 150.0, n_cells)
    sx = rng.uniform(-0.6, 0.6, n_cells)
    sy = rng.uniform(-0.6, 0.6, n_cells)
    kx = rng.uniform(-0.5, 0.5, n_cells)
    ky = rng.uniform(-0.5, 0.5, n_cells)
    kxy = rng.uniform(-0.3, 0.3, n_cells)
    rad = np.sqrt(w) + 1.0
    cc = np.where(mask, cell, 0)
    du = u - sites[cc, 0]
    dv = v - sites[cc, 1]
    s = d[cc] / f                       # depth units per pixel at the patch
    R = rad[cc]
    Zq = d[cc] + s * (sx[cc] * du + sy[cc] * dv
                      + (kx[cc] * du * du + ky[cc] * dv * dv + kxy[cc] * du * dv) / (2 * R))
    Zu = s * (sx[cc] + (2 * kx[cc] * du + kxy[cc] * dv) / (2 * R))
    Zv = s * (sy[cc] + (2 * ky[cc] * dv + kxy[cc] * du) / (2 * R))
    Z = np.where(mask, Zq, np.nan)
    ZU = np.where(mask, Zu, 0.0)
    ZV = np.where(mask, Zv, 0.0)
    nx, ny, nz = _normals_persp(np.where(mask, Z, 100.0), ZU, ZV, u, v, cam)
    nx, ny, nz = _add_noise(nx, ny, nz, noise, rng, mask)
    m8 = mask.astype(np.uint8)
    return Workload(name, _pack(nx, ny, nz, m8), m8, Z, cam,
                    params if params is not None else
                    _params(theta_c_deg=5.0, can_merge=True, freq_merging=5),
                    f"{H}x{W} perspective, {n_cells} power-law cells (quadric patches), "
                    f"noise {noise}", cell)


# --------------------------------------------------------------------------
# config 5: spheres, tori and Gaussian-bump patches at 8192^2
# --------------------------------------------------------------------------

def c5_map(H=8192, W=8192, n_cells=600, valid_frac=0.67, seed=1005, noise=0.01,
           name="c5_8192_persp", params=None) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    cam = _persp_cam(H, W)
    f = cam["fx"]
    # jittered-grid Voronoi sites
    gy = int(round(math.sqrt(n_cells * H / W)))
    gx = int(math.ceil(n_cells / gy))
    sites = []
    for i in range(gy):
        for j in range(gx):
            if len(sites) < n_cells:
                sites.append(((j + rng.uniform(0.1, 0.9)) * W / gx, (i + rng.uniform(0.1, 0.9)) * H / gy))
    sites = np.array(sites)
    n_cells = len(sites)
    kind = rng.integers(0, 3, n_cells)             # 0 sphere cap, 1 torus, 2 bumps
    d = rng.uniform(50.0, 150.0, n_cells)
    sx = rng.uniform(-0.4, 0.4, n_cells)
    sy = rng.uniform(-0.4, 0.4, n_cells)
    Rs = rng.uniform(50.0, 800.0, n_cells)
    Rt = rng.uniform(40.0, 400.0, n_cells)
    rt = Rt * rng.uniform(0.15, 0.5, n_cells)
    nb = 3
    bA = rng.uniform(0.3, 1.5, (n_cells, nb))
    bS = rng.uniform(15.0, 120.0, (n_cells, nb))
    bO = rng.uniform(-1.0, 1.0, (n_cells, nb, 2))
    # holes: random ellipses removed until the valid fraction is reached
    hole_c = []
    nh = 0
    mask = np.ones((H, W), bool)
    coarse = 64
    uc, vc = np.meshgrid(np.arange(0, W, coarse) + coarse / 2, np.arange(0, H, coarse) + coarse / 2)
    keep = np.ones(uc.shape, bool)
    while True:
        cu, cv = rng.uniform(0, W), rng.uniform(0, H)
        a, b = rng.uniform(0.02, 0.08) * W, rng.uniform(0.02, 0.08) * H
        th = rng.uniform(0, math.pi)
        hole_c.append((cu, cv, a, b, th))
        nh += 1
        # estimate on a coarse lattice (holes accumulate: test only the new one)
        c_, s_ = math.cos(th), math.sin(th)
        x = (c_ * (uc - cu) + s_ * (vc - cv)) / a
        y = (-s_ * (uc - cu) + c_ * (vc - cv)) / b
        keep &= (x * x + y * y) > 1.0
        if keep.mean() <= valid_frac or nh > 2000:
            break
    # bounding box of each hole (2-pixel margin): outside it the ellipse test is true
    hole_box = []
    for (hu, hv, ha, hb, ht) in hole_c:
        c_, s_ = math.cos(ht), math.sin(ht)
        ex = math.sqrt((ha * c_) ** 2 + (hb * s_) ** 2)
        ey = math.sqrt((ha * s_) ** 2 + (hb * c_) ** 2)
        hole_box.append((max(0, int(math.floor(hu - ex)) - 2), min(W, int(math.ceil(hu + ex)) + 3),
                         max(0, int(math.floor(hv - ey)) - 2), min(H, int(math.ceil(hv + ey)) + 3)))
    from scipy.spatial import cKDTree
    tree = cKDTree(sites)
    Z = np.full((H, W), np.nan)
    nrm = np.zeros((H, W, 4), np.float32)
    cells = np.full((H, W), -1, np.int32)
    chunk = 512
    u1 = np.arange(W, dtype=np.float64)
    for r0 in range(0, H, chunk):
        r1 = min(H, r0 + chunk)
        v, u = np.mgrid[r0:r1, 0:W].astype(np.float64)
        m = np.ones(u.shape, bool)
        for (hu, hv, ha, hb, ht), (x0, x1, y0, y1) in zip(hole_c, hole_box):
            ya, yb = max(y0, r0), min(y1, r1)
            if ya >= yb or x0 >= x1:
                continue
            uu, vv = u[ya - r0:yb - r0, x0:x1], v[ya - r0:yb - r0, x0:x1]
            c_, s_ = math.cos(ht), math.sin(ht)
            x = (c_ * (uu - hu) + s_ * (vv - hv)) / ha
            y = (-s_ * (uu - hu) + c_ * (vv - hv)) / hb
            m[ya - r0:yb - r0, x0:x1] &= (x * x + y * y) > 1.0
        pts = np.stack([u.ravel(), v.ravel()], 1)
        try:
            _, ci = tree.query(pts, k=1, workers=-1)
        except TypeError:
            _, ci = tree.query(pts, k=1)
        ci = ci.reshape(u.shape).astype(np.int32)
        du = u - sites[ci, 0]
        dv = v - sites[ci, 1]
        s = d[ci] / f
        z = d[ci] + s * (sx[ci] * du + sy[ci] * dv)
        zu = s * sx[ci]
        zv = s * sy[ci]
        k = kind[ci]
        r2 = du * du + dv * dv
        # sphere caps (protruding towards the camera), cut at 0.95 R
        R = Rs[ci]
        cap = (k == 0) & (r2 < (0.95 * R) ** 2)
        h = np.sqrt(np.maximum(R * R - r2, 1e-9))
        z = np.where(cap, z - s * h, z)
        zu = np.where(cap, zu + s * du / h, zu)
        zv = np.where(cap, zv + s * dv / h, zv)
        # tori: tube around a circle of radius Rt, cut at 0.95 of the tube radius
        rho = np.sqrt(np.maximum(r2, 1e-12))
        q = rho - Rt[ci]
        tube = (k == 1) & (np.abs(q) < 0.95 * rt[ci])
        ht = np.sqrt(np.maximum(rt[ci] ** 2 - q * q, 1e-9))
        dh = -q / ht                          # d h / d rho
        z = np.where(tube, z - s * ht, z)
        zu = np.where(tube, zu - s * dh * du / rho, zu)
        zv = np.where(tube, zv - s * dh * dv / rho, zv)
        # Gaussian-bump patches
        for j in range(nb):
            bm = k == 2
            sg = bS[ci, j]
            mu_u = bO[ci, j, 0] * 0.5 * Rs[ci]
            mu_v = bO[ci, j, 1] * 0.5 * Rs[ci]
            eu, ev = du - mu_u, dv - mu_v
            A = bA[ci, j] * sg * s
            g = np.where(bm, A * np.exp(-(eu * eu + ev * ev) / (2 * sg * sg)), 0.0)
            z = z - g
            zu = zu + g * eu / (sg * sg)
            zv = zv + g * ev / (sg * sg)
        nx, ny, nz = _normals_persp(z, zu, zv, u, v, cam)
        nx, ny, nz = _add_noise(nx, ny, nz, noise, rng, m)
        nrm[r0:r1] = _pack(nx, ny, nz, m.astype(np.uint8))
        Z[r0:r1] = np.where(m, z, np.nan)
        cells[r0:r1] = np.where(m, ci, -1)
        mask[r0:r1] = m
    m8 = mask.astype(np.uint8)
    return Workload(name, nrm, m8, Z, cam,
                    params if params is not None else
                    # T = 15 with a merge every 5 iterations and no early stop:
                    # three merge rounds
                    _params(theta_c_deg=3.5, can_merge=True, freq_merging=5, dE_max=0.0),
                    f"{H}x{W} perspective, {n_cells} cells (sphere caps, tori, bump patches), "
                    f"noise {noise}", cells)


# --------------------------------------------------------------------------
# small analytic maps for pins and edge cases
# --------------------------------------------------------------------------

def plane_map(H, W, camera=PERSP, normal=(0.2, -0.1, -1.0), d=100.0, mask=None,
              dtype=np.float64, f_scale=1.5):
    """A single 3D plane n.X = -d (perspective) or z = a u + b v + c (orthographic).
    Returns (normals [H,W,4] of `dtype`, mask, depth_gt, camera)."""
    u, v = _grid(H, W)
    if mask is None:
        mask = np.ones((H, W), np.uint8)
    if camera == PERSP:
        cam = _persp_cam(H, W, f_scale)
        n = np.asarray(normal, np.float64)
        n = n / np.linalg.norm(n)
        tx = (u - cam["cx"]) / cam["fx"]
        ty = (v - cam["cy"]) / cam["fy"]
        z = -d / (n[0] * tx + n[1] * ty + n[2])
        nx = np.full_like(z, n[0]); ny = np.full_like(z, n[1]); nz = np.full_like(z, n[2])
    else:
        cam = {"camera": ORTHO, "fx": 1.0, "fy": 1.0, "cx": 0.0, "cy": 0.0}
        a, b = normal[0], normal[1]
        z = a * u + b * v + d
        nx, ny, nz = _normals_ortho(np.full_like(z, a), np.full_like(z, b))
    out = np.zeros((H, W, 4), dtype)
    m = mask.astype(bool)
    out[..., 0] = np.where(m, nx, 0); out[..., 1] = np.where(m, ny, 0); out[..., 2] = np.where(m, nz, 0)
    return out, mask.astype(np.uint8), np.where(m, z, np.nan), cam


def sphere_map(n, radius_frac=0.45, depth_c=10.0, sphere_r=2.0, f_scale=1.5, dtype=np.float64):
    """Perspective view of a sphere of radius `sphere_r` centred on the optical axis
    at depth `depth_c`, imaged on an n x n grid whose field of view is fixed
    (f = f_scale * n), so that halving the pixel pitch doubles n.  Only pixels
    whose ray hits the sphere well inside its silhouette are valid."""
    cam = _persp_cam(n, n, f_scale)
    u, v = _grid(n, n)
    tx = (u - cam["cx"]) / cam["fx"]
    ty = (v - cam["cy"]) / cam["fy"]
    # ray t*(tx, ty, 1) hits |X - C| = r, C = (0, 0, dc): t^2 |tau|^2 - 2 t dc + dc^2 - r^2 = 0
    a = tx * tx + ty * ty + 1.0
    disc = depth_c ** 2 - a * (depth_c ** 2 - sphere_r ** 2)
    hit = disc > 0
    t = (depth_c - np.sqrt(np.maximum(disc, 0))) / a
    X, Y, Zc = t * tx, t * ty, t
    nx, ny, nz = X / sphere_r, Y / sphere_r, (Zc - depth_c) / sphere_r
    # keep the part of the sphere that faces the camera well (|n.tau|/|tau| > 0.3)
    cosang = -(nx * tx + ny * ty + nz) / np.sqrt(a)
    rr = np.sqrt((u - cam["cx"]) ** 2 + (v - cam["cy"]) ** 2)
    mask = (hit & (cosang > 0.3) & (rr < radius_frac * n)).astype(np.uint8)
    out = np.zeros((n, n, 4), dtype)
    m = mask.astype(bool)
    out[..., 0] = np.where(m, nx, 0); out[..., 1] = np.where(m, ny, 0); out[..., 2] = np.where(m, nz, 0)
    return out, mask, np.where(m, t, np.nan), cam


def random_normal_field(H, W, n_dirs=4, jitter_deg=1.0, hole_frac=0.1, seed=0,
                        block=6):
    """Piecewise-constant normal directions on random blocks, jittered by a few
    degrees, with random holes: a seeding stress field (float32 normals)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dirs = rng.normal(size=(n_dirs, 3))
    dirs[:, 2] = -np.abs(dirs[:, 2]) - 1.0
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    bh, bw = (H + block - 1) // block, (W + block - 1) // block
    lab = rng.integers(0, n_dirs, (bh, bw))
    lab = np.kron(lab, np.ones((block, block), int))[:H, :W]
    n = dirs[lab]
    j = np.deg2rad(jitter_deg)
    n = n + rng.normal(0, j, n.shape)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    mask = (rng.uniform(size=(H, W)) >= hole_frac).astype(np.uint8)
    out = np.zeros((H, W, 4), np.float32)
    out[..., :3] = np.where(mask[..., None] > 0, n, 0)
    cam = _persp_cam(H, W)
    return out, mask, cam


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

_WORKLOADS = {
    "c1": lambda: c1_map(),
    "c2": lambda: c2_type_map(),
    "c3": lambda: c3_map(),
    "c3_small": lambda: c3_map(H=512, W=512, n_cells=30, target_valid=1.5e5, seed=1013,
                               smax=6e4, name="c3_512_persp"),
    "c4_eval": lambda: c2_type_map(H=4096, W=4096, n_cells=400, target_valid=1.2e7, seed=20000,
                                   name="c4_4096_persp",
                                   params=_params(theta_c_deg=3.5, can_merge=True)),
    "c5": lambda: c5_map(),
    "c5_small": lambda: c5_map(H=1024, W=1024, n_cells=24, seed=1015, name="c5_1024_persp"),
}


def workload_names():
    return list(_WORKLOADS)


def make_workload(name: str) -> Workload:
    if name.startswith("c4_train_"):
        s = int(name.split("_")[-1])
        return c2_type_map(H=256, W=256, n_cells=8, target_valid=0.128 * 256 * 256, seed=s,
                           name=name)
    return _WORKLOADS[name]()
