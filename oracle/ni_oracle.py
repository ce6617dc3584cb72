"""Plain, slow FP64 CPU oracle of the paper's method (arXiv 2510.11508).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline / reference legs of ``bench.py``; the product path
(the CUDA library and its Python binding) never imports, links or runs it.

It follows the method's steps in the paper's order (Algorithm 1 of the
supplementary "Pseudocode of our method"), in float64, with scipy.sparse
matrices and its direct sparse solves of the normal equations.  Library primitives used as
steps: sparse matrix products, ``scipy.sparse.csgraph.connected_components``,
``numpy`` sorts and reductions.  Nothing is blocked, fused or reordered beyond
what the equations state: every system is assembled row by row exactly as the
paper writes its design matrices, and solved through the normal equations.

Notation (the paper's):
    z~    log-depth per valid pixel (linear depth for the orthographic reading)
    w~    omega~_{b->a}, the model-of-continuity coefficient of a directed edge
    chi   residual z~_a - z~_b - w~_{b->a}
    pi    pixel -> component map of the current partition
    s~    per-component log-scale

Readings of passages the paper leaves open are marked "Reading:" where used.
Parity status of each function is stated in its docstring; the pins live in
tests/test_oracle_pins.py.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

ORTHO = 0
PERSP = 1
RIGHT = 0
DOWN = 1
DOWN_RIGHT = 2
DOWN_LEFT = 3
# (du, dv) from a to b for each edge direction; 4-connectivity uses the first two
STEP_U = np.array([1, 0, 1, -1], np.int64)
STEP_V = np.array([0, 1, 1, 1], np.int64)


@dataclasses.dataclass
class Camera:
    camera: int = PERSP
    fx: float = 1.0
    fy: float = 1.0
    cx: float = 0.0
    cy: float = 0.0

    @staticmethod
    def from_dict(d):
        return Camera(int(d["camera"]), float(d["fx"]), float(d["fy"]), float(d["cx"]), float(d["cy"]))


@dataclasses.dataclass
class Params:
    """Algorithm 1 inputs (theta_c, can merge, freq_merging, dE_max, T) plus the
    hyper-parameters of the weights (k of the BiNI sigmoid, L and U of the
    outlier reweighting) and the solver tolerances.  theta_c_deg=None is the
    paper's single-pixel limit (every pixel its own component)."""
    theta_c_deg: Optional[float] = 3.5
    k: float = 2.0
    L: float = 1e-5
    U: float = 1e-3
    T: int = 15
    dE_max: float = 1e-3
    can_merge: bool = False
    freq_merging: int = 5
    n_fill_irls: int = 1
    hard_outliers: bool = False
    connectivity: int = 4
    bini_residual: bool = False

    @staticmethod
    def from_dict(d):
        p = Params()
        for k_, v_ in d.items():
            if hasattr(p, k_):
                setattr(p, k_, v_)
        return p


# ---------------------------------------------------------------------------
# geometry: rays, edges, model of continuity (Sec. 3.1)
# ---------------------------------------------------------------------------

def rays(H: int, W: int, cam: Camera) -> np.ndarray:
    """Ray direction tau(u, v) per pixel, [H*W, 3].

    Reading (Sec. 3.1, Eq. 3 names tau only as "ray direction vectors"): for the
    pinhole camera of Eq. 2, tau(u, v) = ((u - c_x)/f_x, (v - c_y)/f_y, 1) with
    u the column and v the row, so that the 3D point is z * tau and z is the depth
    along the optical axis.  Orthographic reading: tau = (0, 0, 1).
    """
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    if cam.camera == PERSP:
        t = np.stack([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, np.ones_like(u)], -1)
    else:
        t = np.stack([np.zeros_like(u), np.zeros_like(u), np.ones_like(u)], -1)
    return t.reshape(-1, 3)


def edge_id(a, d, conn=4):
    """Edge id: 2 * a + dir with 4-connectivity, 4 * a + dir with 8."""
    return (2 if conn == 4 else 4) * np.asarray(a, np.int64) + np.asarray(d, np.int64)


def edge_list(mask: np.ndarray, conn: int = 4):
    """All edges of the pixel graph G_0 = (V, E) (Sec. 3.2): pairs (a, b) of
    valid neighbouring pixels, b the right (dir 0) or lower (dir 1) neighbour
    of a; with 8-connectivity (the setting of the paper's DiLiGenT experiments
    and of its connectivity ablation) also the lower-right (dir 2) and
    lower-left (dir 3) neighbour.  Edges are returned sorted by edge_id."""
    if conn not in (4, 8):
        raise ValueError("connectivity must be 4 or 8")
    H, W = mask.shape
    m = mask.reshape(-1).astype(bool)
    idx = np.arange(H * W, dtype=np.int64)
    u = idx % W
    v = idx // W
    parts_a, parts_d = [], []
    for dr in range(2 if conn == 4 else 4):
        du, dv = int(STEP_U[dr]), int(STEP_V[dr])
        inside = (u + du >= 0) & (u + du < W) & (v + dv < H) & m
        a_ = idx[inside]
        a_ = a_[m[a_ + du + dv * W]]
        parts_a.append(a_)
        parts_d.append(np.full(len(a_), dr, np.int64))
    a = np.concatenate(parts_a)
    d = np.concatenate(parts_d)
    b = a + STEP_U[d] + STEP_V[d] * W
    order = np.argsort(edge_id(a, d, conn), kind="stable")
    return a[order], b[order], d[order]


def _normals64(normals: np.ndarray) -> np.ndarray:
    n = np.asarray(normals)
    return n.reshape(-1, n.shape[-1])[:, :3].astype(np.float64)


def omega(normals, cam: Camera, H: int, W: int, a, b, d) -> np.ndarray:
    """Coefficient w~_{b->a} of the model of continuity for each edge.

    Perspective: Eq. 3 (the model of Milano et al. the paper adopts),
        w~_{b->a} = log( (n_a.tau_m * n_b.tau_b) / (n_a.tau_a * n_b.tau_m) ),
    with m the midpoint of a and b (Reading: "a subpixel that interpolates
    between a and b" is the midpoint).  Reading: the logarithm is taken of the
    absolute value of the ratio (it is positive for any surface seen from both
    rays), each product clamped below at 1e-300.

    Orthographic (Reading: the paper treats central cameras only): the same
    tangent-plane construction with parallel rays in linear depth gives
    z_a - z_b = (n_ax/n_az + n_bx/n_bz) / 2 for b right of a, and the same with
    n_y for b below a; for b = a + (du, dv) on a diagonal, the sum of the two
    (du = +1 or -1, dv = +1); with a and b swapped, the negative.

    Pinned: exact on planes (closed form) and O(h^2) on a sphere.
    """
    n = _normals64(normals)
    if cam.camera == PERSP:
        tau = rays(H, W, cam)
        ua, va = (a % W).astype(np.float64), (a // W).astype(np.float64)
        ub, vb = (b % W).astype(np.float64), (b // W).astype(np.float64)
        um, vm = 0.5 * (ua + ub), 0.5 * (va + vb)
        tm = np.stack([(um - cam.cx) / cam.fx, (vm - cam.cy) / cam.fy, np.ones_like(um)], -1)
        na_tm = np.sum(n[a] * tm, 1)
        nb_tb = np.sum(n[b] * tau[b], 1)
        na_ta = np.sum(n[a] * tau[a], 1)
        nb_tm = np.sum(n[b] * tm, 1)
        num = np.maximum(np.abs(na_tm * nb_tb), 1e-300)
        den = np.maximum(np.abs(na_ta * nb_tm), 1e-300)
        return np.log(num / den)
    gx = n[a, 0] / n[a, 2] + n[b, 0] / n[b, 2]
    gy = n[a, 1] / n[a, 2] + n[b, 1] / n[b, 2]
    # b = a - step(d) (the reversed edge) flips the sign
    sgn = np.sign(np.asarray(b, np.int64) - np.asarray(a, np.int64)).astype(np.float64)
    return sgn * (0.5 * np.select([d == RIGHT, d == DOWN, d == DOWN_RIGHT], [gx, gy, gx + gy], gy - gx))


def gamma(normals, cam: Camera, H: int, W: int, p, d) -> np.ndarray:
    """gamma_{.->p} = f * n_p . tau_p (Sec. 3.1, Eq. 6), the pixel factor of the
    BiNI weight.  Reading: f = f_x for horizontal edges and f_y for vertical
    ones, as in Eq. 2, and sqrt(f_x f_y) for diagonal ones (the paper names a
    single focal length); orthographic: f = 1, tau = (0, 0, 1), so gamma = n_pz."""
    n = _normals64(normals)
    tau = rays(H, W, cam)
    nt = np.sum(n[p] * tau[p], 1)
    if cam.camera == PERSP:
        f = np.select([d == RIGHT, d == DOWN], [cam.fx, cam.fy], math.sqrt(cam.fx * cam.fy))
        return f * nt
    return nt


def sigmoid(x, k=1.0):
    """sigma_k(x) = 1 / (1 + exp(-k x)) (Sec. 3.1, after Eq. 4)."""
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(-k * np.asarray(x, np.float64)))


def bini_weight(zt, gam, a, b, d, H, W, valid, k, same_component=None, omega_of=None):
    """Directed BiNI weight W_{b->a} = gamma_{b->a}^2 * w^BiNI_{b->a}
    (Sec. 3.1, Eqs. 4-5):
        w^BiNI_{b->a} = sigma_k( gamma^2 ((z~_{-b} - z~_a)^2 - (z~_b - z~_a)^2) ),
    where -b is a's neighbour on the side opposite to b.

    Reading: when -b is outside the image, invalid, or (during the component
    fill, `same_component` given) outside a's component, its squared difference
    is taken as 0.
    a, b: endpoints with b = a + step(d) or b = a - step(d); the opposite
    neighbour is a - (b - a).

    Residual-based variant (omega_of given; the outlier-reweighting ablation's
    family of variants, Sec. 3.1 read with the residual chi of Eq. 4 in place
    of the raw log-depth difference):
        w^BiNI_{b->a} = sigma_k( gamma^2 (chi_{-b->a}^2 - chi_{b->a}^2) ),
        chi_{c->a} = z~_a - z~_c - w~_{c->a},
    so that a smooth but steep surface, whose raw differences are large on
    both sides, is not mistaken for a discontinuity.  omega_of(a, c, d) gives
    w~_{c->a} for pixels a, c along direction d.
    Pinned: limits and worked values of the sigmoid form, the opposite
    neighbour on each side, and the same-component branch
    (tests/test_oracle_pins.py, tests/test_oracle_scale_rows_pins.py).
    """
    step = b - a
    ob = a - step
    ua, va = a % W, a // W
    sgn = np.sign(step)
    du = -sgn * STEP_U[d]
    dv = -sgn * STEP_V[d]
    uo, vo = ua + du, va + dv
    inside = (uo >= 0) & (uo < W) & (vo >= 0) & (vo < H)
    obc = np.where(inside, ob, 0)
    ok = inside & valid[obc]
    if same_component is not None:
        ok &= same_component[obc] == same_component[a]
    if omega_of is None:
        opp = np.where(ok, (zt[obc] - zt[a]) ** 2, 0.0)
        x = gam * gam * (opp - (zt[b] - zt[a]) ** 2)
    else:
        chi_o = zt[a] - zt[obc] - omega_of(a, obc, d)
        chi_b = zt[a] - zt[b] - omega_of(a, b, d)
        opp = np.where(ok, chi_o ** 2, 0.0)
        x = gam * gam * (opp - chi_b ** 2)
    return gam * gam * sigmoid(x, k)


def outlier_weight(chi_abs, L=1e-5, U=1e-3, hard=False):
    """Soft outlier reweighting W^out (Sec. 3.4, Eq. 11):
        sigma_1( 4/(L~ - U~) * (2 log10|chi| - (L~ + U~)) ),  ~ = log10,
    mapping |chi| = U to sigma(-4) and |chi| = L to sigma(4).
    Reading: |chi| is clamped below at 1e-30, so |chi| = 0 gives weight 1.
    hard=True is the ablation's hard variant (supplementary): 0 if |chi| >= U,
    else 1."""
    x = np.maximum(np.abs(np.asarray(chi_abs, np.float64)), 1e-30)
    if hard:
        return (x < U).astype(np.float64)
    Lt, Ut = math.log10(L), math.log10(U)
    return sigmoid(4.0 / (Lt - Ut) * (2.0 * np.log10(x) - (Lt + Ut)), 1.0)


# ---------------------------------------------------------------------------
# seeding (Sec. 3.3, first paragraph)
# ---------------------------------------------------------------------------

def cos_theta(theta_c_deg: float) -> float:
    """cos(theta_c) evaluated once, as cos(theta_deg * (pi / 180))."""
    return math.cos(theta_c_deg * (math.pi / 180.0))


def seed_edge_keep(normals, a, b, theta_c_deg) -> np.ndarray:
    """Edge predicate of Sec. 3.3: theta_{a,b} = arccos(n_a . n_b) < theta_c,
    evaluated as n_a . n_b > cos(theta_c) (arccos is decreasing), with the dot
    product of the input values summed in float64 in the order x, y, z.
    theta_c = None keeps no edge (single-pixel components, Sec. 3.2)."""
    if theta_c_deg is None:
        return np.zeros(len(a), bool)
    n = _normals64(normals)
    dot = n[a, 0] * n[b, 0] + n[a, 1] * n[b, 1]
    dot = dot + n[a, 2] * n[b, 2]
    return dot > cos_theta(theta_c_deg)


def canonical_labels(n_nodes: int, nodes: np.ndarray, ea, eb):
    """Connected components of the graph (nodes, edges ea-eb), labelled
    canonically: a component's label is the rank of its smallest node index
    among all components' smallest node indices.  Returns (label per node of
    `nodes`, K).  Reading: the paper leaves the order of pi_m open (Eq. 7)."""
    if len(nodes) == 0:
        return np.zeros(0, np.int64), 0
    pos = np.full(n_nodes, -1, np.int64)
    pos[nodes] = np.arange(len(nodes))
    g = sp.coo_matrix((np.ones(len(ea)), (pos[ea], pos[eb])), shape=(len(nodes), len(nodes)))
    ncc, cc = connected_components(g, directed=False)
    mins = np.full(ncc, np.iinfo(np.int64).max)
    np.minimum.at(mins, cc, nodes)
    rank = np.empty(ncc, np.int64)
    rank[np.argsort(mins, kind="stable")] = np.arange(ncc)
    return rank[cc], int(ncc)


def seed_components(normals, mask, theta_c_deg, conn=4):
    """Initial partition {C_c^(0)}: connected components of the subgraph of G_0
    that keeps the edges with theta_{a,b} < theta_c (Sec. 3.3).  Returns
    (labels int64 [H*W], -1 at invalid pixels; K)."""
    H, W = mask.shape
    a, b, d = edge_list(mask, conn)
    keep = seed_edge_keep(normals, a, b, theta_c_deg)
    valid_idx = np.nonzero(mask.reshape(-1))[0]
    lab, K = canonical_labels(H * W, valid_idx, a[keep], b[keep])
    labels = np.full(H * W, -1, np.int64)
    labels[valid_idx] = lab
    return labels, K


# ---------------------------------------------------------------------------
# linear algebra helpers
# ---------------------------------------------------------------------------

def project_zero_mean(x, block, nblocks):
    """Remove each block's mean (the gauge of a singular Laplacian block)."""
    cnt = np.bincount(block, None, nblocks)
    s = np.bincount(block, x, nblocks)
    mean = np.where(cnt > 0, s / np.maximum(cnt, 1), 0.0)
    return x - mean[block]


# Blocks above this many nodes are solved by CG instead of sparse LU (the LU's
# fill-in of a grid Laplacian of a few million nodes exceeds host memory).
LU_MAX_NODES = 1_500_000
CG_RTOL = 1e-12


def cg_min_norm(M, g, rtol=CG_RTOL, maxiter=None):
    """cg(M, g) from x = 0 (Eq. 10 / Eq. 14 as the paper states them) on one
    connected, singular Laplacian block: Jacobi-preconditioned conjugate
    gradients in float64 until ||g - M x|| <= rtol ||g||, then the block's mean
    removed.  g is first projected onto the range of M (zero sum), which CG from
    0 would otherwise carry as a constant drift.  Returns (x, iterations)."""
    M = sp.csr_matrix(M)
    g = np.asarray(g, np.float64)
    g = g - g.mean()
    n = M.shape[0]
    d = M.diagonal()
    inv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    x = np.zeros(n)
    r = g.copy()
    gn = float(np.linalg.norm(g))
    if gn == 0.0:
        return x, 0
    z = inv * r
    p = z.copy()
    rz = float(r @ z)
    it = 0
    for it in range(1, (maxiter or 20 * n) + 1):
        q = M @ p
        pq = float(p @ q)
        if pq <= 0.0:
            break
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) <= rtol * gn:
            break
        z = inv * r
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x - x.mean(), it


def solve_min_norm(M, g):
    """Minimum-norm solution of the singular normal equations M x = g of a
    weighted graph Laplacian M (the result cg(M, g) approaches from x = 0).

    Written out as its definition, block by block: on each connected block of
    M's graph (off-diagonal entries != 0) one node is pinned to 0, the remaining
    nonsingular system is solved by sparse LU (scipy's spsolve), and the block's
    mean is removed (the null space of a connected Laplacian block is the
    constants).  Isolated nodes get 0.  Blocks of more than LU_MAX_NODES nodes
    are solved by `cg_min_norm` instead (the CG the paper names, to a relative
    residual of 1e-12).  Returns x."""
    from scipy.sparse.linalg import spsolve
    M = sp.csr_matrix(M)
    n = M.shape[0]
    if n == 0:
        return np.zeros(0)
    off = M - sp.diags(M.diagonal())
    off.eliminate_zeros()
    nb, blk = connected_components(off, directed=False)
    g = np.asarray(g, np.float64)
    # blocks made contiguous: the blocks of P M P^T are its diagonal blocks
    order = np.argsort(blk, kind="stable")
    bounds = np.searchsorted(blk[order], np.arange(nb + 1))
    Mp = M[order][:, order].tocsr()
    gp = g[order]
    xp = np.zeros(n)
    for c in range(nb):
        b0, b1 = bounds[c], bounds[c + 1]
        if b1 - b0 < 2:
            continue
        if b1 - b0 > LU_MAX_NODES:
            xp[b0:b1] = cg_min_norm(Mp[b0:b1, b0:b1], gp[b0:b1])[0]
            continue
        # pin the block's first node (its smallest index) to 0
        Mk = Mp[b0 + 1:b1, b0 + 1:b1].tocsc()
        # symmetric minimum-degree ordering: the fill-in of a grid Laplacian
        # stays near-linear, so components of 1e6 pixels fit in host memory
        xp[b0 + 1:b1] = spsolve(Mk, gp[b0 + 1:b1], permc_spec="MMD_AT_PLUS_A")
    x = np.zeros(n)
    x[order] = xp
    return project_zero_mean(x, blk, nb)


# ---------------------------------------------------------------------------
# component fill (Sec. 3.3, Eq. 9-10)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Geometry:
    H: int
    W: int
    valid: np.ndarray    # bool [H*W]
    a: np.ndarray
    b: np.ndarray
    d: np.ndarray
    omega: np.ndarray    # w~_{b->a} per edge
    gam_ba: np.ndarray   # gamma_{b->a} = f n_a.tau_a per edge
    gam_ab: np.ndarray   # gamma_{a->b} = f n_b.tau_b per edge
    conn: int = 4        # pixel connectivity (4 or 8)
    normals: Optional[np.ndarray] = None
    cam: Optional[Camera] = None

    def omega_of(self, a, c, d):
        """w~_{c->a} (Eq. 3) for pixel pairs a, c = a +- step(d)."""
        return omega(self.normals, self.cam, self.H, self.W, np.asarray(a), np.asarray(c), np.asarray(d))


def geometry(normals, mask, cam: Camera, conn: int = 4) -> Geometry:
    H, W = mask.shape
    a, b, d = edge_list(mask, conn)
    return Geometry(H, W, mask.reshape(-1).astype(bool), a, b, d,
                    omega(normals, cam, H, W, a, b, d),
                    gamma(normals, cam, H, W, a, d),
                    gamma(normals, cam, H, W, b, d), conn, normals, cam)


def intra_system(geo: Geometry, labels, zt, k, residual=False):
    """A_c, b_c, W_c of Eq. 9 stacked over all components (block diagonal):
    two rows per intra-component edge (a, b), one per direction,
        row (b->a): +1 at a, -1 at b, rhs w~_{b->a},         weight W_{b->a}
        row (a->b): +1 at b, -1 at a, rhs w~_{a->b} = -w~_{b->a}, weight W_{a->b}
    with W from the BiNI model (Eq. 5) at the current z~ (Reading: -b restricted
    to a's component); residual=True takes the residual-based variant of
    `bini_weight`."""
    n = geo.H * geo.W
    sel = (labels[geo.a] == labels[geo.b]) & (labels[geo.a] >= 0)
    a, b, om = geo.a[sel], geo.b[sel], geo.omega[sel]
    ne = len(a)
    rows = np.repeat(np.arange(2 * ne), 2)
    cols = np.empty(4 * ne, np.int64)
    vals = np.empty(4 * ne)
    cols[0::4], cols[1::4], cols[2::4], cols[3::4] = a, b, b, a
    vals[0::4], vals[1::4], vals[2::4], vals[3::4] = 1.0, -1.0, 1.0, -1.0
    A = sp.csr_matrix((vals, (rows, cols)), shape=(2 * ne, n))
    rhs = np.empty(2 * ne)
    rhs[0::2], rhs[1::2] = om, -om
    w = np.empty(2 * ne)
    of = geo.omega_of if residual else None
    w[0::2] = bini_weight(zt, geo.gam_ba[sel], a, b, geo.d[sel], geo.H, geo.W, geo.valid, k, labels, of)
    w[1::2] = bini_weight(zt, geo.gam_ab[sel], b, a, geo.d[sel], geo.H, geo.W, geo.valid, k, labels, of)
    return A, rhs, w


def fill_components(geo: Geometry, labels, K, k=2.0, n_irls=1, residual=False):
    """Fill each component (Sec. 3.3): z~ initialised to 0, then
    z~_c <- cg(A_c^T W_c A_c, A_c^T W_c b_c) for every component independently
    (the blocks of one block-diagonal system).  The oracle computes the result
    CG converges to from z~ = 0, the minimum-norm (zero-mean per component)
    least-squares solution, directly (`solve_min_norm`).  `n_irls` sweeps
    recompute W at the current z~; the paper finds one sweep sufficient.
    residual=True takes the residual-based BiNI weights in the sweeps after
    the first (Reading: the first sweep starts from z~ = 0, where the paper's
    weights are sigma(0) = 1/2; a residual is only defined once a solution
    exists).
    Returns (z~ [H*W] with NaN at invalid pixels, number of sweeps)."""
    n = geo.H * geo.W
    vidx = np.nonzero(geo.valid)[0]
    zt = np.zeros(n)
    blk = labels[vidx]
    iters = 0
    for sweep in range(max(1, n_irls)):
        A, rhs, w = intra_system(geo, labels, zt, k, residual and sweep > 0)
        Wd = sp.diags(w)
        M = (A.T @ Wd @ A).tocsr()[vidx][:, vidx]
        g = (A.T @ (w * rhs))[vidx]
        zt[vidx] = project_zero_mean(solve_min_norm(M, g), blk, K)
        iters += 1
    out = np.full(n, np.nan)
    out[vidx] = zt[vidx]
    return out, iters


def _fill_crops(task):
    """Worker of fill_components_by_crops: the fill of each component of the
    task on the crop of its bounding box, every pixel outside the component
    masked out and the principal point shifted by the crop's offset.
    Returns [(component, v0, u0, crop mask, z~ on the crop mask)]."""
    cam_t, k, n_irls, conn, items, residual = task
    cam = Camera(*cam_t)
    out = []
    for c, v0, u0, ncrop, m in items:
        cc = Camera(cam.camera, cam.fx, cam.fy, cam.cx - u0, cam.cy - v0)
        geo = geometry(ncrop, m.astype(np.uint8), cc, conn)
        lab = np.where(m.reshape(-1), 0, -1).astype(np.int64)
        z, _ = fill_components(geo, lab, 1, k, n_irls, residual)
        out.append((c, v0, u0, m, z.reshape(m.shape)[m]))
    return out


def fill_components_by_crops(normals, mask, cam: Camera, labels, K, k=2.0, n_irls=1, conn=4, workers=1,
                             task_px=1 << 21, residual=False):
    """The fill of Sec. 3.3 solved component by component, as the paper does
    (its components are filled independently, in parallel processes).

    A component's block of the block-diagonal system involves only its own
    pixels and intra-component edges, and every quantity of Eqs. 3-6 on those
    edges depends only on the two pixels' normals and ray directions.  So the
    block equals `fill_components` run on the crop of the component's bounding
    box with every other pixel masked out and (c_x, c_y) shifted by the crop's
    offset (integer shifts: the ray directions are the same numbers).  The
    opposite neighbour -b then counts only inside the component, which is the
    fill's reading of Eq. 4.  `workers` > 1 spreads the components over a
    spawn process pool.  Returns (z~ [H*W], NaN at invalid pixels; 1 sweep
    count as fill_components)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    H, W = mask.shape
    lab = np.asarray(labels).reshape(H, W)
    nrm = np.asarray(normals).reshape(H, W, -1)
    vv, uu = np.nonzero(lab >= 0)
    cl = lab[vv, uu]
    big = np.iinfo(np.int64).max
    v0 = np.full(K, big); v1 = np.full(K, -1); u0 = np.full(K, big); u1 = np.full(K, -1)
    np.minimum.at(v0, cl, vv); np.maximum.at(v1, cl, vv)
    np.minimum.at(u0, cl, uu); np.maximum.at(u1, cl, uu)
    size = np.bincount(cl, minlength=K)
    cam_t = (cam.camera, cam.fx, cam.fy, cam.cx, cam.cy)
    tasks, cur, cur_px = [], [], 0
    for c in np.argsort(-size, kind="stable"):
        c = int(c)
        if size[c] == 0:
            continue
        sl = (slice(int(v0[c]), int(v1[c]) + 1), slice(int(u0[c]), int(u1[c]) + 1))
        m = lab[sl] == c
        cur.append((c, int(v0[c]), int(u0[c]), np.ascontiguousarray(nrm[sl]), m))
        cur_px += m.size
        if cur_px >= task_px:
            tasks.append((cam_t, k, n_irls, conn, cur, residual)); cur, cur_px = [], 0
    if cur:
        tasks.append((cam_t, k, n_irls, conn, cur, residual))
    zt = np.full(H * W, np.nan)
    zt2 = zt.reshape(H, W)

    def put(res):
        for c, a0, b0, m, z in res:
            blk = zt2[a0:a0 + m.shape[0], b0:b0 + m.shape[1]]
            blk[m] = z

    if workers <= 1 or len(tasks) <= 1:
        for t in tasks:
            put(_fill_crops(t))
    else:
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            for res in ex.map(_fill_crops, tasks):
                put(res)
    return zt, max(1, n_irls)


# ---------------------------------------------------------------------------
# relative-scale optimisation (Sec. 3.4) and merging (Sec. 3.5)
# ---------------------------------------------------------------------------

def inter_edges(geo: Geometry, labels):
    """E_inter^(m) (Eq. 7): edges whose endpoints lie in different components."""
    return np.nonzero((labels[geo.a] != labels[geo.b]) & (labels[geo.a] >= 0))[0]


def residual(geo: Geometry, zt, e):
    """chi_{b->a} = z~_a - z~_b - w~_{b->a} (Eq. 4) on edges e."""
    return zt[geo.a[e]] - zt[geo.b[e]] - geo.omega[e]


def scale_system(geo: Geometry, labels, K, zt, t, params: Params, e=None):
    """A_m, b_m (Eq. 13) and W_m^(t) for iteration t.

    Two rows per inter edge (a, b):
        row (b->a): +1 at pi(a), -1 at pi(b), rhs w~_{b->a} - (z~_a - z~_b)
        row (a->b): +1 at pi(b), -1 at pi(a), rhs w~_{a->b} - (z~_b - z~_a)
    Weights: 1 for t <= 1 (alignment, Sec. 3.4); for t > 1 the BiNI weight W
    (Eq. 5) times W^out (Eq. 11) of |chi^(t-1)|, the residual at the current z~.
    Reading: z~ inside W is the current z~, and -b may be any valid pixel.
    params.bini_residual takes the residual-based BiNI weights (`bini_weight`).
    Pinned: every row of a 3-component map written out by hand at t = 2
    (tests/test_oracle_scale_rows_pins.py) and the dense least-squares solve
    of the same rows (tests/test_oracle_pins.py)."""
    if e is None:
        e = inter_edges(geo, labels)
    a, b = geo.a[e], geo.b[e]
    ne = len(e)
    rho = zt[a] - zt[b] - geo.omega[e]
    pa, pb = labels[a], labels[b]
    rows = np.repeat(np.arange(2 * ne), 2)
    cols = np.empty(4 * ne, np.int64)
    vals = np.empty(4 * ne)
    cols[0::4], cols[1::4], cols[2::4], cols[3::4] = pa, pb, pb, pa
    vals[0::4], vals[1::4], vals[2::4], vals[3::4] = 1.0, -1.0, 1.0, -1.0
    A = sp.csr_matrix((vals, (rows, cols)), shape=(2 * ne, K))
    rhs = np.empty(2 * ne)
    rhs[0::2], rhs[1::2] = -rho, rho
    if t <= 1:
        w = np.ones(2 * ne)
    else:
        wo = outlier_weight(np.abs(rho), params.L, params.U, params.hard_outliers)
        w = np.empty(2 * ne)
        of = geo.omega_of if params.bini_residual else None
        w[0::2] = bini_weight(zt, geo.gam_ba[e], a, b, geo.d[e], geo.H, geo.W, geo.valid, params.k, None, of) * wo
        w[1::2] = bini_weight(zt, geo.gam_ab[e], b, a, geo.d[e], geo.H, geo.W, geo.valid, params.k, None, of) * wo
    return A, rhs, w, e


def quotient_components(K, labels, geo: Geometry, e):
    """Connected components of Q_m (node -> id)."""
    pa, pb = labels[geo.a[e]], labels[geo.b[e]]
    g = sp.coo_matrix((np.ones(len(e)), (pa, pb)), shape=(K, K))
    ncc, cc = connected_components(g, directed=False)
    return cc, ncc


SCALE_RTOL = 1e-12
SCALE_FLOOR = 64.0 * 2.0 ** -53


def solve_scales(A, rhs, w, K, qcc, nq):
    """s~ <- cg(A^T W A, A^T W b) (Eq. 14) from s~ = 0, as the paper states it.

    Reading: the weights of t >= 2 (BiNI times W^out, Eqs. 5 and 11) span
    hundreds of decades on large maps, so this Laplacian can be singular to
    working precision away from its exact null space; a direct solve then
    turns the rounding noise of the right-hand side into arbitrarily large
    offsets, while CG, the solver the paper names, leaves those directions
    nearly untouched.  So the oracle runs CG: Jacobi-preconditioned, FP64, from
    0, until ||g - M s|| <= 1e-12 ||g|| or the residual reaches the rounding
    level of g, 64 eps ||g_abs||, where g_abs sums the absolute values of the
    terms that make up g (a system that is already solved has a right-hand
    side made of rounding noise); at most 4 K + 100 iterations.  The result is
    then given the minimum-norm gauge: zero mean on every block of M's weighted
    graph and on every connected component of Q_m.  Where M is well
    conditioned this is the minimum-norm least-squares solution (pinned against
    the dense pseudo-inverse in tests/test_oracle_pins.py).
    Returns (s~, CG iterations)."""
    Wd = sp.diags(w)
    M = (A.T @ Wd @ A).tocsr()
    wb = w * rhs
    g = A.T @ wb
    gabs = abs(A).T @ np.abs(wb)
    n = M.shape[0]
    d = M.diagonal()
    inv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    stop2 = max(SCALE_RTOL ** 2 * float(g @ g), SCALE_FLOOR ** 2 * float(gabs @ gabs))
    x = np.zeros(n)
    r = np.asarray(g, np.float64).copy()
    it = 0
    if float(r @ r) > stop2:
        z = inv * r
        p = z.copy()
        rz = float(r @ z)
        for it in range(1, 4 * n + 101):
            q = M @ p
            pq = float(p @ q)
            if not pq > 0.0:
                break
            alpha = rz / pq
            x += alpha * p
            r -= alpha * q
            if float(r @ r) <= stop2:
                break
            z = inv * r
            rz_new = float(r @ z)
            p = z + (rz_new / rz) * p
            rz = rz_new
    off = M - sp.diags(d)
    off.eliminate_zeros()
    nb, blk = connected_components(off, directed=False)
    x = project_zero_mean(x, blk, nb)
    return project_zero_mean(x, qcc, nq), it


def energy(A, rhs, w, s):
    """E_t = (A s - b)^T W (A s - b) (Sec. 3.4, last paragraph)."""
    r = A @ s - rhs
    return float(np.sum(w * r * r))


def merge_labels(labels, K, geo: Geometry, e, chi_abs32):
    """Merging (Sec. 3.5).  (i) for every node c of Q_m, the incident inter edge
    with the smallest |chi|; (ii) the subgraph of Q_m with those edges;
    (iii) its connected components are the new partition.

    Reading (tie-break, left open): edges are compared by the float32 value of
    |chi| (its bit pattern), then by the edge id (2 * a + dir with
    4-connectivity, 4 * a + dir with 8).  New labels are the
    ranks of each group's smallest old label (so label order follows the old
    one).  `chi_abs32` is float32 |chi| per edge in `e`.
    Returns (new labels [H*W], K_new, selected edge id per old component or -1)."""
    chi_abs32 = np.asarray(chi_abs32, np.float32)
    bits = chi_abs32.view(np.uint32).astype(np.uint64)
    eid = edge_id(geo.a[e], geo.d[e], geo.conn).astype(np.uint64)
    key = (bits << np.uint64(32)) | eid
    best = np.full(K, np.iinfo(np.uint64).max, np.uint64)
    pa, pb = labels[geo.a[e]], labels[geo.b[e]]
    np.minimum.at(best, pa, key)
    np.minimum.at(best, pb, key)
    has = best != np.iinfo(np.uint64).max
    sel_eid = np.where(has, (best & np.uint64(0xFFFFFFFF)).astype(np.int64), -1)
    # endpoints of the selected edges
    per = 2 if geo.conn == 4 else 4
    ea = sel_eid[has] // per
    ed = sel_eid[has] % per
    eb = ea + STEP_U[ed] + STEP_V[ed] * geo.W
    newlab, Kn = canonical_labels(K, np.arange(K), labels[ea], labels[eb])
    out = labels.copy()
    v = labels >= 0
    out[v] = newlab[labels[v]]
    return out, Kn, sel_eid


def converged_test(t_done, E, params: Params):
    """Stop rule of Algorithm 1: t = T, or relative energy change below dE_max.

    Reading: the energy test compares two consecutive discontinuity-aware
    iterations only (t_done >= 4).  The second alignment iteration re-solves an
    already solved system, so a test there would end every run after the
    alignment phase, against the iteration counts of 3 to 49 the paper reports.
    A previous energy below 1e-300 counts as converged."""
    if t_done >= params.T:
        return True
    if t_done >= 4:
        e1, e0 = E[t_done], E[t_done - 1]
        if e0 < 1e-300:
            return True
        return abs(e1 - e0) / e0 < params.dE_max
    return False


def scale_loop(geo: Geometry, labels, K, zt, params: Params, record=False):
    """The relative-scale loop of Algorithm 1 (Sec. 3.4-3.5), from the filled
    log-depth `zt` and partition `labels` (K components):
      while not converged:
        W_m^(t) = 1 if t <= 1 else W * W^out                   (Sec. 3.4)
        s~ <- cg(A_m^T W A_m, A_m^T W b_m)                      (Eq. 14)
        z~_c <- z~_c + s~_c 1                                   (Eqs. 7-8)
        t <- t + 1
        if can merge and t = 0 (mod freq_merging): merge       (Sec. 3.5)
        E_t; converged <- |E_t - E_(t-1)| / E_(t-1) < dE_max or t = T
    Reading: E_t is the energy of the system just solved, taken before any
    merge of the same iteration.  Returns a dict (z~, labels, K, energies, ...)."""
    params = Params.from_dict(dataclasses.asdict(params)) if isinstance(params, Params) else Params.from_dict(params)
    zt = np.where(geo.valid, np.nan_to_num(zt), 0.0)
    labels = labels.copy()
    E = {0: np.finfo(np.float64).eps}
    Ks = [K]
    t = 0
    merges = []
    steps = []
    e = inter_edges(geo, labels)
    qcc, nq = quotient_components(K, labels, geo, e)
    while True:
        A, rhs, w, e = scale_system(geo, labels, K, zt, t, params, e)
        s, it = solve_scales(A, rhs, w, K, qcc, nq)
        zt = zt + np.where(geo.valid, s[np.maximum(labels, 0)], 0.0)
        E_t = energy(A, rhs, w, s)
        t += 1
        E[t] = E_t
        if record:
            steps.append(dict(t=t, K=K, n_inter=len(e), cg_iters=it, s=s.copy(), E=E_t,
                              z=zt.copy(), labels=labels.copy()))
        if params.can_merge and t % params.freq_merging == 0:
            chi = np.abs(residual(geo, zt, e)).astype(np.float32)
            labels, K, sel = merge_labels(labels, K, geo, e, chi)
            merges.append(dict(t=t, K=K, selected=sel, labels=labels.copy()))
            e = inter_edges(geo, labels)
            qcc, nq = quotient_components(K, labels, geo, e)
        Ks.append(K)
        if converged_test(t, E, params):
            break
    return dict(z=np.where(geo.valid, zt, np.nan), labels=labels, K=K, Ks=Ks,
                energies=[E[i] for i in range(1, t + 1)], iters=t, merges=merges, steps=steps)


def integrate(normals, mask, cam, params, record=False, workers=0):
    """Algorithm 1 end to end: seeding (Sec. 3.3), fill (Eqs. 9-10), then the
    relative-scale loop with optional merging (Sec. 3.4-3.5).  Returns a dict
    with z (log-depth, or depth for the orthographic reading, [H, W], NaN
    invalid), depth (exp(z) for perspective), labels0/K0 after seeding, the
    final labels/K, the energies E_1..E_t and the iteration count.
    workers = 0 fills all components in one block-diagonal solve
    (`fill_components`); workers >= 1 fills them one by one on their crops
    (`fill_components_by_crops`) in that many processes."""
    if isinstance(cam, dict):
        cam = Camera.from_dict(cam)
    if isinstance(params, dict):
        params = Params.from_dict(params)
    mask = np.asarray(mask).astype(np.uint8)
    H, W = mask.shape
    labels, K = seed_components(normals, mask, params.theta_c_deg, params.connectivity)
    if workers >= 1:
        zt, fill_iters = fill_components_by_crops(normals, mask, cam, labels, K, params.k, params.n_fill_irls,
                                                  params.connectivity, workers, residual=params.bini_residual)
    geo = geometry(normals, mask, cam, params.connectivity)
    if workers < 1:
        zt, fill_iters = fill_components(geo, labels, K, params.k, params.n_fill_irls, params.bini_residual)
    r = scale_loop(geo, labels, K, zt, params, record)
    out = r["z"].reshape(H, W)
    depth = np.exp(out) if cam.camera == PERSP else out
    r.update(z=out, depth=depth, z_fill=zt.reshape(H, W), labels0=labels.reshape(H, W), K0=K,
             labels=r["labels"].reshape(H, W), fill_iters=fill_iters)
    return r


# ---------------------------------------------------------------------------
# evaluation helpers (alignment of Sec. 4: each island of the mask up to its own scale or offset)
# ---------------------------------------------------------------------------

def islands(mask, conn=4):
    """Connected components of the valid-pixel graph G_0."""
    H, W = mask.shape
    a, b, _ = edge_list(mask, conn)
    vidx = np.nonzero(mask.reshape(-1))[0]
    lab, n = canonical_labels(H * W, vidx, a, b)
    out = np.full(H * W, -1, np.int64)
    out[vidx] = lab
    return out.reshape(H, W), n


def aligned_rel_rmse(z, z_ref, mask, camera, conn=4):
    """Relative depth RMSE of `z` against `z_ref` after the alignment the
    comparison needs, island by island (each island of the mask is
    reconstructed up to its own scale/offset):
      perspective: scale s* = <z, z_ref>/<z, z> per island, error / RMS(z_ref);
      orthographic: offset o* = mean(z_ref - z) per island, error / (max - min)(z_ref)."""
    isl, n = islands(mask, conn)
    m = isl >= 0
    z = np.asarray(z, np.float64)
    zr = np.asarray(z_ref, np.float64)
    al = np.zeros_like(zr)
    for i in range(n):
        s = isl == i
        if camera == PERSP:
            den = np.sum(z[s] * z[s])
            al[s] = z[s] * (np.sum(z[s] * zr[s]) / den if den > 0 else 1.0)
        else:
            al[s] = z[s] + np.mean(zr[s] - z[s])
    err = np.sqrt(np.mean((al[m] - zr[m]) ** 2))
    if camera == PERSP:
        return float(err / np.sqrt(np.mean(zr[m] ** 2)))
    return float(err / max(np.ptp(zr[m]), 1e-300))


def min_made(depth, depth_gt, labels, K, camera):
    """Minimum theoretical mean absolute depth error of a decomposition
    (supplementary material, the section on the components found for different
    theta_c): the MADE the reconstruction would reach with the best scale of
    each component, i.e. the per-component minimal MADEs weighted by their
    pixel counts.

    depth: [H, W] depth of the reconstruction (exp(z~) for the perspective
    camera, z~ for the orthographic reading), depth_gt: [H, W], labels:
    [H, W] component of each pixel (-1 excluded) or None for one component of
    all pixels (then K = 1: the MADE after the best global scale).  A pixel
    counts if its label is >= 0 and both depths are finite (and positive for
    the perspective camera).

    Reading: the paper gives no formula.  A component's scale multiplies its
    depth for the perspective camera (it adds to the log-depth) and adds to the
    depth for the orthographic reading, whose components are fixed up to an
    offset.  Per component
        E_c = min_s sum_{i in c} |s d_i - g_i|   (perspective)
        E_c = min_s sum_{i in c} |d_i + s - g_i| (orthographic)
    and MADE = sum_c E_c / sum_c n_c.  E_c is a convex piecewise-linear
    function of s whose minimum lies where its slope changes sign: at a
    median of r_i = g_i / d_i weighted by d_i (perspective: |s d - g| =
    d |s - r|), or at a median of r_i = g_i - d_i (orthographic).

    Returns (made, per-component MADE E_c / n_c [K] (0 if n_c = 0),
    per-component minimiser s_c [K] (NaN if n_c = 0)); made is NaN when no
    pixel counts.  Parity pinned by tests/test_made_pins.py (closed forms,
    brute force over the breakpoints, invariance, coarsening)."""
    d = np.asarray(depth, np.float64).reshape(-1)
    g = np.asarray(depth_gt, np.float64).reshape(-1)
    if labels is None:
        lab = np.zeros(d.size, np.int64)
        K = 1
    else:
        lab = np.asarray(labels).reshape(-1).astype(np.int64)
    ok = (lab >= 0) & np.isfinite(d) & np.isfinite(g)
    if camera == PERSP:
        ok &= (d > 0) & (g > 0)
    idx = np.nonzero(ok)[0]
    idx = idx[np.argsort(lab[idx], kind="stable")]
    bounds = np.searchsorted(lab[idx], np.arange(K + 1))
    err = np.zeros(K)
    cnt = np.zeros(K, np.int64)
    scale = np.full(K, np.nan)
    for c in range(K):
        sel = idx[bounds[c]:bounds[c + 1]]
        if sel.size == 0:
            continue
        dc, gc = d[sel], g[sel]
        if camera == PERSP:
            r, w = gc / dc, dc
        else:
            r, w = gc - dc, np.ones_like(dc)
        o = np.argsort(r, kind="stable")
        cw = np.cumsum(w[o])
        s = r[o][np.searchsorted(cw, 0.5 * cw[-1], side="left")]
        e = np.abs(s * dc - gc) if camera == PERSP else np.abs(dc + s - gc)
        err[c] = e.sum()
        cnt[c] = sel.size
        scale[c] = s
    n = int(cnt.sum())
    made = float(err.sum() / n) if n > 0 else float("nan")
    per = np.where(cnt > 0, err / np.maximum(cnt, 1), 0.0)
    return made, per, scale
