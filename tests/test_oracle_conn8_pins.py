"""Pins of the oracle's 8-connectivity (the pixel graph of the paper's DiLiGenT
experiments and of its connectivity ablation in the supplementary material):
diagonal edges enter the seeding, the fill, the scale loop and the merge.

Each test ties the 8-connected oracle to something other than itself: a
brute-force enumeration of the graph, closed forms on planes (Eq. 3 is exact
for any two rays of a plane), second-order convergence on a sphere, dense
least squares assembled row by row, a breadth-first flood fill, and a
brute-force merge.  CPU only."""
import math
from collections import deque

import numpy as np
import pytest

import oracle as O
from synth import generators as G

KING = ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1))


def _cam(d):
    return O.Camera.from_dict(d)


def test_edge_list_is_every_king_move_pair():
    rng = np.random.default_rng(0)
    H, W = 9, 11
    mask = (rng.random((H, W)) > 0.25).astype(np.uint8)
    a, b, d = O.edge_list(mask, 8)
    got = {(min(x, y), max(x, y)) for x, y in zip(a.tolist(), b.tolist())}
    ref = set()
    for v in range(H):
        for u in range(W):
            if not mask[v, u]:
                continue
            for du, dv in KING:
                uu, vv = u + du, v + dv
                if 0 <= uu < W and 0 <= vv < H and mask[vv, uu]:
                    p, q = v * W + u, vv * W + uu
                    ref.add((min(p, q), max(p, q)))
    assert got == ref and len(a) == len(ref)
    # b = a + step(dir), ids 4 a + dir strictly increasing
    np.testing.assert_array_equal(b - a, O.STEP_U[d] + O.STEP_V[d] * W)
    ids = O.edge_id(a, d, 8)
    assert np.all(np.diff(ids) > 0)
    # the 4-connected list is the dir 0/1 part with ids 2 a + dir
    a4, b4, d4 = O.edge_list(mask, 4)
    sel = d < 2
    np.testing.assert_array_equal(a4, a[sel])
    np.testing.assert_array_equal(b4, b[sel])


@pytest.mark.parametrize("normal", [(0.2, -0.1, -1.0), (-0.4, 0.3, -0.8)])
def test_omega_exact_on_perspective_plane_diagonals(normal):
    nrm, mask, z, cam = G.plane_map(9, 11, G.PERSP, normal=normal, d=50.0)
    a, b, d = O.edge_list(mask, 8)
    assert (d >= 2).sum() > 0
    om = O.omega(nrm, _cam(cam), 9, 11, a, b, d)
    zz = z.reshape(-1)
    np.testing.assert_allclose(om, np.log(zz[a]) - np.log(zz[b]), rtol=0, atol=1e-12)


def test_omega_exact_on_orthographic_plane_diagonals():
    nrm, mask, z, cam = G.plane_map(7, 8, G.ORTHO, normal=(0.3, -0.2), d=5.0)
    a, b, d = O.edge_list(mask, 8)
    om = O.omega(nrm, _cam(cam), 7, 8, a, b, d)
    zz = z.reshape(-1)
    np.testing.assert_allclose(om, zz[a] - zz[b], atol=1e-12)
    np.testing.assert_allclose(O.omega(nrm, _cam(cam), 7, 8, b, a, d), -om, atol=1e-12)


def test_gamma_on_diagonals_with_equal_focal_lengths():
    """With f_x = f_y every reading of "the focal length" agrees: the diagonal
    gamma equals the axis gamma of the same pixel, -f d / z on the plane
    n.X = -d."""
    nrm, mask, z, cam = G.plane_map(5, 6, G.PERSP, normal=(0.1, 0.2, -1.0), d=40.0)
    c = _cam(cam)
    assert c.fx == c.fy
    a, b, d = O.edge_list(mask, 8)
    g = O.gamma(nrm, c, 5, 6, a, d)
    np.testing.assert_allclose(g, -c.fx * 40.0 / z.reshape(-1)[a], rtol=1e-12)


def test_bini_weight_diagonal_opposite_neighbour():
    """The opposite neighbour of a along a diagonal edge (a, b) is a - (b - a)."""
    H, W = 3, 3
    valid = np.ones(9, bool)
    gam = np.array([3.0])
    a = np.array([4])
    for b_, opp in ((8, 0), (0, 8), (6, 2), (2, 6)):     # down-right, up-left, down-left, up-right
        d = np.array([O.DOWN_RIGHT if abs(b_ - 4) == W + 1 else O.DOWN_LEFT])
        z = np.zeros(9)
        z[b_] = 5.0                                   # jump towards b, smooth towards -b
        assert O.bini_weight(z, gam, a, np.array([b_]), d, H, W, valid, 2.0)[0] / 9.0 < 1e-6
        z = np.zeros(9)
        z[opp] = 5.0                                  # jump on the opposite side: the edge is trusted
        assert O.bini_weight(z, gam, a, np.array([b_]), d, H, W, valid, 2.0)[0] / 9.0 > 1 - 1e-6
    # corner pixel: -b outside the image -> squared difference 0
    z = np.zeros(9)
    z[4] = 1.0
    w = O.bini_weight(z, gam, np.array([0]), np.array([4]), np.array([O.DOWN_RIGHT]), H, W, valid, 2.0)[0]
    assert w / 9.0 == pytest.approx(1.0 / (1.0 + math.exp(2.0 * 9.0)))


def _flood_fill_8(normals, mask, theta):
    H, W = mask.shape
    n = normals.reshape(-1, 4).astype(np.float64)
    c = math.cos(theta * (math.pi / 180.0))
    lab = -np.ones(H * W, int)
    nxt = 0
    m = mask.reshape(-1)
    for s in range(H * W):
        if not m[s] or lab[s] >= 0:
            continue
        lab[s] = nxt
        dq = deque([s])
        while dq:
            p = dq.popleft()
            u, v = p % W, p // W
            for du, dv in KING:
                uu, vv = u + du, v + dv
                if 0 <= uu < W and 0 <= vv < H:
                    q = vv * W + uu
                    if m[q] and lab[q] < 0 and n[p, 0] * n[q, 0] + n[p, 1] * n[q, 1] + n[p, 2] * n[q, 2] > c:
                        lab[q] = nxt
                        dq.append(q)
        nxt += 1
    return lab, nxt


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_seeding_8_matches_flood_fill(seed):
    H, W = 30, 27
    nrm, mask, cam = G.random_normal_field(H, W, n_dirs=3, jitter_deg=1.5, hole_frac=0.3, seed=seed)
    lab, K = O.seed_components(nrm, mask, 2.5, 8)
    ref, Kr = _flood_fill_8(nrm, mask, 2.5)
    assert K == Kr
    np.testing.assert_array_equal(lab, ref)
    _, K4 = O.seed_components(nrm, mask, 2.5, 4)
    assert K <= K4


def _align_max(z, zref, mask, conn):
    isl, n = O.islands(mask, conn)
    z = z.reshape(mask.shape)
    zr = zref.reshape(mask.shape)
    return max(np.max(np.abs((z[isl == i] - z[isl == i].mean()) - (zr[isl == i] - zr[isl == i].mean())))
               for i in range(n))


@pytest.mark.parametrize("camera", [G.PERSP, G.ORTHO])
def test_fill_8_exact_on_plane_with_islands(camera):
    H, W = 12, 12
    mask = np.ones((H, W), np.uint8)
    mask[:, 5] = 0
    mask[3, 8] = 0
    mask[7, 9] = 0
    nrm, mask, z, cam = G.plane_map(H, W, camera, normal=(0.3, -0.2, -1.0) if camera else (0.3, -0.2),
                                    d=30.0, mask=mask)
    geo = O.geometry(nrm, mask, _cam(cam), 8)
    lab, K = O.seed_components(nrm, mask, 5.0, 8)
    assert K == 2
    zt, _ = O.fill_components(geo, lab, K)
    zref = np.log(z) if camera == G.PERSP else z
    assert _align_max(zt, zref, mask, 8) < 1e-10


def test_fill_8_second_order_on_sphere():
    errs = []
    for n in (32, 64, 128):
        nrm, mask, z, cam = G.sphere_map(n)
        geo = O.geometry(nrm, mask, _cam(cam), 8)
        lab, K = O.seed_components(nrm, mask, 90.0, 8)
        assert K == 1
        zt, _ = O.fill_components(geo, lab, K)
        errs.append(O.aligned_rel_rmse(np.exp(zt.reshape(n, n)), z, mask, G.PERSP, 8))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.6 < s < 2.4 for s in slopes), (errs, slopes)


def _dense_min_norm(rows, rhs, w, n):
    A = np.zeros((len(rows), n))
    for r, (i, j) in enumerate(rows):
        A[r, i] += 1.0
        A[r, j] -= 1.0
    sw = np.sqrt(w)
    x, *_ = np.linalg.lstsq(A * sw[:, None], rhs * sw, rcond=None)
    return x


def test_fill_8_matches_dense_least_squares():
    H, W = 10, 12
    nrm, mask, cam = G.random_normal_field(H, W, n_dirs=2, jitter_deg=2.0, hole_frac=0.1, seed=4, block=5)
    geo = O.geometry(nrm, mask, _cam(cam), 8)
    lab, K = O.seed_components(nrm, mask, 4.0, 8)
    zt, _ = O.fill_components(geo, lab, K)
    assert (geo.d >= 2).any()
    for comp in range(K):
        pix = np.nonzero(lab == comp)[0]
        if len(pix) < 2:
            continue
        pos = {p: i for i, p in enumerate(pix)}
        rows, rhs, w = [], [], []
        for e in range(len(geo.a)):
            a, b = geo.a[e], geo.b[e]
            if lab[a] == comp and lab[b] == comp:
                rows.append((pos[a], pos[b])); rhs.append(geo.omega[e]); w.append(0.5 * geo.gam_ba[e] ** 2)
                rows.append((pos[b], pos[a])); rhs.append(-geo.omega[e]); w.append(0.5 * geo.gam_ab[e] ** 2)
        x = _dense_min_norm(rows, np.array(rhs), np.array(w), len(pix))
        np.testing.assert_allclose(zt[pix], x - x.mean(), atol=1e-9)


def _small_problem_8(seed, theta=4.0):
    nrm, mask, cam = G.random_normal_field(11, 12, n_dirs=3, jitter_deg=2.0, hole_frac=0.05, seed=seed, block=4)
    geo = O.geometry(nrm, mask, _cam(cam), 8)
    lab, K = O.seed_components(nrm, mask, theta, 8)
    zt, _ = O.fill_components(geo, lab, K)
    return nrm, mask, geo, lab, K, np.nan_to_num(zt)


@pytest.mark.parametrize("t", [0, 2])
def test_scale_solve_8_matches_dense_least_squares(t):
    nrm, mask, geo, lab, K, zt = _small_problem_8(1)
    A, rhs, w, e = O.scale_system(geo, lab, K, zt, t, O.Params(connectivity=8))
    assert (geo.d[e] >= 2).any()
    qcc, nq = O.quotient_components(K, lab, geo, e)
    s, _ = O.solve_scales(A, rhs, w, K, qcc, nq)
    rows = []
    for i in e:
        pa, pb = lab[geo.a[i]], lab[geo.b[i]]
        rows.append((pa, pb)); rows.append((pb, pa))
    x = _dense_min_norm(rows, rhs, w, K)
    np.testing.assert_allclose(s, x, atol=1e-8 * max(1, np.abs(x).max()))


def test_pixel_level_limit_8_first_iteration_is_global_least_squares():
    H, W = 8, 8
    nrm, mask, cam = G.random_normal_field(H, W, n_dirs=2, jitter_deg=3.0, hole_frac=0.0, seed=11)
    geo = O.geometry(nrm, mask, _cam(cam), 8)
    lab, K = O.seed_components(nrm, mask, None, 8)
    zt, _ = O.fill_components(geo, lab, K)
    r = O.scale_loop(geo, lab, K, zt, O.Params(T=1, connectivity=8))
    rows, rhs = [], []
    for v in range(H):
        for u in range(W):
            for du, dv in ((1, 0), (0, 1), (1, 1), (-1, 1)):
                uu, vv = u + du, v + dv
                if 0 <= uu < W and vv < H:
                    p, q = v * W + u, vv * W + uu
                    e = np.nonzero((geo.a == p) & (geo.b == q))[0][0]
                    rows.append((p, q)); rhs.append(geo.omega[e])
                    rows.append((q, p)); rhs.append(-geo.omega[e])
    assert len(rows) == 2 * len(geo.a)
    x = _dense_min_norm(rows, np.array(rhs), np.ones(len(rows)), H * W)
    np.testing.assert_allclose(r["z"], x - x.mean(), atol=1e-9)


def _brute_merge_8(lab, K, geo, e, chi32):
    best = {}
    for j, i in enumerate(e):
        a, b = geo.a[i], geo.b[i]
        key = (float(chi32[j]), 4 * int(a) + int(geo.d[i]))
        for cmp_ in (lab[a], lab[b]):
            if cmp_ not in best or key < best[cmp_][0]:
                best[cmp_] = (key, (lab[a], lab[b]))
    parent = list(range(K))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x
    for _, (x, y) in best.values():
        rx, ry = find(x), find(y)
        if rx != ry:
            parent[max(rx, ry)] = min(rx, ry)
    roots = sorted({find(c) for c in range(K)})
    rank = {r: i for i, r in enumerate(roots)}
    new = np.array([rank[find(c)] for c in range(K)])
    out = lab.copy()
    out[lab >= 0] = new[lab[lab >= 0]]
    return out, len(roots)


@pytest.mark.parametrize("seed", [0, 4, 9])
def test_merge_8_matches_brute_force(seed):
    nrm, mask, geo, lab, K, zt = _small_problem_8(seed, theta=2.0)
    e = O.inter_edges(geo, lab)
    rng = np.random.default_rng(seed)
    chi = np.abs(rng.normal(0, 1e-3, len(e))).astype(np.float32)
    chi[::5] = chi[0]                # planted ties, broken by the 8-connected edge id
    new, Kn, sel = O.merge_labels(lab, K, geo, e, chi)
    ref, Kr = _brute_merge_8(lab, K, geo, e, chi)
    assert Kn == Kr
    np.testing.assert_array_equal(new, ref)


@pytest.mark.parametrize("camera", [G.PERSP, G.ORTHO])
def test_plane_split_8_is_reassembled_exactly(camera):
    nrm, mask, z, cam = G.plane_map(6, 7, camera, normal=(0.25, 0.1, -1.0) if camera else (0.25, 0.1), d=20.0)
    r = O.integrate(nrm, mask, cam, O.Params(theta_c_deg=None, T=4, dE_max=0.0, connectivity=8))
    zref = np.log(z) if camera == G.PERSP else z
    assert _align_max(np.nan_to_num(r["z"]).reshape(-1), zref.reshape(-1), mask, 8) < 1e-9
