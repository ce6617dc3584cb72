"""Hand-worked pins of the discontinuity-aware weights of the oracle.

* `scale_system` at t >= 2 (Sec. 3.4, Eq. 13 with the weights of Eqs. 5 and
  11): every row of a 3-component 3x4 map is written out here, edge by edge,
  from per-pixel quantities (gamma of the row's own pixel, the opposite
  neighbour of that pixel, W^out of the edge's residual) and compared with the
  oracle's (A, rhs, w) element by element.  Swapping gamma_{b->a} and
  gamma_{a->b} between the two rows of an edge, taking the opposite neighbour
  on the wrong side, or dropping W^out from one of the rows fails here.
* `bini_weight(..., same_component=...)` (Sec. 3.1, Eqs. 4-5, with the fill's
  reading that an opposite neighbour outside a's component counts as absent).
* the residual-based variant of the BiNI weight: the same rows written out
  with residuals, and closed forms where the model of continuity is exact.
"""
import math

import numpy as np
import pytest

import oracle as O


def _sig(x, k):
    return 1.0 / (1.0 + math.exp(-k * x))


def _wout_plotted(chi):
    """The outlier weight for L = 1e-5, U = 1e-3 in the closed form the paper
    plots for Eq. 11 (Fig. 7): 1 / (1 + exp(2 (2 x + 8))), x = log10 |chi|."""
    x = math.log10(max(abs(chi), 1e-30))
    return 1.0 / (1.0 + math.exp(2.0 * (2.0 * x + 8.0)))


def _map_3x4(seed):
    """3 rows x 4 columns, perspective, f_x != f_y, one invalid pixel.
    Components (hand-assigned, -1 invalid):
        0 0 1 1
        0 0 1 1
        2 2 2 -1
    """
    H, W = 3, 4
    rng = np.random.default_rng(seed)
    n = np.zeros((H, W, 4), np.float32)
    g = np.stack([rng.uniform(-0.3, 0.3, (H, W)), rng.uniform(-0.3, 0.3, (H, W)), -np.ones((H, W))], -1)
    g /= np.linalg.norm(g, axis=-1, keepdims=True)
    n[..., :3] = g
    mask = np.ones((H, W), np.uint8)
    mask[2, 3] = 0
    labels = np.array([[0, 0, 1, 1], [0, 0, 1, 1], [2, 2, 2, -1]], np.int64).reshape(-1)
    cam = O.Camera(O.PERSP, 8.0, 6.0, 1.5, 1.0)
    # log-depth: arbitrary values, spread so that W^out and the BiNI sigmoid
    # take values well inside (0, 1) on some edges
    zt = rng.normal(0.0, 0.03, H * W)
    zt[labels < 0] = 0.0
    return H, W, n, mask, labels, cam, zt


def _pix_gamma(n, cam, W, p, horizontal):
    """gamma at pixel p: f n_p . tau_p with tau_p = ((u - c_x)/f_x, (v - c_y)/f_y, 1)
    and f = f_x for a horizontal edge, f_y for a vertical one (Eq. 6)."""
    u, v = p % W, p // W
    nn = n.reshape(-1, 4)[p, :3].astype(np.float64)
    tau = np.array([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, 1.0])
    return (cam.fx if horizontal else cam.fy) * float(nn @ tau)


def _expected_rows(H, W, n, mask, labels, cam, zt, omega_of, k, residual=False):
    """Every inter edge's two rows of Eq. 13 at t >= 2, written out pixel by pixel."""
    valid = mask.reshape(-1) > 0

    def z_at(p, ok):
        return zt[p] if ok else None

    rows = {}
    for v in range(H):
        for u in range(W):
            a = v * W + u
            for du, dv in ((1, 0), (0, 1)):
                ub, vb = u + du, v + dv
                if ub >= W or vb >= H:
                    continue
                b = vb * W + ub
                if not (valid[a] and valid[b]) or labels[a] == labels[b]:
                    continue
                horizontal = du == 1
                om = omega_of(a, b)                       # w~_{b->a}
                chi = zt[a] - zt[b] - om                  # Eq. 4's residual of the edge
                wo = _wout_plotted(chi)
                # row (b->a): the BiNI weight of pixel a, its opposite neighbour a - (b - a)
                uo, vo = u - du, v - dv
                ok = 0 <= uo < W and 0 <= vo < H and valid[vo * W + uo]
                ga = _pix_gamma(n, cam, W, a, horizontal)
                if residual:   # chi_{c->a} = z_a - z_c - w~_{c->a} on both sides
                    o = vo * W + uo
                    opp = (zt[a] - zt[o] - omega_of(a, o)) ** 2 if ok else 0.0
                    main = chi ** 2
                else:
                    opp = (zt[vo * W + uo] - zt[a]) ** 2 if ok else 0.0
                    main = (zt[b] - zt[a]) ** 2
                w_ba = ga * ga * _sig(ga * ga * (opp - main), k) * wo
                # row (a->b): the BiNI weight of pixel b, its opposite neighbour b + (b - a)
                uo, vo = ub + du, vb + dv
                ok = 0 <= uo < W and 0 <= vo < H and valid[vo * W + uo]
                gb = _pix_gamma(n, cam, W, b, horizontal)
                if residual:   # chi_{a->b} = z_b - z_a - w~_{a->b} = -chi_{b->a}
                    o = vo * W + uo
                    opp = (zt[b] - zt[o] - omega_of(b, o)) ** 2 if ok else 0.0
                    main = chi ** 2
                else:
                    opp = (zt[vo * W + uo] - zt[b]) ** 2 if ok else 0.0
                    main = (zt[a] - zt[b]) ** 2
                w_ab = gb * gb * _sig(gb * gb * (opp - main), k) * wo
                ca, cb = labels[a], labels[b]
                rows[(a, b)] = (
                    # (+1 at pi(a), -1 at pi(b), rhs w~_{b->a} - (z~_a - z~_b), weight)
                    (ca, cb, om - (zt[a] - zt[b]), w_ba),
                    # (+1 at pi(b), -1 at pi(a), rhs w~_{a->b} - (z~_b - z~_a), weight)
                    (cb, ca, -om - (zt[b] - zt[a]), w_ab),
                )
    return rows


@pytest.mark.parametrize("seed,k,residual", [(0, 2.0, False), (1, 2.0, False), (2, 1.0, False),
                                             (0, 2.0, True), (3, 1.0, True)])
def test_scale_rows_at_t2_written_out_by_hand(seed, k, residual):
    H, W, n, mask, labels, cam, zt = _map_3x4(seed)
    geo = O.geometry(n, mask, cam)
    K = 3
    p = O.Params(k=k, bini_residual=residual)
    A, rhs, w, e = O.scale_system(geo, labels, K, zt, 2, p)
    # w~_{c->a} of any neighbouring pair, from the oracle's Eq. 3 (pinned on planes)
    om_map = {(int(geo.a[i]), int(geo.b[i])): float(geo.omega[i]) for i in range(len(geo.a))}

    def omega_of(a, c):
        return om_map[(a, c)] if (a, c) in om_map else -om_map[(c, a)]
    exp_rows = _expected_rows(H, W, n, mask, labels, cam, zt, omega_of, k, residual)
    # the hand enumeration: 5 inter edges (2 horizontal, 3 vertical)
    assert sorted(exp_rows) == sorted((int(geo.a[i]), int(geo.b[i])) for i in e)
    assert len(exp_rows) == 5
    Ad = A.toarray()
    assert Ad.shape == (2 * len(e), K)
    for j, i in enumerate(e):
        key = (int(geo.a[i]), int(geo.b[i]))
        for r, (cp, cm, rh, wt) in zip((2 * j, 2 * j + 1), exp_rows[key]):
            row = np.zeros(K)
            row[cp] += 1.0
            row[cm] -= 1.0
            np.testing.assert_array_equal(Ad[r], row)
            assert rhs[r] == pytest.approx(rh, rel=1e-12, abs=1e-15)
            assert w[r] == pytest.approx(wt, rel=1e-10, abs=1e-300)
    # the two rows of an edge carry different gammas: the pin sees a swap
    assert np.all(np.abs(w[0::2] - w[1::2]) > 1e-6 * np.maximum(w[0::2], w[1::2]))


def test_scale_rows_at_t1_are_uniform():
    H, W, n, mask, labels, cam, zt = _map_3x4(0)
    geo = O.geometry(n, mask, cam)
    A, rhs, w, e = O.scale_system(geo, labels, 3, zt, 1, O.Params())
    np.testing.assert_array_equal(w, np.ones(2 * len(e)))


def test_bini_weight_opposite_neighbour_in_another_component():
    """During the fill the opposite neighbour -b counts only inside a's
    component (the fill's reading of Eq. 4): with -b valid but in another
    component, its squared difference is taken as 0."""
    H, W = 1, 5
    valid = np.ones(5, bool)
    a, b, d = np.array([2]), np.array([3]), np.array([0])
    gam = np.array([3.0])
    z = np.array([0.0, 5.0, 0.0, 0.5, 0.0])     # -b = pixel 1, far from a; b close to a
    comp_same = np.array([0, 0, 0, 0, 0])
    comp_other = np.array([0, 1, 0, 0, 0])       # pixel 1 in another component
    # -b counted: x = 9 (25 - 0.25) >> 0, the edge is trusted
    w_same = O.bini_weight(z, gam, a, b, d, H, W, valid, 2.0, comp_same)[0]
    assert w_same == pytest.approx(9.0 * _sig(9.0 * (25.0 - 0.25), 2.0), rel=1e-14)
    # -b in another component: x = 9 (0 - 0.25) = -2.25, W = 9 sigma_2(-2.25)
    w_other = O.bini_weight(z, gam, a, b, d, H, W, valid, 2.0, comp_other)[0]
    assert w_other == pytest.approx(9.0 / (1.0 + math.exp(4.5)), rel=1e-14)
    # without a component map (the scale loop's reading) -b is any valid pixel
    w_any = O.bini_weight(z, gam, a, b, d, H, W, valid, 2.0)[0]
    assert w_any == pytest.approx(w_same, rel=1e-14)
    # the same on a vertical edge, reversed direction: a = 1, b = 0, -b = 2
    z = np.array([0.2, 0.0, 3.0])
    w_v = O.bini_weight(z, gam, np.array([1]), np.array([0]), np.array([1]), 3, 1,
                        np.ones(3, bool), 2.0, np.array([0, 0, 1]))[0]
    assert w_v == pytest.approx(9.0 * _sig(9.0 * (0.0 - 0.04), 2.0), rel=1e-14)


def test_fill_weights_ignore_opposite_neighbours_in_other_components():
    """intra_system passes the labels as the component map: a row whose
    opposite neighbour lies in another component gets gamma^2 sigma_k(-gamma^2
    (z~_b - z~_a)^2), written out here for a 1x4 strip split 0 0 | 1 1."""
    n = np.zeros((1, 4, 4), np.float32)
    n[..., 2] = -1.0
    mask = np.ones((1, 4), np.uint8)
    cam = O.Camera(O.ORTHO, 1.0, 1.0, 0.0, 0.0)
    geo = O.geometry(n, mask, cam)
    labels = np.array([0, 0, 1, 1])
    zt = np.array([0.0, 0.3, 5.0, 5.1])
    A, rhs, w = O.intra_system(geo, labels, zt, 2.0)
    # intra edges (0,1) and (2,3); gamma = n_z = -1 everywhere
    # edge (0,1): row 1->0 at a = 0 has no opposite neighbour (outside);
    #             row 0->1 at b = 1 has opposite neighbour 2, in component 1: ignored
    # edge (2,3): row 3->2 at a = 2 has opposite 1, in component 0: ignored;
    #             row 2->3 at b = 3 has no opposite neighbour (outside)
    exp = [_sig(-0.09, 2.0), _sig(-0.09, 2.0), _sig(-0.01, 2.0), _sig(-0.01, 2.0)]
    np.testing.assert_allclose(w, exp, rtol=1e-14)


def test_residual_bini_weight_is_one_half_where_the_model_is_exact():
    """Where Eq. 3 is exact every residual chi vanishes, so the residual-based
    weight is gamma^2 sigma_k(0) = gamma^2 / 2 on every edge with an opposite
    neighbour, however steep or curved the surface:
      * a perspective plane (Eq. 3 is exact on planes);
      * an orthographic paraboloid z = 0.3 u^2 + 0.2 v^2: the orthographic
        reading of Eq. 3 is the trapezoid rule on the slopes, exact for
        quadratics.  There the raw-difference form is not 1/2: its two sides
        differ by the curvature."""
    from synth import generators as G
    nrm, mask, z, cam = G.plane_map(6, 7, G.PERSP, normal=(0.6, -0.3, -1.0), d=20.0)
    geo = O.geometry(nrm, mask, O.Camera.from_dict(cam))
    zt = np.log(z.reshape(-1))
    w_res = O.bini_weight(zt, geo.gam_ba, geo.a, geo.b, geo.d, 6, 7, geo.valid, 2.0, None, geo.omega_of)
    has = np.where(geo.d == 0, geo.a % 7 > 0, geo.a // 7 > 0)
    np.testing.assert_allclose(w_res[has], 0.5 * geo.gam_ba[has] ** 2, rtol=1e-9)
    # orthographic paraboloid, float64 normals n ~ (-z_u, -z_v, 1)
    H, W = 7, 9
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    zq = 0.3 * u * u + 0.2 * v * v
    g = np.stack([-0.6 * u, -0.4 * v, np.ones_like(u)], -1)
    nq = np.zeros((H, W, 4))
    nq[..., :3] = g / np.linalg.norm(g, axis=-1, keepdims=True)
    geo = O.geometry(nq, np.ones((H, W), np.uint8), O.Camera(O.ORTHO, 1.0, 1.0, 0.0, 0.0))
    zt = zq.reshape(-1)
    w_res = O.bini_weight(zt, geo.gam_ba, geo.a, geo.b, geo.d, H, W, geo.valid, 2.0, None, geo.omega_of)
    w_raw = O.bini_weight(zt, geo.gam_ba, geo.a, geo.b, geo.d, H, W, geo.valid, 2.0)
    has = np.where(geo.d == 0, geo.a % W > 0, geo.a // W > 0)
    half = 0.5 * geo.gam_ba[has] ** 2
    np.testing.assert_allclose(w_res[has], half, rtol=1e-12)
    assert np.max(np.abs(w_raw[has] / half - 1.0)) > 0.5


def test_residual_fill_sweep_on_a_plane_stays_exact():
    """A second fill sweep with residual-based weights keeps a plane exact
    (its residuals are zero, so every weight is gamma^2 / 2 again)."""
    from synth import generators as G
    nrm, mask, z, cam = G.plane_map(9, 8, G.PERSP, normal=(0.3, 0.2, -1.0), d=30.0)
    c = O.Camera.from_dict(cam)
    geo = O.geometry(nrm, mask, c)
    lab, K = O.seed_components(nrm, mask, 5.0)
    z1, _ = O.fill_components(geo, lab, K, 2.0, 1)
    z2, _ = O.fill_components(geo, lab, K, 2.0, 2, residual=True)
    zr = np.log(z.reshape(-1))
    zr = zr - zr.mean()
    np.testing.assert_allclose(z1, zr, atol=1e-10)
    np.testing.assert_allclose(z2, zr, atol=1e-10)
