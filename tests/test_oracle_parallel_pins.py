"""Pins of the oracle's large-map paths against its plain block-diagonal solve.

* `cg_min_norm` (the CG the paper names, Eq. 10, used for blocks too large for
  the sparse LU) against the pseudo-inverse on a small Laplacian and against
  the LU solve of every fill block of C1, C2 and C3-small;
* `fill_components_by_crops` (components filled one by one on their crops, in
  parallel processes, as the paper fills them) against `fill_components`
  (one block-diagonal solve of the whole map);
* `integrate(..., workers=2)` against `integrate(...)` end to end.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import oracle.ni_oracle as NO
from synth import make_workload


def _fill_inputs(name):
    w = make_workload(name)
    p = O.Params.from_dict(w.params)
    cam = O.Camera.from_dict(w.camera)
    lab, K = O.seed_components(w.normals, w.mask, p.theta_c_deg)
    return w, p, cam, lab, K


def test_cg_min_norm_against_pseudo_inverse():
    rng = np.random.default_rng(5)
    n = 40
    rows, cols, vals = [], [], []
    for i in range(n - 1):                       # a path keeps the block connected
        wgt = rng.uniform(1e-2, 10.0)
        rows += [i, i + 1, i, i + 1]; cols += [i, i + 1, i + 1, i]; vals += [wgt, wgt, -wgt, -wgt]
    for _ in range(60):
        i, j = rng.integers(0, n, 2)
        if i != j:
            wgt = rng.uniform(1e-2, 10.0)
            rows += [i, j, i, j]; cols += [i, j, j, i]; vals += [wgt, wgt, -wgt, -wgt]
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    g = rng.normal(size=n)
    x, its = O.cg_min_norm(M, g)
    ref = np.linalg.pinv(M.toarray()) @ g          # minimum norm: the range part of g
    np.testing.assert_allclose(x, ref, atol=1e-10 * max(1.0, np.abs(ref).max()))
    assert 0 < its <= 20 * n


@pytest.mark.parametrize("name", ["c1", "c2", "c3_small"])
def test_cg_blocks_match_lu_blocks(name, monkeypatch):
    w, p, cam, lab, K = _fill_inputs(name)
    geo = O.geometry(w.normals, w.mask, cam)
    z_lu, _ = O.fill_components(geo, lab, K, p.k, p.n_fill_irls)
    monkeypatch.setattr(NO, "LU_MAX_NODES", 50)     # every block of more than 50 pixels by CG
    z_cg, _ = O.fill_components(geo, lab, K, p.k, p.n_fill_irls)
    v = w.mask.reshape(-1) > 0
    np.testing.assert_allclose(z_cg[v], z_lu[v], rtol=0, atol=1e-10 * max(1.0, np.abs(z_lu[v]).max()))


@pytest.mark.parametrize("name,workers", [("c2", 1), ("c3_small", 1), ("c1", 2)])
def test_fill_by_crops_equals_block_diagonal_fill(name, workers):
    w, p, cam, lab, K = _fill_inputs(name)
    geo = O.geometry(w.normals, w.mask, cam)
    z0, _ = O.fill_components(geo, lab, K, p.k, p.n_fill_irls)
    z1, _ = O.fill_components_by_crops(w.normals, w.mask, cam, lab, K, p.k, p.n_fill_irls, 4, workers,
                                       task_px=4096)
    v = w.mask.reshape(-1) > 0
    assert np.array_equal(np.isnan(z1), ~v)
    np.testing.assert_allclose(z1[v], z0[v], rtol=0, atol=1e-12)


def test_fill_by_crops_with_irls_sweeps_and_8_connectivity():
    w, p, cam, _, _ = _fill_inputs("c3_small")
    lab, K = O.seed_components(w.normals, w.mask, p.theta_c_deg, 8)
    geo = O.geometry(w.normals, w.mask, cam, 8)
    z0, _ = O.fill_components(geo, lab, K, p.k, 2)
    z1, _ = O.fill_components_by_crops(w.normals, w.mask, cam, lab, K, p.k, 2, 8, 1)
    v = w.mask.reshape(-1) > 0
    np.testing.assert_allclose(z1[v], z0[v], rtol=0, atol=1e-12)


def test_integrate_with_workers_equals_plain_integrate():
    w = make_workload("c3_small")
    p = O.Params.from_dict(dict(w.params, T=8))
    r0 = O.integrate(w.normals, w.mask, w.camera, p)
    r1 = O.integrate(w.normals, w.mask, w.camera, p, workers=2)
    assert (r0["K0"], r0["K"], r0["iters"]) == (r1["K0"], r1["K"], r1["iters"])
    np.testing.assert_array_equal(r0["labels"], r1["labels"])
    v = w.mask > 0
    np.testing.assert_allclose(r1["z"][v], r0["z"][v], rtol=0, atol=1e-10)
