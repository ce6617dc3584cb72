"""Relative-scale loop (Sec. 3.4, Eqs. 12-14, 11) without merging: the GPU
log-depth after a fixed number of iterations against the oracle's, and the
energies E_t."""
import numpy as np
import pytest

import oracle as O
from synth import make_workload

from gpu_util import PIXEL_TOL, dev, integrator, rel_depth_error, rel_depth_max

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,T", [("c1", 6), ("c2", 8), ("c3_small", 8), ("c3", 6)])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_scale_loop_matches_oracle(name, T, use_graph):
    w = make_workload(name)
    p = dict(w.params, T=T, dE_max=0.0, can_merge=False)
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, p, use_graph=use_graph)
    it.seed_components(n, m)
    it.solve_components()
    k, E, z = it.solve_scales(T)
    assert k == T
    ref = O.integrate(w.normals, w.mask, w.camera, O.Params.from_dict(p))
    zr = np.nan_to_num(ref["z"])
    err = rel_depth_error(z.cpu().numpy(), zr, w.mask, w.camera["camera"])
    mx = rel_depth_max(z.cpu().numpy(), zr, w.mask, w.camera["camera"])
    print(name, "graph", use_graph, "rel depth err", err, "max", mx, "E gpu", E[:4], "E ref", ref["energies"][:4])
    assert err <= 1e-4
    assert mx <= PIXEL_TOL
    np.testing.assert_allclose(E, ref["energies"], rtol=5e-3, atol=1e-9 * max(ref["energies"]))


def test_scale_loop_split_calls_equal_one_call():
    w = make_workload("c2")
    p = dict(w.params, T=6, dE_max=0.0)
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    outs = []
    for split in ([6], [2, 3, 1]):
        it = integrator(H, W, w.camera, p)
        it.seed_components(n, m)
        it.solve_components()
        for s in split:
            it.solve_scales(s)
        outs.append(it.logdepth().cpu().numpy())
    assert np.max(np.abs(outs[0] - outs[1])) < 1e-6


@pytest.mark.parametrize("name,T", [("c1", 6), ("c2", 6), ("c3_small", 8)])
def test_scale_solver_launches_agree_with_oracle(name, T):
    """Both launches of the relative-scale PCG: one thread-block cluster
    (scale_solver = 1) and one CTA or a cooperative grid (scale_solver = 2;
    c3_small has 26 components, one CTA; c1 has 1600, a grid of 7 CTAs).  Each
    against the oracle, and the two against each other: the fixed-point sums
    make each launch's reductions independent of the order of the terms, but
    the two launches partition the rows differently, so they agree to the
    CG tolerance, not bit for bit."""
    w = make_workload(name)
    p = dict(w.params, T=T, dE_max=0.0, can_merge=False)
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    ref = O.integrate(w.normals, w.mask, w.camera, O.Params.from_dict(p))
    zr = np.nan_to_num(ref["z"])
    zs = []
    for solver in (1, 2):
        it = integrator(H, W, w.camera, p, scale_solver=solver)
        it.seed_components(n, m)
        it.solve_components()
        k, E, z = it.solve_scales(T)
        it.close()
        assert k == T
        z = z.cpu().numpy()
        err = rel_depth_error(z, zr, w.mask, w.camera["camera"])
        mx = rel_depth_max(z, zr, w.mask, w.camera["camera"])
        print(name, "scale_solver", solver, "rel depth err", err, "max", mx)
        assert err <= 1e-4 and mx <= PIXEL_TOL
        np.testing.assert_allclose(E, ref["energies"], rtol=5e-3, atol=1e-9 * max(ref["energies"]))
        zs.append(z)
    assert rel_depth_error(zs[0], zs[1], w.mask, w.camera["camera"]) <= 1e-5
