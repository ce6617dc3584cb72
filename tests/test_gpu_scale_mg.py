"""The relative-scale PCG with the quotient-graph multigrid preconditioner
(`scale_precond = 1`) against the oracle and against the Jacobi-preconditioned
solve: the same system, tolerance and stop test, so the same log-depth,
energies and merges.  Skipped until it has run on a GPU (the option is off by
default)."""
import numpy as np
import pytest

import oracle as O
from synth import make_workload

from gpu_util import dev, integrator, rel_depth_error

pytestmark = [pytest.mark.gpu,
              pytest.mark.skip(reason="scale_precond = 1 has not yet run on a GPU")]


@pytest.mark.parametrize("name,T", [("c1", 6), ("c2", 8), ("c3_small", 8), ("c5_small", 6)])
def test_scale_loop_multigrid_matches_oracle(name, T):
    w = make_workload(name)
    p = dict(w.params, T=T, dE_max=0.0, can_merge=False)
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    it = integrator(H, W, w.camera, p, scale_precond=1)
    it.seed_components(n, m)
    it.solve_components()
    k, E, z = it.solve_scales(T)
    assert k == T
    ref = O.integrate(w.normals, w.mask, w.camera, O.Params.from_dict(p))
    err = rel_depth_error(z.cpu().numpy(), np.nan_to_num(ref["z"]), w.mask, w.camera["camera"])
    print(name, "rel depth err", err)
    assert err <= 1e-4
    np.testing.assert_allclose(E, ref["energies"], rtol=5e-3, atol=1e-9 * max(ref["energies"]))


@pytest.mark.parametrize("name", ["c1", "c2", "c3_small"])
def test_integrate_multigrid_equals_jacobi(name):
    """End to end with merging: labels identical, depth within the tolerance,
    and far fewer scale PCG iterations."""
    w = make_workload(name)
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    outs = []
    for sp in (0, 1):
        it = integrator(H, W, w.camera, w.params, scale_precond=sp)
        depth, labels, st = it.integrate(n, m)
        outs.append((depth.cpu().numpy(), labels.cpu().numpy(), st))
    (d0, l0, s0), (d1, l1, s1) = outs
    print(name, "scale PCG iterations (max per solve): Jacobi", s0["scale_cg_iters"], "multigrid", s1["scale_cg_iters"],
          "ms_scale", s0["ms_scale"], s1["ms_scale"])
    np.testing.assert_array_equal(l0, l1)
    z0 = np.log(d0) if w.camera["camera"] == 1 else d0
    z1 = np.log(d1) if w.camera["camera"] == 1 else d1
    assert rel_depth_error(np.nan_to_num(z1), np.nan_to_num(z0), w.mask, w.camera["camera"]) <= 1e-4
    assert s1["scale_cg_iters"] < s0["scale_cg_iters"]
