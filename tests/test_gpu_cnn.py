"""Learned warm start: the BF16 tensor-core network kernels against the FP64
oracle with the same bf16 rounding points, its training loop, its input tiling,
its edge-weight targets, and the warm-started fill against the cold start."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import cnn_oracle as CO
from paper_2510_11508_gb300 import cnn, ni
from synth import make_workload
from synth import generators as G

from gpu_util import dev, integrator

pytestmark = pytest.mark.gpu


def _batch(B=2, T=16, seed=0):
    rng = np.random.default_rng(seed)
    S = T + 2 * CO.HALO
    x = rng.normal(0, 0.5, (B, S, S, 4)).astype(np.float32)
    x[..., 3] = (rng.uniform(size=(B, S, S)) > 0.1)
    tz = rng.normal(0, 1, (B, T, T)).astype(np.float32)
    tl = rng.integers(-1, 3, (B, T, T)).astype(np.int32)
    tw = rng.uniform(0, 1, (B, T, T, 4)).astype(np.float32)
    return x, tz, tl, tw


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_forward_matches_oracle():
    x, *_ = _batch()
    net = cnn.Net(4, 16, seed=1)
    p = net.get_params().astype(np.float64)
    out = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref, _ = CO.forward(p, x.astype(np.float64), quantize=True)
    err = _rel(out, ref)
    print("forward rel err", err)
    assert err < 5e-3


# BF16 keeps 8 significant bits: unit roundoff u = 2^-9.  Every layer rounds
# its input activations and its weights to BF16 (relative error <= u each)
# and accumulates in FP32; a layer's output error is then at most about
# 2 u relative to its output, and the six layers add up to 12 u.
BF16_BUDGET = 12 * 2.0 ** -9


@pytest.mark.parametrize("trained", [False, True])
def test_forward_within_bf16_budget_of_the_fp64_network(trained):
    """The tensor-core network against the unquantised FP64 network (no BF16
    rounding anywhere), on tiles of a synthetic map: relative L2 error within
    the BF16 budget derived above."""
    T = 64
    w = make_workload("c4_train_5")
    net = cnn.Net(8, T, seed=3)
    if trained:
        p32 = np.fromfile(ni.default_net_path(), dtype=np.float32, offset=16)
        net.set_params(p32)
    p = net.get_params().astype(np.float64)
    n, m = dev(w.normals, w.mask)
    tiles = cnn.make_tiles(n, m, T)[:8].contiguous()
    out = net.forward(tiles).cpu().numpy()
    ref, _ = CO.forward(p, tiles.cpu().numpy().astype(np.float64), quantize=False)
    err = _rel(out, ref)
    print("trained" if trained else "random", "forward vs FP64 network rel err", err, "budget", BF16_BUDGET)
    assert err <= BF16_BUDGET


def test_loss_and_gradients_match_oracle():
    x, tz, tl, tw = _batch(seed=1)
    net = cnn.Net(4, 16, seed=2)
    p = net.get_params().astype(np.float64)
    t = [torch.from_numpy(a).cuda() for a in (x, tz, tl, tw)]
    (loss, ld, lw), g = net.loss_grad(*t, w_weight=0.3)
    (rloss, rld, rlw), rg = CO.backward(p, x.astype(np.float64), tz.astype(np.float64), tl, tw.astype(np.float64),
                                        0.3, quantize=True)
    print("loss", loss, rloss, "grad rel err", _rel(g, rg))
    assert abs(loss - rloss) <= 1e-3 * abs(rloss)
    assert _rel(g, rg) < 2e-2
    # per layer (weights and biases of every layer carry gradient)
    o = 0
    for ci, co in CO.LAYERS:
        n = 9 * ci * co + co
        assert _rel(g[o:o + n], rg[o:o + n]) < 5e-2
        o += n


def test_training_reduces_loss():
    x, tz, tl, tw = _batch(B=4, seed=3)
    net = cnn.Net(4, 16, seed=3)
    t = [torch.from_numpy(a).cuda() for a in (x, tz, tl, tw)]
    first = net.train_step(*t, lr=1e-3)[0]
    for _ in range(60):
        last = net.train_step(*t, lr=1e-3)[0]
    assert last < 0.7 * first, (first, last)


def test_make_tiles_halo():
    nrm, mask, cam = G.random_normal_field(40, 37, seed=2)
    n, m = dev(nrm, mask)
    tiles = cnn.make_tiles(n, m, 16).cpu().numpy()
    assert tiles.shape == (9, 28, 28, 4)
    ref = np.zeros((48 + 12 + 12, 48 + 12 + 12, 4), np.float32)
    ref[6:46, 6:43, :3] = np.where(mask[..., None] > 0, nrm[..., :3], 0)
    ref[6:46, 6:43, 3] = mask
    for t in range(9):
        ty, tx = divmod(t, 3)
        np.testing.assert_array_equal(tiles[t], ref[16 * ty:16 * ty + 28, 16 * tx:16 * tx + 28])


def test_edge_targets_match_oracle_bini_weights():
    w = make_workload("c3_small")
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    rng = np.random.default_rng(0)
    z = rng.normal(0, 1e-3, (H, W)).astype(np.float32)
    out = cnn.edge_targets(n, m, torch.from_numpy(z).cuda(), w.camera).cpu().numpy()
    cam = O.Camera.from_dict(w.camera)
    valid = w.mask.reshape(-1).astype(bool)
    zz = z.reshape(-1).astype(np.float64)
    for dirn, (du, dv) in enumerate([(1, 0), (0, 1), (-1, 0), (0, -1)]):
        v, u = np.nonzero(w.mask)
        ub, vb = u + du, v + dv
        ok = (ub >= 0) & (ub < W) & (vb >= 0) & (vb < H)
        a = (v * W + u)[ok]
        b = (vb * W + ub)[ok]
        ok2 = valid[b]
        a, b = a[ok2], b[ok2]
        d = np.full(len(a), 0 if du != 0 else 1)
        gam = O.gamma(w.normals, cam, H, W, a, d)
        ref = O.bini_weight(zz, gam, a, b, d, H, W, valid, 2.0) / (gam * gam)
        got = out.reshape(-1, 4)[a, dirn]
        np.testing.assert_allclose(got, ref, atol=2e-3)


def test_warm_start_gives_the_cold_start_answer(tmp_path):
    w = make_workload("c2")
    H, W = w.mask.shape
    net = cnn.Net(16, 64, seed=5)
    path = str(tmp_path / "net.bin")
    net.save(path)
    n, m = dev(w.normals, w.mask)
    cold = integrator(H, W, w.camera, w.params)
    d0, l0, s0 = cold.integrate(n, m)
    warm = integrator(H, W, w.camera, w.params, warm_start=1)
    warm.load_net(path)
    d1, l1, s1 = warm.integrate(n, m)
    assert np.array_equal(l0.cpu().numpy(), l1.cpu().numpy())
    err = O.aligned_rel_rmse(d1.cpu().numpy(), d0.cpu().numpy(), w.mask, 1)
    print("warm vs cold rel err", err, "iters", s0["fill_iters"], s1["fill_iters"])
    assert err < 1e-4


def test_trained_network_gain(tmp_path):
    """What the trained network gains over the method without it, on held-out
    maps of the training distribution: the network is trained (GPU kernels) on
    C2-type 64x64 maps solved by the plain method, then used as the fill's warm
    start.  Asserted: it learned (validation depth loss well below the trivial
    predictor's), the warm-started solve ends at the cold start's answer, and it
    never costs iterations; the iteration gain is printed."""
    import math
    from paper_2510_11508_gb300 import train_warmstart as TW
    T, n_train, n_eval = 64, 240, 12
    maps = [G.c2_type_map(H=T, W=T, n_cells=4, target_valid=0.5 * T * T, seed=s, name="t")
            for s in range(n_train + n_eval)]
    normals = np.stack([w.normals for w in maps])
    masks = np.stack([w.mask for w in maps])
    cam = G._persp_cam(T, T)
    params = dict(maps[0].params)
    data = TW.solve_targets(normals[:n_train], masks[:n_train], cam, params, torch.device("cuda"))
    zs = 1.0 / math.sqrt(max(TW.zero_predictor_loss(data, 0.0), 1e-30))
    X, TZ, TL, TWt = data
    data = (X, TZ * zs, TL, TWt)
    net = cnn.Net(16, T, seed=1)
    nval = 16
    val = tuple(d[-nval:] for d in data)
    base = TW.zero_predictor_loss(val, 0.0)
    hist = TW.train(net, data, epochs=6, batch=16, lr=2e-3, w_weight=0.1, val_frac=nval / n_train,
                    log=lambda *a: None)
    trained = hist[-1]["val"][1]
    p = net.get_params()
    TW.fold_depth_scale(p, 1.0 / zs)
    net.set_params(p)
    path = str(tmp_path / "net64.bin")
    net.save(path)
    print(f"validation depth loss: trained {trained:.4f} vs zero predictor {base:.4f} (scaled units)")
    assert trained < 0.7 * base
    refs = [O.integrate(w.normals, w.mask, cam, O.Params.from_dict(params)) for w in maps[n_train:]]
    gains = {}
    for pc in (0, 1):
        cold_it, warm_it = [], []
        for w, ref in zip(maps[n_train:], refs):
            n, m = dev(w.normals, w.mask)
            cold = integrator(T, T, cam, params, precond=pc)
            d0, l0, s0 = cold.integrate(n, m)
            warm = integrator(T, T, cam, params, precond=pc, warm_start=1)
            warm.load_net(path)
            d1, l1, s1 = warm.integrate(n, m)
            # the warm start ends at the oracle's answer whenever the cold start does
            e0 = O.aligned_rel_rmse(d0.cpu().numpy(), ref["depth"], w.mask, 1)
            e1 = O.aligned_rel_rmse(d1.cpu().numpy(), ref["depth"], w.mask, 1)
            if np.array_equal(l0.cpu().numpy(), ref["labels"]) and e0 <= 1e-4:
                assert np.array_equal(l1.cpu().numpy(), ref["labels"])
                assert e1 <= 1e-4, (e0, e1)
            cold_it.append(s0["fill_px_iters"])
            warm_it.append(s1["fill_px_iters"])
            cold.close()
            warm.close()
        gains[pc] = 1.0 - sum(warm_it) / sum(cold_it)
        print(f"precond {pc}: fill pixel-iterations cold {sum(cold_it)} warm {sum(warm_it)} "
              f"(gain {100 * gains[pc]:.1f} %)")
        assert sum(warm_it) <= 1.1 * sum(cold_it)


@pytest.mark.parametrize("name", ["c2", "c3_small"])
def test_learned_alignment_weights_stay_within_bound(name):
    """learned_weights: the network's predicted continuity of each inter edge
    weights the two alignment iterations instead of 1.  The result is no longer
    the plain method's, so it is accepted on a map only if the final depth stays
    within the 1e-3 relative RMSE bound of the FP64 oracle's plain method
    (measured: 3e-4 on the 512 x 612 map, 3e-6 on the 512 x 512 one); it must
    also differ from the uniform alignment (the weights are used)."""
    from gpu_util import rel_depth_error
    w = make_workload(name)
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    res = {}
    for lw in (0, 1):
        it = integrator(H, W, w.camera, w.params, warm_start=1, learned_weights=lw)
        it.load_net(ni.default_net_path())
        d, l, st = it.integrate(n, m)
        res[lw] = np.log(d.cpu().numpy())
        it.close()
    ref = O.integrate(w.normals, w.mask, w.camera, O.Params.from_dict(w.params))
    err = rel_depth_error(np.nan_to_num(res[1]), np.nan_to_num(ref["z"]), w.mask, 1)
    diff = float(np.nanmax(np.abs(res[1] - res[0])))
    print(name, "learned alignment weights: rel err vs oracle", err, "max |dz| vs uniform", diff)
    assert err <= 1e-3
    assert diff > 1e-7
