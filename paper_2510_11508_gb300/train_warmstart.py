"""Train the learned warm start on synthetic maps solved by the plain method.

Pipeline (every numerical step on the GPU runs in libni's kernels):
  1. generate n seeded C2-type maps of tile x tile pixels (synth, CPU processes);
  2. solve each with libni (seeding, fill, relative-scale loop): the fill's
     log-depth is the depth target, the seeding labels select the intra-component
     edges of the loss, and the BiNI weights of the final log-depth
     (ni_cnn_edge_targets) are the edge-weight targets;
  3. train the network with its BF16 tensor-core forward/backward kernels and
     Adam (ni_cnn_train_step); write the weights with Net.save.

    python -m paper_2510_11508_gb300.train_warmstart --maps 10000 --epochs 3 --out net.bin
"""
from __future__ import annotations

import argparse
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _gen(args):
    seed, tile = args
    from synth.generators import c2_type_map
    w = c2_type_map(H=tile, W=tile, n_cells=8, target_valid=0.128 * tile * tile, seed=seed, name="train")
    return w.normals, w.mask


def generate(n_maps: int, seed0: int, tile: int, workers: int):
    """Seeded C2-type maps (normals float32 [n, t, t, 4], mask uint8 [n, t, t])."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        res = pool.map(_gen, [(seed0 + i, tile) for i in range(n_maps)], chunksize=16)
    normals = np.stack([r[0] for r in res])
    masks = np.stack([r[1] for r in res])
    from synth.generators import _persp_cam
    return normals, masks, _persp_cam(tile, tile)


def solve_targets(normals, masks, camera, params, device):
    """Plain-method targets for every map: (inputs, fill log-depth, labels, edge weights)."""
    import torch
    from paper_2510_11508_gb300 import cnn, ni
    n, t = normals.shape[0], normals.shape[1]
    cfg = ni.config_for(t, t, camera, params, batched=1, validate=0, use_graph=0)
    it = ni.Integrator(cfg)
    S = t + 2 * cnn.HALO
    X = torch.empty((n, S, S, 4), dtype=torch.float32, device=device)
    TZ = torch.empty((n, t, t), dtype=torch.float32, device=device)
    TL = torch.empty((n, t, t), dtype=torch.int32, device=device)
    TW = torch.empty((n, t, t, 4), dtype=torch.float32, device=device)
    for i in range(n):
        nd = torch.from_numpy(normals[i]).to(device)
        md = torch.from_numpy(masks[i]).to(device)
        lab, _ = it.seed_components(nd, md)
        z_fill = it.solve_components(allow_unconverged=True)
        it.solve_scales(int(params.get("T", 15)))
        z_final = it.logdepth()
        X[i] = cnn.make_tiles(nd, md, t)[0]
        TZ[i] = z_fill
        TL[i] = lab
        TW[i] = cnn.edge_targets(nd, md, z_final, camera, params.get("k", 2.0))
    torch.cuda.synchronize()
    it.close()
    return X, TZ, TL, TW


def train(net, data, epochs: int, batch: int, lr: float, w_weight: float, val_frac=0.02, log=print):
    import torch
    X, TZ, TL, TW = data
    n = X.shape[0]
    nval = max(1, int(n * val_frac))
    ntr = n - nval
    steps_per_epoch = max(1, ntr // batch)
    total = epochs * steps_per_epoch
    g = torch.Generator(device="cpu").manual_seed(0)
    history = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(ntr, generator=g).to(X.device)
        acc = 0.0
        for s in range(steps_per_epoch):
            idx = perm[s * batch:(s + 1) * batch]
            lr_s = lr * 0.5 * (1 + math.cos(math.pi * step / total))
            loss = net.train_step(X[idx].contiguous(), TZ[idx].contiguous(), TL[idx].contiguous(),
                                  TW[idx].contiguous(), lr=lr_s, w_weight=w_weight)
            acc += loss[0]
            step += 1
        vl = evaluate_loss(net, (X[ntr:], TZ[ntr:], TL[ntr:], TW[ntr:]), batch, w_weight)
        history.append(dict(epoch=ep, train=acc / steps_per_epoch, val=vl))
        log(f"epoch {ep}: train loss {acc / steps_per_epoch:.5f}  val (loss, depth, weight) {vl}")
    return history


def evaluate_loss(net, data, batch, w_weight):
    X, TZ, TL, TW = data
    tot = np.zeros(3)
    cnt = 0
    for s in range(0, X.shape[0], batch):
        sl = slice(s, min(X.shape[0], s + batch))
        (l, ld, lw), _ = net.loss_grad(X[sl].contiguous(), TZ[sl].contiguous(), TL[sl].contiguous(),
                                       TW[sl].contiguous(), w_weight=w_weight, want_grad=False)
        k = X[sl].shape[0]
        tot += np.array([l, ld, lw]) * k
        cnt += k
    return tuple(float(v) for v in tot / cnt)


def zero_predictor_loss(data, w_weight):
    """Loss of the trivial predictor (z = 0, logits = 0): the baseline the trained
    network is compared with."""
    import torch
    X, TZ, TL, TW = data
    tz, tl = TZ.double(), TL
    nd, sd = 0, 0.0
    for dim in (2, 1):
        a = tl.narrow(dim, 0, tl.shape[dim] - 1)
        b = tl.narrow(dim, 1, tl.shape[dim] - 1)
        m = (a >= 0) & (a == b)
        d = tz.narrow(dim, 0, tz.shape[dim] - 1) - tz.narrow(dim, 1, tz.shape[dim] - 1)
        sd += float((d * d)[m].sum())
        nd += int(m.sum())
    return sd / max(nd, 1)


def fold_depth_scale(p, scale):
    """Multiply the network's depth output (channel 0 of the last layer) by `scale`
    by rescaling that channel's weights and bias in the flat parameter vector."""
    from paper_2510_11508_gb300 import cnn
    n_last = 9 * 32 * 5
    off = cnn.num_params() - (n_last + 5)
    W = p[off:off + n_last].reshape(3, 3, 32, 5)
    W[..., 0] *= scale
    p[off + n_last] *= scale


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--maps", type=int, default=10000)
    ap.add_argument("--seed0", type=int, default=0)
    ap.add_argument("--tile", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--w-weight", type=float, default=0.1)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--out", default="warmstart_net.bin")
    args = ap.parse_args()
    t0 = time.time()
    normals, masks, cam = generate(args.maps, args.seed0, args.tile, args.workers)   # before any CUDA call
    t1 = time.time()
    import torch
    from paper_2510_11508_gb300 import cnn
    from synth.generators import DEFAULT_PARAMS
    params = dict(DEFAULT_PARAMS, theta_c_deg=3.5)
    data = solve_targets(normals, masks, cam, params, torch.device("cuda"))
    t2 = time.time()
    net = cnn.Net(args.batch, args.tile, seed=1)
    # train on depth targets scaled to unit RMS edge difference; the scale is
    # folded back into the last layer's depth channel before saving
    zscale = 1.0 / math.sqrt(max(zero_predictor_loss(data, 0.0), 1e-30))
    X, TZ, TL, TW = data
    data = (X, TZ * zscale, TL, TW)
    nval = max(1, int(args.maps * 0.02))
    base = zero_predictor_loss(tuple(d[-nval:] for d in data), args.w_weight)
    hist = train(net, data, args.epochs, args.batch, args.lr, args.w_weight)
    t3 = time.time()
    p = net.get_params()
    fold_depth_scale(p, 1.0 / zscale)
    net.set_params(p)
    net.save(args.out)
    print(f"maps {args.maps}: generate {t1 - t0:.1f} s, solve {t2 - t1:.1f} s, train {t3 - t2:.1f} s; "
          f"validation depth loss {hist[-1]['val'][1]:.6f} vs zero predictor {base:.6f} "
          f"(depth targets scaled by {zscale:.4g}); saved {args.out}")


if __name__ == "__main__":
    main()
