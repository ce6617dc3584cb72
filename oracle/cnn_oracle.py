"""FP64 CPU oracle of the learned warm-start network (an extension beyond the paper,
not a method of the paper).  TEST INFRASTRUCTURE ONLY.

Network: 6 valid 3x3 convolutions, channels 4 -> 32 -> 32 -> 32 -> 32 -> 32 -> 5,
ReLU after the first five; NHWC arrays; parameters in the flat layout
W_l[3][3][cin][cout] then b_l[cout] per layer.

`quantize=True` rounds to bfloat16 exactly where the GPU kernels store BF16
values (the input, the weights, every hidden activation, the output gradient and
the masked activation gradients), and computes everything else in float64, so
GPU and oracle differ only by the order of FP32 accumulation.  `quantize=False`
is a plain float64 network, used to pin the backward pass by finite differences.

Loss (gauge-free, see ni_cnn.h): mean over intra-component right/down edges of
((z_a - z_b) - (t_a - t_b))^2, plus w_weight times the mean binary cross-entropy
of the four edge logits against their targets.
"""
from __future__ import annotations

import numpy as np

LAYERS = [(4, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 5)]
HALO = 6


def num_params():
    return sum(9 * ci * co + co for ci, co in LAYERS)


def unpack(params):
    out, o = [], 0
    for ci, co in LAYERS:
        W = params[o:o + 9 * ci * co].reshape(3, 3, ci, co)
        o += 9 * ci * co
        b = params[o:o + co]
        o += co
        out.append((W, b))
    return out


def bf16(x):
    """Round float64 values to bfloat16 (round to nearest even) via float32."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv_valid(x, W):
    """x [B,H,W,ci], W [3,3,ci,co] -> [B,H-2,W-2,co] (cross-correlation)."""
    B, H, Wd, _ = x.shape
    out = np.zeros((B, H - 2, Wd - 2, W.shape[3]))
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("bhwc,cd->bhwd", x[:, dy:dy + H - 2, dx:dx + Wd - 2, :], W[dy, dx])
    return out


def forward(params, x, quantize=True):
    """x [B, T+12, T+12, 4] -> (output [B, T, T, 5], list of layer inputs)."""
    q = bf16 if quantize else (lambda a: np.asarray(a, np.float64))
    layers = unpack(np.asarray(params, np.float64))
    a = q(x)
    acts = [a]
    for i, (W, b) in enumerate(layers):
        z = conv_valid(a, q(W)) + np.asarray(b, np.float32).astype(np.float64)
        if i < len(layers) - 1:
            a = q(np.maximum(z, 0.0))
            acts.append(a)
        else:
            out = z.astype(np.float32).astype(np.float64) if quantize else z
    return out, acts


def loss_and_grad_out(out, tz, tl, tw, w_weight):
    """Loss terms and d loss / d output ([B,T,T,5])."""
    B, T = tz.shape[0], tz.shape[1]
    z = out[..., 0]
    g = np.zeros_like(out)
    ld_sum, nd = 0.0, 0
    for axis in (2, 1):   # right edges (x), down edges (y)
        za, zb = np.moveaxis(z, axis, 0)[:-1], np.moveaxis(z, axis, 0)[1:]
        ta, tb = np.moveaxis(tz, axis, 0)[:-1], np.moveaxis(tz, axis, 0)[1:]
        la, lb = np.moveaxis(tl, axis, 0)[:-1], np.moveaxis(tl, axis, 0)[1:]
        m = (la >= 0) & (la == lb)
        d = np.where(m, (za - zb) - (ta - tb), 0.0)
        ld_sum += float(np.sum(d * d))
        nd += int(m.sum())
        gz = np.zeros_like(np.moveaxis(z, axis, 0))
        gz[:-1] += 2 * d
        gz[1:] -= 2 * d
        g[..., 0] += np.moveaxis(gz, 0, axis)
    valid = tl >= 0
    lw_sum, nw = 0.0, 0
    logits = out[..., 1:5]
    gl = np.zeros_like(logits)
    shifts = [(0, 1), (1, 0), (0, -1), (-1, 0)]   # right, down, left, up as (dy, dx)
    for dirn, (dy, dx) in enumerate(shifts):
        nb = np.zeros_like(valid)
        ys = slice(max(0, -dy), T - max(0, dy))
        xs = slice(max(0, -dx), T - max(0, dx))
        yt = slice(max(0, dy), T - max(0, -dy))
        xt = slice(max(0, dx), T - max(0, -dx))
        nb[:, ys, xs] = valid[:, yt, xt]
        m = valid & nb
        lg = logits[..., dirn]
        wt = tw[..., dirn]
        sp = np.logaddexp(0.0, lg)
        lw_sum += float(np.sum(np.where(m, sp - wt * lg, 0.0)))
        nw += int(m.sum())
        gl[..., dirn] = np.where(m, 1.0 / (1.0 + np.exp(-lg)) - wt, 0.0)
    ld = ld_sum / nd if nd else 0.0
    lw = lw_sum / nw if nw else 0.0
    g[..., 0] = g[..., 0] / nd if nd else 0.0
    g[..., 1:5] = w_weight * gl / nw if nw else 0.0
    return ld + w_weight * lw, ld, lw, g


def backward(params, x, tz, tl, tw, w_weight, quantize=True):
    """(loss, grads [num_params]) with the GPU's quantisation points."""
    q = bf16 if quantize else (lambda a: np.asarray(a, np.float64))
    layers = unpack(np.asarray(params, np.float64))
    out, acts = forward(params, x, quantize)
    loss, ld, lw, g = loss_and_grad_out(out, tz, tl, tw, w_weight)
    g = q(g)
    grads = []
    for i in range(len(layers) - 1, -1, -1):
        W, b = layers[i]
        a = acts[i]
        Ho = g.shape[1]
        dW = np.zeros_like(W)
        for dy in range(3):
            for dx in range(3):
                dW[dy, dx] = np.einsum("bhwc,bhwd->cd", a[:, dy:dy + Ho, dx:dx + Ho, :], g)
        db = g.sum(axis=(0, 1, 2))
        grads.append((dW, db))
        if i == 0:
            break
        # gradient w.r.t. the layer input: full convolution with the flipped kernel
        gp = np.pad(g, ((0, 0), (2, 2), (2, 2), (0, 0)))
        Wf = q(W)[::-1, ::-1].transpose(0, 1, 3, 2)
        da = conv_valid(gp, Wf)
        g = q(da * (acts[i] > 0))
    flat = []
    for dW, db in reversed(grads):
        flat.append(dW.reshape(-1))
        flat.append(db)
    return (loss, ld, lw), np.concatenate(flat)
