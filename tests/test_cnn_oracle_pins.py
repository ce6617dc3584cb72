"""Pins of the warm-start network's oracle (oracle/cnn_oracle.py): its bf16
rounding against torch's, its convolution against brute-force loops, its
backward pass against central finite differences of the float64 network, and
the gauge freedom of its depth loss."""
import numpy as np
import pytest
import torch

from oracle import cnn_oracle as CO


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000), [0.0, -0.0, 1.0, 3.0e38]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(CO.bf16(x), ref)


def test_conv_valid_brute_force():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 6, 7, 3))
    W = rng.normal(size=(3, 3, 3, 4))
    out = CO.conv_valid(x, W)
    ref = np.zeros((2, 4, 5, 4))
    for b in range(2):
        for y in range(4):
            for xx in range(5):
                for co in range(4):
                    ref[b, y, xx, co] = sum(x[b, y + dy, xx + dx, ci] * W[dy, dx, ci, co]
                                            for dy in range(3) for dx in range(3) for ci in range(3))
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def _problem(T=4, B=1, seed=2):
    rng = np.random.default_rng(seed)
    S = T + 2 * CO.HALO
    x = rng.normal(0, 0.5, (B, S, S, 4))
    x[..., 3] = (rng.uniform(size=(B, S, S)) > 0.1).astype(float)
    p = rng.normal(0, 0.3, CO.num_params())
    tz = rng.normal(0, 1, (B, T, T))
    tl = rng.integers(-1, 2, (B, T, T))
    tw = rng.uniform(0, 1, (B, T, T, 4))
    return p, x, tz, tl, tw


def test_backward_matches_finite_differences():
    p, x, tz, tl, tw = _problem()
    (loss, _, _), g = CO.backward(p, x, tz, tl, tw, 0.3, quantize=False)
    rng = np.random.default_rng(3)
    idx = rng.choice(len(p), 40, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        lp = CO.backward(pp, x, tz, tl, tw, 0.3, quantize=False)[0][0]
        lm = CO.backward(pm, x, tz, tl, tw, 0.3, quantize=False)[0][0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 2e-5 * max(1.0, abs(fd)), (i, fd, g[i])


def test_depth_loss_is_blind_to_per_component_offsets():
    p, x, tz, tl, tw = _problem(T=8, seed=4)
    out, _ = CO.forward(p, x, quantize=False)
    l0 = CO.loss_and_grad_out(out, tz, tl, tw, 0.0)[0]
    tz2 = tz + np.where(tl >= 0, 5.0 * (tl + 1), 0.0)
    l1 = CO.loss_and_grad_out(out, tz2, tl, tw, 0.0)[0]
    assert abs(l0 - l1) < 1e-9 * max(1, l0)


def test_committed_network_file_layout():
    """The trained warm-start network shipped with the package: magic, parameter
    count of the architecture, tile size, finite weights."""
    import os
    import struct
    path = os.path.join(os.path.dirname(__file__), "..", "paper_2510_11508_gb300", "nets", "warmstart_256.bin")
    raw = open(path, "rb").read()
    assert raw[:8] == b"NICNN001"
    n, tile = struct.unpack("<ii", raw[8:16])
    assert n == CO.num_params() and tile == 256
    w = np.frombuffer(raw[16:], np.float32)
    assert w.size == n and np.isfinite(w).all()
