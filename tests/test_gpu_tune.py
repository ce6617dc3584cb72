"""The run-time tuning table (ni_load_tuning): the knobs it picks for the
2048 x 2048 map give the oracle's answer and are no slower than the built-in
defaults; malformed tables are rejected."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2510_11508_gb300 import ni
from synth import make_workload

from gpu_util import PIXEL_TOL, dev, integrator, rel_depth_error, rel_depth_max

pytestmark = pytest.mark.gpu


def _median_ms(it, n, m, reps=7):
    it.integrate(n, m)
    ts = []
    for _ in range(reps):
        ts.append(it.integrate(n, m)[2]["ms_total"])
    return float(np.median(ts))


def test_tuned_knobs_match_oracle_and_are_not_slower():
    path = ni.default_tuning_path()
    assert os.path.exists(path)
    w = make_workload("c3")
    H, W = w.mask.shape
    n, m = dev(w.normals, w.mask)
    base = integrator(H, W, w.camera, w.params)
    tuned = integrator(H, W, w.camera, w.params)
    tuned.load_tuning(path)
    ms0 = _median_ms(base, n, m)
    ms1 = _median_ms(tuned, n, m)
    depth, labels, st = tuned.integrate(n, m)
    ref = O.integrate(w.normals, w.mask, w.camera, O.Params.from_dict(w.params), workers=4)
    zg = np.log(depth.cpu().numpy())
    err = rel_depth_error(np.nan_to_num(zg), np.nan_to_num(ref["z"]), w.mask, 1)
    mx = rel_depth_max(np.nan_to_num(zg), np.nan_to_num(ref["z"]), w.mask, 1)
    print("c3 default", ms0, "ms, tuned", ms1, "ms, err", err, "max", mx)
    assert st["K_final"] == ref["K"] and st["scale_iters"] == ref["iters"]
    np.testing.assert_array_equal(labels.cpu().numpy(), ref["labels"])
    assert err <= 1e-4 and mx <= PIXEL_TOL
    assert ms1 <= 1.05 * ms0


def test_malformed_tuning_table_is_rejected(tmp_path):
    it = integrator(64, 64, {"camera": 1, "fx": 96.0, "fy": 96.0, "cx": 32.0, "cy": 32.0})
    bad = tmp_path / "bad.txt"
    bad.write_text("100 10 4 256 1.5 0\n")          # mg_omega outside [0, 1)
    with pytest.raises(ni.NIError):
        it.load_tuning(str(bad))
    with pytest.raises(ni.NIError):
        it.load_tuning(str(tmp_path / "missing.txt"))
    good = tmp_path / "good.txt"
    good.write_text("# comment\n4096 100 2 512 0.85 2\n")
    it.load_tuning(str(good))
