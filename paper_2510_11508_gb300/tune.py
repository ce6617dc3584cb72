"""Autotuner of the launch shapes and preconditioner knobs, and the tuning
table the library reads at run time (ni_load_tuning).

Runs ni_integrate on a map for every point of a small search space and
returns the configuration with the lowest median time whose labels are equal to
the reference configuration's and whose log-depth agrees with it to `rtol`
(the tuner never trades accuracy for speed).  Knobs:

  ctas_per_sm       CTAs per SM of the persistent fill kernel (occupancy vs.
                    grid-barrier cost);
  mg_cta_cells      coarse-level cells per CTA of a multigrid pass (a pass syncs
                    only its CTAs: fewer barrier arrivals vs. serial work);
  mg_omega          damped-Jacobi weight of the V-cycle smoother;
  scale_solver      relative-scale PCG in one thread-block cluster (1) or a
                    cooperative grid (2).

`--write PATH` tunes a list of maps of growing size and writes one table row
per map, keyed by its grid pixels and its components after seeding; the
library then picks the knobs of the first row that covers a new map:

    python -m paper_2510_11508_gb300.tune --workload c3
    python -m paper_2510_11508_gb300.tune --write table.txt --workloads c2,c3,c4_eval,c5
"""
from __future__ import annotations

import argparse
import itertools
import os
import sys
from typing import Dict, Iterable, Optional

import numpy as np
import torch

from . import ni

SPACE = {
    "ctas_per_sm": [2, 4],
    "mg_cta_cells": [256, 512],
    "mg_omega": [0.85, 0.9, 0.95],
    "scale_solver": [1, 2],
}
# the library's defaults of the same knobs (what a 0 in the config means)
DEFAULTS = {"ctas_per_sm": 4, "mg_cta_cells": 256, "mg_omega": 0.9, "scale_solver": 0}


def _time(it, n, m, reps):
    ts = []
    out = None
    for _ in range(reps):
        out = it.integrate(n, m, allow_unconverged=True)
        ts.append(out[2]["ms_total"])
    return float(np.median(ts)), out


def tune(normals: torch.Tensor, mask: torch.Tensor, camera: Dict, params: Optional[Dict] = None,
         space: Optional[Dict[str, Iterable]] = None, reps: int = 3, rtol: float = 1e-4, log=print):
    """Grid search over `space` (default SPACE) with precond = 1; returns
    (best knob dict, list of (knobs, ms, fill_iters))."""
    H, W = mask.shape
    space = dict(SPACE if space is None else space)
    base = ni.Integrator(ni.config_for(H, W, camera, params, precond=1))
    ms0, (d0, l0, s0) = _time(base, normals, mask, reps)
    base.close()
    l0 = l0.cpu().numpy()
    z0 = torch.log(d0).cpu().numpy() if camera["camera"] == 1 else d0.cpu().numpy()
    valid = mask.cpu().numpy() > 0
    table = []
    best, best_ms = {}, ms0
    keys = list(space)
    for vals in itertools.product(*(space[k] for k in keys)):
        knobs = dict(zip(keys, vals))
        it = ni.Integrator(ni.config_for(H, W, camera, params, precond=1, **knobs))
        try:
            ms, (d, l, s) = _time(it, normals, mask, reps)
        finally:
            it.close()
        z = torch.log(d).cpu().numpy() if camera["camera"] == 1 else d.cpu().numpy()
        dz = (z - z0)[valid]
        dz = dz - dz.mean() if dz.size else dz
        ok = (s["fill_unconverged"] == 0 and np.array_equal(l.cpu().numpy(), l0)
              and (dz.size == 0 or float(np.sqrt(np.mean(dz * dz))) <= rtol))
        table.append((knobs, ms, s["fill_iters"], ok))
        log(f"{knobs} {ms:8.3f} ms fill_iters {s['fill_iters']:5d} {'ok' if ok else 'REJECTED'}")
        if ok and ms < best_ms:
            best, best_ms = knobs, ms
    log(f"default {ms0:.3f} ms -> best {best_ms:.3f} ms with {best}")
    return best, table, ms0, best_ms, s0


def write_table(path: str, rows, log=print):
    """rows: (max_px, max_k0, knobs) in increasing max_px; a last catch-all row
    keeps the defaults."""
    with open(path, "w") as f:
        f.write("# tuning table of libni (ni_load_tuning), written by paper_2510_11508_gb300.tune\n")
        f.write("# max_px max_k0 ctas_per_sm mg_cta_cells mg_omega scale_solver\n")
        for max_px, max_k0, knobs, note in rows:
            k = dict(DEFAULTS, **knobs)
            f.write(f"{max_px} {max_k0} {k['ctas_per_sm']} {k['mg_cta_cells']} {k['mg_omega']} "
                    f"{k['scale_solver']}  # {note}\n")
        f.write(f"{1 << 40} {1 << 40} 0 0 0 0  # anything larger: the built-in defaults\n")
    log(f"wrote {path}")


def main():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from synth import make_workload
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c3")
    ap.add_argument("--workloads", default="c2,c3,c4_eval,c5")
    ap.add_argument("--write", default=None, help="tune every map of --workloads and write the table here")
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    if a.write is None:
        w = make_workload(a.workload)
        n = torch.from_numpy(w.normals).cuda()
        m = torch.from_numpy(w.mask).cuda()
        tune(n, m, w.camera, w.params, reps=a.reps)
        return
    rows = []
    for name in a.workloads.split(","):
        w = make_workload(name)
        n = torch.from_numpy(w.normals).cuda()
        m = torch.from_numpy(w.mask).cuda()
        best, _, ms0, ms1, s0 = tune(n, m, w.camera, w.params, reps=a.reps)
        H, W = w.mask.shape
        rows.append((H * W, 4 * max(1, s0["K0"]), best,
                     f"{w.name}: K0 {s0['K0']}, default {ms0:.2f} ms, tuned {ms1:.2f} ms"))
        del n, m
        torch.cuda.empty_cache()
    rows.sort(key=lambda r: r[0])
    write_table(a.write, rows)


if __name__ == "__main__":
    main()
