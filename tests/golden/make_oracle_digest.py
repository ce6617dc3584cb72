"""Write the FP64 oracle's digest of a full-size workload.

The oracle (oracle/, the plain FP64 CPU implementation of Algorithm 1) runs
on the whole map once, with its components filled in parallel processes, and
this script stores what a GPU run is checked against without re-running it:

  input_sha256      sha256 of the normals (float32) and mask (uint8) bytes,
                    so a check can tell that it sees the same synthetic input
  K0, labels0_sha256  seeding: number of components and the sha256 of the
                    int32 label map (bit-exact comparison)
  K, labels_sha256  the final partition after the relative-scale loop and its
                    merges
  iters, energies   iterations of the loop and E_1..E_t
  sample_idx        seeded sample of valid pixels (raster indices, sorted)
  sample_island     island of the mask (4-connected valid region) of each
  sample_depth      the oracle's depth there (float64)
  merge_t, merge_maps  for every merge, the label each seeding component
                    belongs to after it (seeding label -> label), so a
                    partition that differs can be traced to the merge and the
                    components where it first differs

Nothing here comes from the CUDA path.  Usage:
    python tests/golden/make_oracle_digest.py c5 [--workers N] [--samples S]
"""
import argparse
import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SAMPLE_SEED = 7


def input_sha256(normals, mask):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(normals, dtype=np.float32).tobytes())
    h.update(np.ascontiguousarray(mask, dtype=np.uint8).tobytes())
    return h.hexdigest()


def labels_sha256(labels):
    return hashlib.sha256(np.ascontiguousarray(labels, dtype=np.int32).tobytes()).hexdigest()


def digest_path(workload_name):
    return os.path.join(HERE, f"{workload_name}.oracle.npz")


def main():
    import oracle as O
    from synth import make_workload

    ap = argparse.ArgumentParser()
    ap.add_argument("config")
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--samples", type=int, default=1 << 16)
    args = ap.parse_args()

    t0 = time.perf_counter()
    w = make_workload(args.config)
    t_gen = time.perf_counter() - t0
    H, W = w.mask.shape
    t0 = time.perf_counter()
    ref = O.integrate(w.normals, w.mask, w.camera, O.Params.from_dict(w.params), workers=args.workers)
    t_oracle = time.perf_counter() - t0
    isl, n_isl = O.islands(w.mask)
    valid = np.nonzero(w.mask.reshape(-1) > 0)[0]
    rng = np.random.default_rng(SAMPLE_SEED)
    idx = np.sort(rng.choice(valid, size=min(args.samples, valid.size), replace=False)).astype(np.int32)
    depth = np.asarray(ref["depth"], np.float64).reshape(-1)
    lab0 = np.asarray(ref["labels0"]).reshape(-1)
    first = np.full(int(ref["K0"]), lab0.size, np.int64)
    v0 = lab0 >= 0
    np.minimum.at(first, lab0[v0], np.nonzero(v0)[0])
    merge_t = np.array([m["t"] for m in ref["merges"]], np.int32)
    merge_maps = (np.stack([np.asarray(m["labels"]).reshape(-1)[first] for m in ref["merges"]]).astype(np.int32)
                  if ref["merges"] else np.zeros((0, int(ref["K0"])), np.int32))
    meta = {"workload": w.name, "config": args.config, "H": H, "W": W, "params": w.params,
            "camera": w.camera, "oracle_seconds": t_oracle, "generate_seconds": t_gen,
            "workers": args.workers, "host": platform.machine(), "cpu_count": os.cpu_count(),
            "n_valid": int(valid.size), "islands": int(n_isl)}
    np.savez_compressed(
        digest_path(w.name),
        meta=json.dumps(meta),
        input_sha256=input_sha256(w.normals, w.mask),
        K0=int(ref["K0"]), labels0_sha256=labels_sha256(ref["labels0"]),
        K=int(ref["K"]), labels_sha256=labels_sha256(ref["labels"]),
        iters=int(ref["iters"]), energies=np.asarray(ref["energies"], np.float64),
        sample_idx=idx, sample_island=isl.reshape(-1)[idx].astype(np.int32), sample_depth=depth[idx],
        merge_t=merge_t, merge_maps=merge_maps)
    print(json.dumps(dict(meta, K0=int(ref["K0"]), K=int(ref["K"]), iters=int(ref["iters"]))))


if __name__ == "__main__":
    main()
