"""The replicas-only multi-GPU contract of bench.py on the host: world size 2
over gloo (one process per rank), the slowest rank's time sets the job's time
and the value counts every rank's pixels."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    seconds = bench.max_over_ranks(1.0 + rank)          # rank 1 is the slow one
    value = bench.replica_throughput(seconds, units_per_rank=1_000_000, steps=3)
    q.put((rank, seconds, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, seconds, value in got:
        assert seconds == pytest.approx(2.0)                 # max over ranks
        assert value == pytest.approx(2 * 1e6 * 3 / 2.0 / 1e6)   # both ranks' pixels / slowest time


def test_single_process_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.replica_throughput(2.0, 4_000_000, 5) == pytest.approx(10.0)


def test_mask_islands_match_the_oracle():
    """The bench's island labels (error alignment against the ground truth) are
    the oracle's islands of the mask, label for label."""
    import numpy as np
    import bench
    import oracle as O
    rng = np.random.default_rng(2)
    for H, W in ((1, 1), (17, 23), (64, 50)):
        mask = (rng.random((H, W)) > 0.45).astype(np.uint8)
        lab, n = bench.mask_islands(mask)
        ref, nr = O.islands(mask)
        assert n == nr and lab.dtype == np.int32
        np.testing.assert_array_equal(lab, ref)
