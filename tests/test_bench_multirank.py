"""The multi-rank logic of bench.py on the CPU: two gloo processes stand in
for two GPUs.  Each rank runs an independent replica of the step, so the
whole-job value is the units of all ranks divided by the slowest rank's time,
and only rank 0 prints."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed 100 + 50 r ms for 1000 (r + 1) pairs
        t, u = bench.reduce_over_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1), world, torch.device("cpu"))
        dist.barrier()
        out[rank] = (t, u, u / (t * 1e-3))
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, u, v = res[r]
        assert t == 150.0 and u == 3000.0
        assert v == pytest.approx(3000.0 / 0.150)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(12.5, 7, 1, None) == (12.5, 7.0)


def test_reference_arm_other_ranks_do_nothing():
    sys.path.insert(0, ROOT)
    import bench
    # rank 1 returns before loading anything
    assert bench.run_reference(None, 1, 2) is None
