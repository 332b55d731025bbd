"""The multi-GPU path of bench.py (independent replicas, one process per GPU) on CPU: two
gloo ranks check the job timing (the slowest rank's time, units of all ranks) and that only
rank 0 of the reference arm does any work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    assert bench.dist_init() == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 25.0 * rank                       # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (ms, bench.job_ms_per_unit(ms, 10, world))
        # the reference arm: every rank but 0 returns at once without touching its inputs
        if rank:
            assert bench.run_reference(None, None, None, world, rank) is None
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_job_timing_on_gloo():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        ms, per_unit = out[rank]
        assert ms == 125.0                     # the maximum over ranks, seen by every rank
        assert per_unit == 125.0 / (10 * 2)   # 20 solves done by the job in that time


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_ms_per_unit(50.0, 10, 1) == 5.0
