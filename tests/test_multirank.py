"""The N > 1 host logic of bench.py as two gloo ranks on the CPU: replicas
per rank with no data-path collective, the timed region's maximum over
ranks, the whole-job value, and the reference arm running on rank 0 only."""
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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    # rank r timed 10 + 5 r ms for its own units
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    value = bench.job_mlups(1_000_000, world, ms)

    class A:
        steps, warmup, gpus = 1, 1, world
    ref = bench.run_reference(A, rank) if rank != 0 else "rank0"
    out[rank] = (ms, value, ref)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    slowest = 10.0 + 5.0 * (world - 1)
    for r in range(world):
        ms, value, ref = out[r]
        assert ms == pytest.approx(slowest)
        assert value == pytest.approx(1_000_000 * world / (slowest * 1e-3) / 1e6)
    assert out[1][2] is None  # the reference arm does no work off rank 0
