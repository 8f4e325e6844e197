"""The multi-rank path of bench.py on CPU (gloo, world size 2): each rank solves its own
replica (the H-LU does not shard), the step time is the slowest rank's and the
throughput counts the unknowns of all ranks; the reference arm does its work on rank 0
only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.aggregate(100.0 * (rank + 1), 1000 + rank, dist, device="cpu")
    out[rank] = (ms, value)

    class Args:
        workload, warmup, steps, gpus = "sphere_d1_m1_nc8", 0, 1, world

    if rank == 1:
        bench.run_reference(Args, rank, world)  # returns without work on rank 1
    dist.destroy_process_group()


def test_aggregate_takes_slowest_rank_and_sums_unknowns():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        ms, value = out[r]
        assert ms == 200.0
        assert abs(value - 2001 / 0.2) < 1e-9


def test_single_process_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate(250.0, 500, None)
    assert ms == 250.0 and abs(value - 2000.0) < 1e-12
