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


def test_reference_arm_prints_the_contract_line():
    # the reference arm (the oracle on the host cores) prints one JSON line with the keys the
    # bench contract names, on the same workload description as the native arm
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "sphere_d1_m1_nc8", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["workload"] == "sphere_d1_m1_nc8" and line["config"]["unknowns"] == 768
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
