"""The N > 1 path of bench.py (independent replicas, one process per GPU) on
CPU: two gloo ranks check the job-level aggregation -- the slowest rank's
time and the products of all ranks -- without a GPU."""
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 150.0][rank]          # rank 1 is the slowest
        ms, gflops = bench.job_throughput(local_ms, 3, 1_000_000_000, world, dist, device="cpu")
        e2e = bench.max_over_ranks([7.0, 5.0][rank], dist, device="cpu")
        out[rank] = (ms, gflops, e2e)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ms, gflops, e2e = out[r]
        assert ms == pytest.approx(50.0)                       # 150 ms / 3 steps, max over ranks
        assert gflops == pytest.approx(2 * 2 * 1e9 / 0.050 / 1e9)
        assert e2e == 7.0


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    ms, gflops = bench.job_throughput(90.0, 3, 10**9, 1, None)
    assert ms == pytest.approx(30.0) and gflops == pytest.approx(2e9 / 0.030 / 1e9)
