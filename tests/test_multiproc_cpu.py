"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Nothing in this build uses more than one GPU: under torchrun the benchmark
runs one independent image per rank (replicas) and reports all ranks' voxels
over the slowest rank's time. These tests check that reduction with real
processes, without any GPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        step_ms = [2.0, 5.0, 3.0][rank]
        value, slowest = bench.aggregate(1_000_000, step_ms, world)
        mx = bench._max_over_ranks(float(rank * 10), world)
        q.put((rank, value, slowest, mx))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replicas_aggregate_over_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slow = max([2.0, 5.0, 3.0][:world])
    for rank, value, slowest, mx in out:
        assert slowest == slow
        assert abs(value - world * 1e6 / (slow * 1e-3) / 1e9) < 1e-12
        assert mx == float((world - 1) * 10)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, slowest = bench.aggregate(2_000_000, 4.0, 1)
    assert slowest == 4.0 and abs(value - 0.5) < 1e-12
