"""Multi-process logic on CPU: gloo ranks on 127.0.0.1.

Nothing in this build uses more than one GPU: under torchrun the benchmark
runs one independent image per rank (replicas) and reports all ranks' voxels
over the slowest rank's time. These tests check that reduction with real
processes, without any GPU, and the sharding scheme of one image over
processes (Sec. 3 "Parallel Computations" and "Post-Processing"): each rank
computes the partial VCEC of a range of planes, one int64 all-reduce sums
them and a prefix sum gives the curve. Here the oracle does each rank's part;
the library's per-device step, ecc_compute_vcec_chunk, is compared with the
oracle on the GPU (tests/test_gpu_chunks.py)."""
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


def _shard_worker(rank, world, port, q, conv):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1705_02045_gb300 import synth
        img = synth.smooth_u8((23, 17, 19), 1.5, synth.SEED_BASE + 2300)
        ncoord = img.shape[0] + 1  # cell coordinates along axis 0: 0 .. n0
        lo, hi = ncoord * rank // world, ncoord * (rank + 1) // world
        part = torch.from_numpy(oracle.vcec_int_zrange(img, 256, lo, hi, conv))
        dist.all_reduce(part)  # one int64[bins] sum over the ranks
        q.put((rank, oracle.ecc_from_vcec(part.numpy()).tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("conv", ["V", "T"])
@pytest.mark.parametrize("world", [2, 3])
def test_plane_sharding_with_one_allreduce_over_gloo(world, conv):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1705_02045_gb300 import synth
    want = oracle.ecc_int(synth.smooth_u8((23, 17, 19), 1.5, synth.SEED_BASE + 2300), 256, conv)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q, conv))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, curve in out:
        assert curve == want.tolist()
