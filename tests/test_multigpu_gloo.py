"""Host logic of the multi-GPU path on CPU with the gloo backend (world size 2): the weak-scaling
rate takes the slowest rank's time, shard ranges cover a global batch exactly once, and the
tensor-field loss split over the ranks adds up to the loss of the whole field through its one
all_reduce. The decomposition itself has no exchange step: each rank works on its own matrices."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rate, elapsed = bench.whole_job_rate(1.0 + rank, 1000, world, "cpu")
        import workloads as W
        A, _ = W.sym3_precision(64, seed=rank)
        q.put((rank, rate, elapsed, float(A.abs().sum())))
    finally:
        dist.destroy_process_group()


def _field_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import workloads as W
        S = W.structure_tensor_field((16, 16, 9), seed=0, device="cpu", dtype=torch.float32)
        seen = []

        # stand-in for the loss kernel on a shard (the host logic under test is the split and the
        # reduction): per-voxel sums of the entries and of their squares, in float64
        def shard(a, b):
            seen.append((a, b))
            X = S[:, a:b].double()
            return torch.stack([X.sum(), (X * X).sum()])
        tot = bench.sharded_st_loss(S.shape[1], rank, world, shard)
        q.put((rank, seen, tot.tolist(), [float(S.double().sum()), float((S.double() ** 2).sum())]))
    finally:
        dist.destroy_process_group()


def test_sharded_field_loss_adds_up_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_field_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = 16 * 16 * 9
    assert out[0][1] == [bench.shard_range(n, 0, 2)] and out[1][1] == [bench.shard_range(n, 1, 2)]
    for _, _, tot, full in out:
        assert tot == pytest.approx(full, rel=1e-12)


def test_weak_scaling_rate_uses_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # 2 ranks x 1000 units in max(1.0, 2.0) s
    assert out[0][1] == pytest.approx(1000.0) and out[1][1] == pytest.approx(1000.0)
    assert out[0][2] == 2.0 and out[1][2] == 2.0
    # each rank draws its own batch (seed = rank)
    assert out[0][3] != out[1][3]


@pytest.mark.parametrize("n,world", [(0, 2), (7, 2), (10, 3), (1 << 20, 8), (5, 8)])
def test_shard_ranges_cover_the_batch_once(n, world):
    ranges = [bench.shard_range(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c and a <= b
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_single_rank_rate_needs_no_process_group():
    rate, elapsed = bench.whole_job_rate(0.5, 100, 1)
    assert rate == 200.0 and elapsed == 0.5
