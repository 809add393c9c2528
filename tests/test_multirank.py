"""The N > 1 path of bench.py on CPU (gloo, world size 2): every rank times its own
replica, the job's time is the maximum over ranks and the throughput counts every
rank's ciphertexts (weak scaling, no data-path collective)."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own = [120.0, 150.0][rank]  # this rank's timed region, ms
        t = bench.max_over_ranks(own, dist)
        q.put((rank, t, bench.replica_throughput(world, 256, 5, t / 1e3)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, value in res:
        assert t == 150.0  # both ranks see the slowest rank's time
        assert value == pytest.approx(2 * 256 * 5 / 0.150)


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(42.0, None) == 42.0
    assert bench.replica_throughput(1, 256, 5, 2.0) == 640.0
