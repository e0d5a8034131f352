"""The bench's multi-rank timing on CPU: two gloo ranks, max over ranks and
the weak-scaling throughput (every rank searches its own light curves; no
data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, torch, torch.device("cpu"))
    val = bench.weak_scaling_value(194400, world, ms)
    q.put((rank, ms, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_weak_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, val in res:
        assert ms == 150.0                       # slowest rank
        assert val == pytest.approx(2 * 194400 / 0.150)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, torch, torch.device("cpu")) == 12.5
