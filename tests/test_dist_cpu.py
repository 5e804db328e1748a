"""The multi-GPU path of bench.py is replicas only (every rank solves its
own copy; the method has no exchange step here): its barrier and
max-over-ranks timing are checked with two gloo ranks on the CPU."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    mx = bench.reduce_max(10.0 + 5.0 * rank, world)
    out.put((rank, mx))
    bench.barrier(world)
    dist.destroy_process_group()


def test_replica_timing_takes_the_max_over_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res == [(0, 15.0), (1, 15.0)]


def test_single_rank_helpers_are_identities():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)
    assert bench._dist_env() == (0, 0, 1) or "RANK" in os.environ
