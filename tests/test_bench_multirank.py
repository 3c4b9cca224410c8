"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
replica's pair count and device time, aggregate to (sum, max) -- the
whole-job throughput is the units of all ranks over the slowest rank."""
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
    units = [3.0e11, 5.0e11][rank]
    ms = [120.0, 150.0][rank]
    tot, mx = bench.aggregate_ranks(units, ms, dist, "cpu")
    out.put((rank, tot, mx))
    dist.destroy_process_group()


def test_two_rank_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, tot, mx in res:
        assert tot == 8.0e11
        assert mx == 150.0


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_ranks(7.0, 3.0, None, "cpu") == (7.0, 3.0)
