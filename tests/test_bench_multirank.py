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


def _run_bench(args, env_extra=None):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py")] + args, cwd=root,
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference: the oracle on the host cores, one JSON line with
    the suspension metric, a cpu_baseline describing the run and an e2e record
    with no host-device traffic."""
    import bench
    (line,) = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1"])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 1 and line["warmup"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert isinstance(cb["sample"], str) and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    assert _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1"],
                      {"RANK": "1", "WORLD_SIZE": "2"}) == []
