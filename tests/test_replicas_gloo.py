"""The multi-GPU path of bench.py on CPU: world_size-2 gloo ranks.

The solve has no data exchange, so N GPUs run N replicas and the job is timed by its slowest
rank; these tests run that reduction and the job-rate formula on two gloo ranks (no GPU).
"""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], "cpu")
        ws, r, _ = bench._dist()
        q.put((rank, ms, ws, r, bench.job_rate(6, ws, ms)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_times_the_job():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [812.5, 1003.25]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, ms, ws, r_env, rate) in enumerate(out):
        assert r == rank and r_env == rank and ws == 2
        assert ms == max(times)  # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 6 / (max(times) / 1e3))


def test_single_process_is_its_own_maximum():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(123.5, "cpu") == 123.5
    assert bench.job_rate(6, 1, 1000.0) == pytest.approx(6.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle and prints; the other ranks exit at once."""
    sys.path.insert(0, ROOT)
    import types

    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "oracle_sample", lambda budget: pytest.fail("rank 1 ran the oracle"))
    bench.bench_reference(types.SimpleNamespace(warmup=1, steps=1, cpu_budget=1.0))
    assert capsys.readouterr().out == ""
