"""bench.py's multi-GPU path is replicas only: every rank times its own
independent run, the job's time is the slowest rank's, and the value counts
all ranks' steps.  The aggregation is tested here with two gloo processes on
the CPU (no GPU, no NCCL), and the reference arm's rule that only rank 0
runs and prints."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    secs = 1.0 + rank * 0.5                # rank 1 is the slower replica
    t_max = bench.replica_time(dist, secs, "cpu")
    out.put((rank, t_max, bench.replica_value(world, 5, t_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, value in got:
        assert t_max == 1.5
        assert value == pytest.approx(2 * 5 / 1.5)


def test_single_process_needs_no_group():
    import bench
    assert bench.replica_time(None, 2.0, "cpu") == 2.0
    assert bench.replica_value(1, 4, 2.0) == 2.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(type("A", (), {"steps": 1, "gpus": 2})())
    assert buf.getvalue() == ""
