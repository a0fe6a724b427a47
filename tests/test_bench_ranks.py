"""The bench's multi-rank path on CPU: two gloo ranks (world size 2), as torchrun
launches them. Solves are independent replicas (weak scaling, no data-path
collective): each rank times its own matrix, the job's time is the slowest rank's,
and the value counts every rank's solves. The reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        def max_over_ranks(v):
            t = torch.tensor([v], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())
        job_ms, value = bench.job_throughput(local_ms[rank], 30, world, max_over_ranks)
        out.put((rank, job_ms, value, bench.replica_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_rank_throughput_is_slowest_rank_and_all_units():
    world, port = 2, _free_port()
    local_ms = [240.0, 255.5]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, local_ms, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, job_ms, value, seed in res:
        assert job_ms == max(local_ms)
        assert value == pytest.approx(30 * world / (max(local_ms) / 1e3))
    assert len({seed for *_, seed in res}) == world  # independent replicas


def test_single_rank_needs_no_collective():
    job_ms, value = bench.job_throughput(100.0, 10, 1)
    assert (job_ms, value) == (100.0, 100.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(Args(), 64) == 0
    assert buf.getvalue() == ""
