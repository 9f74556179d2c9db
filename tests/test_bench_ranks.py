"""The multi-rank aggregation of bench.py on the CPU: two gloo ranks report
different step times; both must see the slower one, and the whole-job rate is
the units of all ranks over that time.  Under torchrun the reference arm runs
on rank 0 alone, and the other ranks return without work."""
from __future__ import annotations

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [3.0, 5.0][rank]
        ms_max = bench.max_over_ranks(ms, world, "cpu")
        e2e = bench.max_over_ranks([0.25, 0.125][rank], world, "cpu")
        dist.barrier()
        out.put((rank, ms_max, bench.whole_job_rate(1.0, world, ms_max / 1e3),
                 bench.whole_job_rate(1.0, world, e2e)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value, e2e in res:
        assert ms_max == 5.0
        assert value == pytest.approx(2 / 5e-3)       # 400 steps/s over both ranks
        assert e2e == pytest.approx(2 / 0.25)


def test_single_rank_is_the_identity():
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert bench.whole_job_rate(3.0, 1, 0.5) == 6.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    # rank 1 of 2 returns before it reads its arguments, does work or prints
    assert bench.run_reference(None, 1, 2) is None
    assert capsys.readouterr().out == ""
