"""bench.py's multi-process path (one replica per GPU under torchrun): the
job's time is the slowest rank's, the rate counts every rank's keys, and the
reference arm runs on rank 0 alone.  Checked here with gloo ranks on the CPU
(world size 2), without a GPU."""
from __future__ import annotations

import importlib.util
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        secs = b.max_over_ranks(1.0 + 0.5 * rank, dist)      # rank r took 1 + r/2 s
        rate = b.whole_job_rate(world, 1000, secs)          # 1000 keys per rank
        q.put((rank, secs, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time; the rate counts both ranks' keys
    assert [g[1] for g in got] == [1.5, 1.5]
    assert all(abs(g[2] - 2000 / 1.5) < 1e-9 for g in got)


def test_single_process_helpers():
    b = _bench()
    assert b.max_over_ranks(3.25) == 3.25
    assert b.whole_job_rate(1, 10, 2.0) == 5.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    """Under torchrun only rank 0 runs and prints the reference line; another
    rank returns 0 at once (it would fail loudly if it touched the oracle
    with the arguments below)."""
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--cpu-sample", "-1"])
    a = b.parse()
    assert b.run_reference(a) == 0
    assert capsys.readouterr().out == ""
