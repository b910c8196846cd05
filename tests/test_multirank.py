"""The N > 1 path of bench.py on the CPU: two ranks on the gloo backend
(one process each, rendezvous on 127.0.0.1), each timing its own replica.
The job time is the slowest rank's, the job rate counts every rank's cells,
and the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench._dist()
        assert (ws, r, local) == (world, rank, rank)
        bench.barrier(ws)
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, ws, torch.device("cpu"))
        rate = bench.job_rate(1000, 4, ws, ms)
        out.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, rate in got:
        assert ms == pytest.approx(15.0)                   # the slowest rank's time on every rank
        assert rate == pytest.approx(1000 * 4 * 2 / 15e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(7.5, 1, None) == 7.5
    assert bench.job_rate(100, 10, 1, 1.0) == pytest.approx(1e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(None)          # rank 1: returns before any work, prints nothing
    assert capsys.readouterr().out == ""
